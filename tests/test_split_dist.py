"""Host logic of the multi-GPU split (paper_1801_00202_gb300/split.py) on CPU:
the partition of the root's children, the modulo-2^64 result vector, and a
world-size-2 gloo run in which each rank searches its share of the root's
children with the CPU oracle standing in for the GPU and one all-reduce
gives every rank the whole graph's result."""
from __future__ import annotations

import os
import socket
import sys

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _split():
    sys.path.insert(0, ROOT)
    import importlib
    return importlib.import_module("paper_1801_00202_gb300.split")


class OracleGraph:
    """The two calls enumerate_sharded needs, answered by the CPU oracle."""

    def __init__(self, n, uv, mode):
        self.n, self.uv, self.mode = n, uv, mode

    def root_children(self, opts=None):
        return oracle.root_children(self.n, self.uv, self.mode)

    def enumerate_part(self, children, count_root, opts=None):
        r = oracle.ordered_part(self.n, self.uv, self.mode, children, count_root)
        r["max_size"] = max((k for k, v in enumerate(r["hist"]) if v), default=0)
        return r


def test_partition_covers_every_child_once():
    split = _split()
    rng = np.random.default_rng(7)
    for parts in (1, 2, 3, 8):
        sizes = rng.integers(0, 500, size=101)
        p = split.partition(sizes, parts)
        assert len(p) == parts
        flat = sorted(t for x in p for t in x)
        assert flat == list(range(101))
        assert all(x == sorted(x) for x in p)
        loads = [int(sizes[x].sum()) if x else 0 for x in p]
        assert max(loads) - min(loads) <= int(sizes.max())   # boustrophedon deal: within one child
    assert split.partition([5, 9, 1, 7], 2) == [[1, 2], [0, 3]]  # 9 -> 0, 7 -> 1, 5 -> 1, 1 -> 0


def test_result_vector_wraps_modulo_2_64():
    split = _split()
    a = {"count": 3, "nodes": 2 ** 64 - 1, "internal": 1, "dead_ends": 0, "hash": 2 ** 63 + 5,
         "hist": np.array([0, 1, 2], dtype=np.uint64), "max_size": 2}
    b = {"count": 4, "nodes": 2, "internal": 1, "dead_ends": 7, "hash": 2 ** 63 + 9,
         "hist": np.array([0, 0, 2], dtype=np.uint64), "max_size": 1}
    s = split.pack(a, 2) + split.pack(b, 2)           # int64 addition wraps like uint64
    u = split.unpack(s, 2, 2)
    assert (u["count"], u["nodes"], u["internal"], u["dead_ends"]) == (7, 1, 2, 7)
    assert u["hash"] == (2 ** 63 + 5 + 2 ** 63 + 9) % 2 ** 64
    assert u["hist"].tolist() == [0, 1, 4]


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


CASES = [(60, 0.5, 910, "greedy"), (45, 0.9, 911, "tomita"), (80, 0.3, 912, "tx")]


def _rank(rank: int, world: int, port: int, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    split = _split()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = []
        for n, p, seed, mode in CASES:
            g = OracleGraph(n, synth.gnp(n, p, seed), mode)
            r = split.enumerate_sharded(g, dist=dist)
            out.append({k: (v.tolist() if isinstance(v, np.ndarray) else v) for k, v in r.items()})
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_sharded_search_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for i, (n, p, seed, mode) in enumerate(CASES):
        uv = synth.gnp(n, p, seed)
        whole = oracle.ordered(n, uv, mode)
        ref = oracle.tomita(n, uv)
        parts = [got[r][i]["part"] for r in range(2)]
        assert sum(x["children"] for x in parts) == parts[0]["of"]
        assert 0 < parts[0]["count"] < whole["count"]    # both ranks did real work
        for r in range(2):                                 # every rank holds the whole result
            res = got[r][i]
            assert (res["count"], res["hash"]) == (ref["count"], ref["hash"])
            assert (res["nodes"], res["internal"], res["dead_ends"]) == \
                (whole["nodes"], whole["internal"], whole["dead_ends"])
            assert res["hist"] == ref["hist"].tolist()
            assert res["max_size"] == max(k for k, v in enumerate(ref["hist"]) if v)
