"""GPU parity of the root-children split (mce_root_children,
mce_enumerate_part), on one GPU: the children's candidate-set sizes equal the
oracle's, and the parts of any partition of the root's children, searched one
after another, add up exactly to the whole search and to the oracle (count,
hash, histogram, nodes, internal, dead ends)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
MASK = (1 << 64) - 1


@pytest.fixture(scope="module")
def mce():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_00202_gb300 as m
    m.build()
    m.lib()
    return m


@pytest.fixture(scope="module")
def ctx(mce):
    c = mce.Context(0)
    yield c
    c.close()


def _sum(parts, n):
    out = {"count": 0, "nodes": 0, "internal": 0, "dead_ends": 0, "hash": 0,
           "hist": np.zeros(n + 1, dtype=np.uint64)}
    for r in parts:
        for k in ("count", "nodes", "internal", "dead_ends", "hash"):
            out[k] = (out[k] + r[k]) & MASK
        out["hist"] = out["hist"] + r["hist"]
    return out


CASES = [(1, 0.5, 920, "greedy"), (90, 0.5, 921, "greedy"), (300, 0.3, 922, "tomita"), (45, 0.9, 923, "tx"),
         (700, 0.1, 924, "nx"), (1500, 0.05, 925, "greedy"), (4096, 0.01, 926, "tomita")]


@pytest.mark.parametrize("n,p,seed,mode", CASES)
@pytest.mark.parametrize("parts", [1, 2, 3, 8])
def test_parts_add_up_to_the_whole(ctx, mce, n, p, seed, mode, parts):
    from paper_1801_00202_gb300 import split
    uv = synth.gnp(n, p, seed)
    g = ctx.load_edges(n, uv)
    o = mce.options(pivot=mode)
    try:
        sizes = g.root_children(o)
        assert sizes.tolist() == oracle.root_children(n, uv, mode).tolist()
        got = [g.enumerate_part(ch, r == 0, o) for r, ch in enumerate(split.partition(sizes, parts))]
        whole = g.enumerate(o)
    finally:
        g.free()
    tot = _sum(got, n)
    ref = oracle.tomita(n, uv)
    tree = oracle.ordered(n, uv, mode)
    assert (tot["count"], tot["hash"]) == (ref["count"], ref["hash"])
    assert np.array_equal(tot["hist"], ref["hist"])
    assert (tot["nodes"], tot["internal"], tot["dead_ends"]) == (tree["nodes"], tree["internal"], tree["dead_ends"])
    assert (whole["count"], whole["hash"], whole["nodes"]) == (tot["count"], tot["hash"], tot["nodes"])


def test_single_children_match_the_oracle(ctx, mce):
    # Moon-Moser on 30 vertices branches on one triangle: three equal children
    # of 3^9 cliques each; a 5%-deleted variant gives uneven children
    for n, uv in ((30, synth.moon_moser(10)), (45, synth.moon_moser_deleted(15, 0.05, 3))):
        g = ctx.load_edges(n, uv)
        try:
            k = len(g.root_children())
            for t in range(k):
                r = g.enumerate_part([t], t == 0)
                want = oracle.ordered_part(n, uv, "greedy", [t], t == 0)
                assert (r["count"], r["hash"], r["nodes"], r["internal"], r["dead_ends"]) == \
                    (want["count"], want["hash"], want["nodes"], want["internal"], want["dead_ends"])
                assert np.array_equal(r["hist"], want["hist"])
        finally:
            g.free()
    r = ctx.load_edges(30, synth.moon_moser(10))
    assert r.root_children().tolist() == [27, 27, 27]
    r.free()


def test_bad_child_lists_are_rejected(ctx, mce):
    n, uv = 50, synth.gnp(50, 0.4, 927)
    g = ctx.load_edges(n, uv)
    try:
        k = len(g.root_children())
        assert g.enumerate_part([1, 0], True, raise_on_error=False)["rc"] == mce.MCE_EINVAL   # not increasing
        assert g.enumerate_part([k], True, raise_on_error=False)["rc"] == mce.MCE_EINVAL      # beyond |L|
        assert g.enumerate_part([0], True)["rc"] == 0                                        # context still fine
        empty = g.enumerate_part([], True)                                                   # the root alone
        assert (empty["nodes"], empty["internal"], empty["count"]) == (1, 1, 0)
    finally:
        g.free()
