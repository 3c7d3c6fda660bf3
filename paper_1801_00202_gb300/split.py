"""One search split over several GPUs (one process per GPU).

The root's children of Alg. 4 are independent subtrees (the decomposition
Alg. 3 makes over vertices, Section 3.3): child t branches on the t-th
vertex of the root's branching set with the earlier ones already in X, and
reports exactly the maximal cliques that contain it and none of them.  So
every rank

  1. asks its own copy of the graph for the children's candidate-set sizes
     (``Graph.root_children``, identical on every rank: no exchange),
  2. takes its share of a partition of the children (``part_of``: largest
     first, dealt out in boustrophedon order 0, 1, .., N-1, N-1, .., 0 so
     that estimated work evens out),
  3. searches it (``Graph.enumerate_part``; rank 0 also counts the root),
  4. and one sum all-reduce of the result vector (count, nodes, internal,
     dead ends, hash, histogram; all modulo 2^64) plus a max all-reduce of
     the largest clique size gives every rank the whole graph's result.

Only the host logic lives here; the search runs in the CUDA kernels of
``libmce.so``.  ``torch.distributed`` carries the reduction (NCCL between
GPUs, gloo on CPU in the tests).
"""
from __future__ import annotations

import numpy as np

_MASK = (1 << 64) - 1
FIELDS = ("count", "nodes", "internal", "dead_ends", "hash")


def partition(sizes, parts: int) -> list:
    """Children 0..len(sizes)-1 split into ``parts`` lists (each ascending):
    by decreasing estimated size (ties: lower index first), dealt out in
    boustrophedon order."""
    sizes = np.asarray(sizes, dtype=np.int64).reshape(-1)
    order = sorted(range(sizes.size), key=lambda t: (-int(sizes[t]), t))
    out = [[] for _ in range(parts)]
    for i, t in enumerate(order):
        r, lap = i % parts, (i // parts) % 2
        out[r if lap == 0 else parts - 1 - r].append(t)
    return [sorted(x) for x in out]


def part_of(sizes, rank: int, world: int) -> list:
    return partition(sizes, world)[rank]


def pack(res: dict, n: int) -> np.ndarray:
    """Result dict -> int64 vector [count, nodes, internal, dead_ends, hash,
    hist[0..n]] (unsigned values reinterpreted, so sums wrap modulo 2^64)."""
    v = np.zeros(len(FIELDS) + n + 1, dtype=np.uint64)
    for i, f in enumerate(FIELDS):
        v[i] = np.uint64(int(res[f]) & _MASK)
    v[len(FIELDS):] = np.asarray(res["hist"], dtype=np.uint64)[:n + 1]
    return v.view(np.int64)


def unpack(vec: np.ndarray, n: int, max_size: int) -> dict:
    u = np.asarray(vec, dtype=np.int64).view(np.uint64)
    out = {f: int(u[i]) for i, f in enumerate(FIELDS)}
    out["hist"] = u[len(FIELDS):len(FIELDS) + n + 1].copy()
    out["max_size"] = int(max_size)
    return out


def all_reduce_result(res: dict, n: int, dist=None, device=None) -> dict:
    """Sum (modulo 2^64) of every rank's part and the largest clique size."""
    if dist is None:
        return unpack(pack(res, n), n, res.get("max_size", 0))
    import torch
    t = torch.from_numpy(pack(res, n)).to(device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    m = torch.tensor([int(res.get("max_size", 0))], dtype=torch.int64, device=t.device)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return unpack(t.cpu().numpy(), n, int(m.item()))


def enumerate_sharded(graph, opts=None, dist=None, device=None) -> dict:
    """The whole graph's result from this rank's share of the root's
    children.  ``graph`` offers root_children(opts) and
    enumerate_part(children, count_root, opts) (a ``Graph``)."""
    rank = dist.get_rank() if dist is not None else 0
    world = dist.get_world_size() if dist is not None else 1
    sizes = graph.root_children(opts)
    mine = part_of(sizes, rank, world)
    r = graph.enumerate_part(mine, rank == 0, opts)
    out = all_reduce_result(r, graph.n, dist, device)
    out["part"] = {"children": len(mine), "of": int(len(sizes)), "count": int(r["count"]),
                   "nodes": int(r["nodes"]), "kernel_ms": r.get("kernel_ms")}
    return out
