"""GPU parity of Alg. 3's outer loop (MCE_OUTER, and every graph with more
than MCE_NMAX vertices): results equal Alg. 2's, and the search-tree counters
equal the oracle's outer loop node for node (same degeneracy order, same
subproblems, same ordered search inside)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


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


def outer_on_gpu(ctx, mce, n, uv, **kw):
    g = ctx.load_edges(n, uv)
    try:
        return g.enumerate(mce.options(outer=True, **kw))
    finally:
        g.free()


def expect_outer(got, n, uv, mode="greedy", what=""):
    ref = oracle.tomita(n, uv)
    tree = oracle.outer(n, uv, mode)
    assert (got["count"], got["hash"]) == (ref["count"], ref["hash"]), what
    assert np.array_equal(np.asarray(got["hist"], dtype=np.uint64), ref["hist"]), what
    assert (got["nodes"], got["internal"], got["dead_ends"]) == \
        (tree["nodes"], tree["internal"], tree["dead_ends"]), what


@pytest.mark.parametrize("n,p,seed", [(1, 0.5, 0), (2, 1.0, 0), (7, 0.5, 1), (40, 0.3, 2), (100, 0.1, 3),
                                      (300, 0.05, 4), (600, 0.02, 5), (200, 0.4, 6)])
def test_outer_small_graphs(ctx, mce, n, p, seed):
    uv = synth.gnp(n, p, seed)
    expect_outer(outer_on_gpu(ctx, mce, n, uv), n, uv, what=f"G({n},{p})")


@pytest.mark.parametrize("mode", ["tx", "tomita", "nx"])
def test_outer_pivot_rules(ctx, mce, mode):
    n, uv = 250, synth.gnp(250, 0.1, 7)
    expect_outer(outer_on_gpu(ctx, mce, n, uv, pivot=mode), n, uv, mode=mode, what=mode)


def test_outer_structured(ctx, mce):
    for n, uv in [(30, synth.complete(30)), (50, synth.empty(50)), (45, synth.moon_moser(15)),
                  (12, synth.complete_multipartite([3, 4, 5])), (20, synth.cycle(20))]:
        expect_outer(outer_on_gpu(ctx, mce, n, uv), n, uv, what=str(n))


@pytest.mark.parametrize("n,p,seed", [(5000, 0.01, 1), (10000, 0.001, 0), (10000, 0.003, 2), (8000, 0.002, 3)])
def test_sparse_graphs_beyond_the_bitset_path(ctx, mce, n, p, seed):
    uv = synth.gnp(n, p, seed)
    g = ctx.load_edges(n, uv)
    try:
        got = g.enumerate()                      # n > MCE_NMAX: the outer loop
    finally:
        g.free()
    expect_outer(got, n, uv, what=f"G({n},{p})")


def test_outer_with_offsets_beyond_shared_memory(ctx, mce):
    """n = 60,000 as 15,000 disjoint K4: too many vertices for the
    degeneracy kernel to stage the offsets in shared memory beside the
    degrees, so it reads them from global memory.  The order finishes one K4
    before the next (the others keep degree 3 while the current one's drop),
    every component runs the same subproblems, so the counters are 15,000
    times those of one K4 in the oracle, and the hash is the sum of the
    15,000 clique hashes."""
    k = 15000
    one = oracle.outer(4, synth.complete(4))
    pairs = np.array([(a, b) for a in range(4) for b in range(a + 1, 4)], dtype=np.uint32)
    uv = ((np.arange(k, dtype=np.uint32) * 4)[:, None, None] + pairs[None, :, :]).reshape(-1, 2)
    g = ctx.load_edges(4 * k, uv)
    try:
        got = g.enumerate()
    finally:
        g.free()
    assert got["count"] == k * one["count"] == k
    assert (got["nodes"], got["internal"], got["dead_ends"]) == \
        (k * one["nodes"], k * one["internal"], k * one["dead_ends"])
    h = 0
    for c in range(k):
        h = (h + oracle.clique_hash(np.arange(4 * c, 4 * c + 4))) & ((1 << 64) - 1)
    assert got["hash"] == h
    assert int(got["hist"][4]) == k and int(got["hist"].sum()) == k


def test_sparse_limits(ctx, mce):
    # a vertex of degree >= MCE_NMAX has a subproblem beyond the bitset path
    n = 5000
    star = np.array([[0, v] for v in range(1, n)], dtype=np.uint32)
    g = ctx.load_edges(n, star)
    try:
        assert g.enumerate(raise_on_error=False)["rc"] == mce.MCE_ENOTIMPL
        # listing is not offered on the outer loop
        assert g.enumerate(mce.options(flags=mce.MCE_LIST), raise_on_error=False, list_cap=10,
                           off_cap=10)["rc"] == mce.MCE_ENOTIMPL
    finally:
        g.free()
    with pytest.raises(mce.MceError):
        ctx.load_edges(mce.MCE_NMAX_SPARSE + 1, np.zeros((0, 2), np.uint32))
    with pytest.raises(mce.MceError):                  # self-loop
        ctx.load_edges(6000, np.array([[7, 7]], dtype=np.uint32))
    with pytest.raises(mce.MceError):                  # id >= n
        ctx.load_edges(6000, np.array([[1, 6000]], dtype=np.uint32))
    big = ctx.load_edges(6000, synth.gnp(6000, 0.001, 1))
    try:
        with pytest.raises(mce.MceError):              # no bitset: not for batches or serving
            mce.Batch(ctx, [big])
        with pytest.raises(mce.MceError):
            ctx.submit(big)
    finally:
        big.free()


def test_sparse_duplicate_edges_and_both_orientations(ctx, mce):
    n = 4500
    uv = synth.gnp(n, 0.002, 9)
    doubled = np.concatenate([uv, uv[:, ::-1], uv[:100]])
    g = ctx.load_edges(n, doubled)
    try:
        got = g.enumerate()
    finally:
        g.free()
    expect_outer(got, n, uv)
