"""Clique listing (MCE_LIST / MCE_LIST_SORTED) through mce_enumerate.

Small and mid-size graphs: the GPU listing equals the oracle's listing
(Alg. 2 with the Tomita pivot; each clique ascending, cliques in
lexicographic order) exactly, under every pivot rule and under launch shapes
that force frames (and with them R) through every hand-over path: block
ring, global ring, breadth-first split, stack spill.  Full-size workloads:
the Moon-Moser listing against its closed form (one vertex from each
triangle, in lexicographic order), and G(1000, 0.3) against the stored
oracle count, histogram and hash plus per-clique checks on a sample.
"""
from __future__ import annotations

import json
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


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


def listed(ctx, mce, n, uv, sort=True, **kw):
    g = ctx.load_edges(n, uv)
    try:
        flags = mce.MCE_LIST | (mce.MCE_LIST_SORTED if sort else 0)
        return g.enumerate(mce.options(flags=flags, **kw))
    finally:
        g.free()


def as_tuples(res, mce):
    return [tuple(int(x) for x in c) for c in mce.cliques(res)]


def check_against_oracle(res, mce, n, uv, sort=True, what=""):
    ref = oracle.tomita(n, uv, listing=True)
    got = as_tuples(res, mce)
    assert res["count"] == ref["count"] == len(got), what
    assert res["hash"] == ref["hash"], what
    assert all(list(c) == sorted(c) for c in got), what
    if sort:
        assert got == ref["listing"], what
    else:
        assert sorted(got) == ref["listing"], what


# --- exact listings on small and mid-size graphs -----------------------------

@pytest.mark.parametrize("n,p,seed", [(1, 0.5, 0), (2, 1.0, 0), (5, 0.5, 1), (31, 0.5, 2), (32, 0.4, 3),
                                      (33, 0.6, 4), (64, 0.5, 5), (65, 0.3, 6), (100, 0.5, 0), (150, 0.55, 7),
                                      (257, 0.3, 8), (400, 0.25, 9), (1100, 0.05, 10)])
def test_sorted_listing_equals_oracle(ctx, mce, n, p, seed):
    uv = synth.gnp(n, p, seed)
    check_against_oracle(listed(ctx, mce, n, uv), mce, n, uv, what=f"G({n},{p}) seed {seed}")


@pytest.mark.parametrize("pivot", ["greedy", "tx", "tomita"])
def test_listing_every_pivot_rule(ctx, mce, pivot):
    n, uv = 140, synth.gnp(140, 0.5, 11)
    check_against_oracle(listed(ctx, mce, n, uv, pivot=pivot), mce, n, uv, what=pivot)


def test_unsorted_listing_is_the_same_set(ctx, mce):
    n, uv = 180, synth.gnp(180, 0.45, 12)
    res = listed(ctx, mce, n, uv, sort=False)
    check_against_oracle(res, mce, n, uv, sort=False)


@pytest.mark.parametrize("kw", [dict(blocks=1, threads=32), dict(blocks=2, threads=64, split_min_p=1),
                                dict(stack_levels=3, queue_log2=20), dict(stack_levels=2, split_min_p=2),
                                dict(lanes=32, words=1), dict(lanes=1, words=4, threads=64),
                                dict(lanes=2, words=2, blocks=3)])
def test_listing_through_every_hand_over(ctx, mce, kw):
    n, uv = 110, synth.gnp(110, 0.55, 13)
    check_against_oracle(listed(ctx, mce, n, uv, **kw), mce, n, uv, what=str(kw))


def test_listing_identity_order(ctx, mce):
    n, uv = 20, synth.gnp(20, 0.5, 14)
    check_against_oracle(listed(ctx, mce, n, uv, identity_order=True), mce, n, uv)


def test_listing_degenerate_graphs(ctx, mce):
    # n = 0: the empty set is the one maximal clique
    res = listed(ctx, mce, 0, np.zeros((0, 2), np.uint32))
    assert res["count"] == 1 and list(res["list_off"]) == [0, 0] and res["list_ids"].size == 0
    # empty graph on 70 vertices: every vertex alone
    res = listed(ctx, mce, 70, synth.empty(70))
    assert as_tuples(res, mce) == [(v,) for v in range(70)]
    # complete graph: one clique of every vertex
    res = listed(ctx, mce, 300, synth.complete(300))
    assert as_tuples(res, mce) == [tuple(range(300))]
    # complete multipartite K_{3,4,5}: one vertex from each part
    uv = synth.complete_multipartite([3, 4, 5])
    res = listed(ctx, mce, 12, uv)
    assert as_tuples(res, mce) == [(a, b, c) for a in range(3) for b in range(3, 7) for c in range(7, 12)]


def test_listing_truncation_reports_sizes(ctx, mce):
    n, uv = 90, synth.gnp(90, 0.5, 15)
    ref = oracle.tomita(n, uv)
    g = ctx.load_edges(n, uv)
    try:
        opts = mce.options(flags=mce.MCE_LIST_SORTED)
        short = g.enumerate(opts, raise_on_error=False, list_cap=10, off_cap=5)
        assert short["rc"] == mce.MCE_ETRUNC
        assert short["count"] == ref["count"] and short["hash"] == ref["hash"]
        need = int(sum(k * int(c) for k, c in enumerate(ref["hist"])))
        assert short["list_ids_needed"] == need
        full = g.enumerate(opts, list_cap=need, off_cap=ref["count"] + 1)
        assert full["rc"] == 0 and int(full["list_off"][-1]) == need
    finally:
        g.free()


def test_listing_rejected_where_not_supported(ctx, mce):
    import torch
    n, uv = 40, synth.gnp(40, 0.5, 16)
    opts = mce.options(flags=mce.MCE_LIST)
    with pytest.raises(mce.MceError):
        mce.mce_scratch_bytes(n, opts)
    out = torch.zeros(mce.MCE_OUT_WORDS(n), dtype=torch.int64, device="cuda")
    rows = torch.from_numpy(synth.to_bitset(n, uv).view(np.int32).reshape(-1)).cuda()
    scratch = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    rc = mce.mce_enumerate_device(n, synth.words_per_row(n), rows, opts, scratch, scratch.numel(), out)
    assert rc == mce.MCE_ENOTIMPL


# --- full-size workloads -------------------------------------------------------

def test_moon_moser_45_listing_closed_form(ctx, mce):
    k = 15
    res = listed(ctx, mce, 3 * k, synth.moon_moser(k))
    assert res["count"] == 3 ** k
    ids = res["list_ids"].reshape(-1, k).astype(np.int64)
    assert np.array_equal(res["list_off"], np.arange(3 ** k + 1, dtype=np.uint64) * k)
    # clique j picks vertex 3i + (digit i of j in base 3, most significant first)
    j = np.arange(3 ** k, dtype=np.int64)
    for i in range(k):
        digit = (j // 3 ** (k - 1 - i)) % 3
        assert np.array_equal(ids[:, i], 3 * i + digit), i


_M1, _M2 = np.uint64(0xBF58476D1CE4E5B9), np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    # SplitMix64 finaliser (Steele, Lea, Flood, OOPSLA 2014), vectorised, to
    # recompute the clique hash of a whole listing
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def test_gnp_1000_listing_against_stored_oracle(ctx, mce):
    gold = json.load(open(os.path.join(GOLDEN, "config_results.json")))["gnp_1000_0.3_s1"]
    n, uv = 1000, synth.gnp(1000, 0.3, 1)
    res = listed(ctx, mce, n, uv, sort=False)
    off, ids = res["list_off"].astype(np.int64), res["list_ids"]
    sizes = np.diff(off)
    assert res["count"] == gold["count"] == sizes.size
    hist = np.zeros(n + 1, dtype=np.int64)
    for k, c in gold["hist"].items():
        hist[int(k)] = c
    assert np.array_equal(np.bincount(sizes, minlength=n + 1), hist)
    with np.errstate(over="ignore"):
        terms = _mix64(ids.astype(np.uint64) + np.uint64(1))
        S = np.add.reduceat(terms, off[:-1])
        h = _mix64(S ^ _mix64(sizes.astype(np.uint64)))
        assert int(h.sum(dtype=np.uint64)) == gold["hash"]
    # ascending members, and a sample of cliques checked for maximality
    starts = off[:-1]
    inner = np.ones(ids.size, dtype=bool)
    inner[starts] = False
    assert np.all(np.diff(ids.astype(np.int64))[inner[1:]] > 0)
    adj = np.zeros((n, n), dtype=bool)
    adj[uv[:, 0], uv[:, 1]] = adj[uv[:, 1], uv[:, 0]] = True
    rng = np.random.default_rng(0)
    for c in rng.choice(sizes.size, 2000, replace=False):
        K = ids[off[c]:off[c + 1]]
        sub = adj[np.ix_(K, K)]
        assert sub.sum() == K.size * (K.size - 1)
        common = adj[K].all(axis=0)
        common[K] = False
        assert not common.any()


# --- streaming listing (mce_enumerate_stream): no buffers sized up front ------

def _mix64_np(z):
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(0xBF58476D1CE4E5B9)
        z ^= z >> np.uint64(27)
        z *= np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return z


def _stream_summary(chunks, n):
    """count, histogram and clique hash of streamed (ids, off) chunks,
    vectorised: S(K) = sum of mix64(label + 1), h(K) = mix64(S ^ mix64(|K|))."""
    count, hist, h = 0, np.zeros(n + 1, dtype=np.uint64), np.uint64(0)
    for ids, off in chunks:
        k = np.diff(off).astype(np.int64)
        count += k.size
        np.add.at(hist, k, 1)
        terms = _mix64_np(ids.astype(np.uint64) + np.uint64(1))
        with np.errstate(over="ignore"):
            s = np.add.reduceat(terms, off[:-1].astype(np.int64)) if ids.size else np.zeros(k.size, np.uint64)
            s[k == 0] = 0
            h = h + np.sum(_mix64_np(s ^ _mix64_np(k.astype(np.uint64))), dtype=np.uint64)
    return count, hist, int(h)


@pytest.mark.parametrize("sort", [True, False])
@pytest.mark.parametrize("n,p,seed", [(0, 0.0, 0), (1, 0.0, 0), (60, 0.5, 30), (300, 0.4, 31), (1100, 0.05, 32)])
def test_streamed_listing_equals_oracle(ctx, mce, sort, n, p, seed):
    uv = synth.gnp(n, p, seed) if n > 1 else synth.empty(n)
    g = ctx.load_edges(n, uv)
    got = []
    try:
        flags = mce.MCE_LIST_SORTED if sort else mce.MCE_LIST
        res = g.enumerate_stream(lambda ids, off, k: got.extend(
            tuple(int(x) for x in ids[off[i]:off[i + 1]]) for i in range(k)), mce.options(flags=flags))
    finally:
        g.free()
    ref = oracle.tomita(n, uv, listing=True)
    want = ref["listing"]
    assert (res["count"], res["hash"]) == (ref["count"], ref["hash"])
    assert (got if sort else sorted(got)) == want


def test_streamed_listing_full_size_and_early_stop(ctx, mce):
    gold = json.load(open(os.path.join(GOLDEN, "config_results.json")))["gnp_1000_0.3_s1"]
    n, uv = 1000, synth.gnp(1000, 0.3, 1)
    g = ctx.load_edges(n, uv)
    chunks = []
    try:
        res = g.enumerate_stream(lambda ids, off, k: chunks.append((ids, off)))
        count, hist, h = _stream_summary(chunks, n)
        assert count == res["count"] == gold["count"]
        assert h == gold["hash"] == res["hash"]
        assert {str(k): int(v) for k, v in enumerate(hist) if v} == gold["hist"]
        assert len(chunks) > 1                                   # 15.4 M cliques come in several chunks
        seen = []
        res2 = g.enumerate_stream(lambda ids, off, k: seen.append(k) or True)   # stop after the first chunk
        assert res2["rc"] == 0 and len(seen) == 1
    finally:
        g.free()
