"""GPU parity of the batched form: every graph of a batch gives exactly the
result it gives alone and the oracle's (count, histogram, hash, search-tree
counters), whatever shapes the batch mixes."""
from __future__ import annotations

import os
import sys

import numpy as np
import pytest

import oracle
import synth

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))

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


def _check(got, n, uv, mode="greedy"):
    ref = oracle.tomita(n, uv)
    tree = oracle.ordered(n, uv, mode)
    assert got["status"] == 0
    assert (got["count"], got["hash"]) == (ref["count"], ref["hash"])
    assert np.array_equal(got["hist"], ref["hist"])
    assert (got["nodes"], got["internal"], got["dead_ends"]) == (tree["nodes"], tree["internal"], tree["dead_ends"])


def mixed_specs():
    specs = [(0, synth.empty(0)), (1, synth.empty(1)), (30, synth.gnp(30, 0.5, 1)), (45, synth.moon_moser(8)[:0]),
             (45, synth.moon_moser(15)[:600]), (64, synth.gnp(64, 0.6, 2)), (100, synth.gnp(100, 0.5, 0)),
             (129, synth.gnp(129, 0.3, 3)), (200, synth.gnp(200, 0.25, 4)), (256, synth.gnp(256, 0.2, 5)),
             (300, synth.gnp(300, 0.2, 6)), (512, synth.gnp(512, 0.1, 7)), (700, synth.gnp(700, 0.05, 8)),
             (1100, synth.gnp(1100, 0.02, 9)), (20, synth.complete(20)), (90, synth.cycle(90))]
    return specs


@pytest.mark.parametrize("mode", ["greedy", "tx", "tomita", "nx"])
def test_mixed_batch_matches_oracle(ctx, mce, mode):
    specs = mixed_specs()
    graphs = [ctx.load_edges(n, uv) for n, uv in specs]
    res = mce.enumerate_batch(ctx, graphs, mce.options(pivot=mode))
    for (n, uv), got in zip(specs, res):
        _check(got, n, uv, mode)
    for g in graphs:
        g.free()


@pytest.mark.parametrize("mode", ["greedy", "tx", "tomita", "nx"])
def test_heavy_graphs_split_into_root_child_parts(ctx, mce, mode):
    # two heavy graphs among light ones: the plan splits each heavy graph into
    # parts that search every k-th root child on different blocks (the dense
    # one has only a few root children, so few parts); the parts add up to
    # the oracle's result and the plan replays with the same result
    specs = [(150, synth.gnp(150, 0.5, 300)), (60, synth.gnp(60, 0.8, 301))] + \
            [(40, synth.gnp(40, 0.3, 310 + i)) for i in range(30)]
    graphs = [ctx.load_edges(n, uv) for n, uv in specs]
    b = mce.Batch(ctx, graphs, mce.options(pivot=mode))
    try:
        info = b.buckets()
        assert sum(x["split_graphs"] for x in info) == 2
        assert sum(x["work_items"] for x in info) > len(specs) + 2
        assert sum(x["graphs"] for x in info) == len(specs)
        first = b.run()
        for (n, uv), got in zip(specs, first):
            _check(got, n, uv, mode)
        again = b.run()
        assert [(r["count"], r["hash"], r["nodes"]) for r in again] == \
            [(r["count"], r["hash"], r["nodes"]) for r in first]
    finally:
        b.close()
        for g in graphs:
            g.free()


def test_batch_equals_alone_and_replays(ctx, mce):
    specs = [(int(n), synth.gnp(int(n), p, 100 + i)) for i, (n, p) in
             enumerate([(40, 0.7), (80, 0.5), (150, 0.4), (260, 0.3), (400, 0.2), (500, 0.15)] * 6)]
    graphs = [ctx.load_edges(n, uv) for n, uv in specs]
    alone = [g.enumerate() for g in graphs]
    b = mce.Batch(ctx, graphs)
    for _ in range(3):                      # the captured graph replays
        res = b.run()
        for a, r in zip(alone, res):
            assert (a["count"], a["hash"], a["nodes"]) == (r["count"], r["hash"], r["nodes"])
            assert np.array_equal(a["hist"], r["hist"])
    b.close()
    for g in graphs:
        g.free()


@pytest.mark.parametrize("kw", [dict(threads=32), dict(threads=512), dict(blocks=1, threads=64),
                                dict(lanes=32, words=1), dict(stack_levels=3, queue_log2=18)])
def test_batch_launch_shapes(ctx, mce, kw):
    sizes = (33, 70, 140) if "stack_levels" in kw else (33, 70, 140, 250, 400)
    specs = [(n, synth.gnp(n, 0.35, 200 + n)) for n in sizes]
    graphs = [ctx.load_edges(n, uv) for n, uv in specs]
    try:
        res = mce.enumerate_batch(ctx, graphs, mce.options(**kw))
        for (n, uv), got in zip(specs, res):
            _check(got, n, uv)
    finally:
        for g in graphs:
            g.free()


def test_batch_of_workload_graphs(ctx, mce):
    """A slice of the 4096-graph batched workload (capped G(n, p))."""
    specs = synth.batch_graphs(64)
    graphs = [ctx.load_edges(s.n, s.uv) for s in specs]
    res = mce.enumerate_batch(ctx, graphs)
    checked = 0
    for s, got in zip(specs, res):
        if synth.expected_maximal_cliques(s.n, s.p) > 2e5 or checked == 24:
            continue
        checked += 1
        ref = oracle.ordered(s.n, s.uv)
        assert (got["count"], got["hash"], got["nodes"]) == (ref["count"], ref["hash"], ref["nodes"])
    for g in graphs:
        g.free()


def test_autotuned_batch_matches_oracle_and_reuses_choices(ctx, mce):
    # 48 graphs of each words class 1, 2, 4 and 8 (n = 20..256), G(n, 0.3)
    specs = [(n, synth.gnp(n, 0.3, 300 + i)) for i, n in
             enumerate([20 + (i % 12) for i in range(48)] + [40 + (i % 24) for i in range(48)] +
                       [70 + (i % 58) for i in range(48)] + [130 + (i % 126) for i in range(48)])]
    graphs = [ctx.load_edges(n, uv) for n, uv in specs]
    b = mce.Batch(ctx, graphs, mce.options(autotune=True))
    res = b.run()
    for (n, uv), r in list(zip(specs, res))[::7]:
        _check(r, n, uv)
    alone = [g.enumerate() for g in graphs]
    assert [(r["count"], r["hash"], r["nodes"]) for r in res] == [(a["count"], a["hash"], a["nodes"]) for a in alone]
    buckets = b.buckets()
    assert sum(x["graphs"] for x in buckets) == len(graphs)
    assert all(x["tuned"] == 1 for x in buckets)
    for x in buckets:
        assert x["lanes_per_subtree"] * x["words_per_lane"] >= x["words_class"]
        assert x["threads_per_block"] in (128, 256, 512) and x["tuned_ms_per_graph"] > 0
    # a second batch of the same classes takes the cached choices
    b2 = mce.Batch(ctx, graphs[::2], mce.options(autotune=True))
    assert {(x["lanes_per_subtree"], x["words_per_lane"], x["threads_per_block"], x["split_min_p"])
            for x in b2.buckets()} <= {(x["lanes_per_subtree"], x["words_per_lane"], x["threads_per_block"],
                                        x["split_min_p"]) for x in buckets}
    r2 = b2.run()
    assert [(r["count"], r["hash"]) for r in r2] == [(a["count"], a["hash"]) for a in alone[::2]]
    b.close()
    b2.close()
    for g in graphs:
        g.free()


def _gen_batch_rows(i):
    g = synth.batch_graph(i)
    return g.n, synth.to_bitset(g.n, g.uv)


def test_whole_batched_workload_matches_oracle(ctx, mce):
    """All 4096 graphs of the batched workload (capped G(n, p), n in
    [32, 512]) in one captured launch, each against the oracle's stored
    count, hash, histogram and GreedyBB tree
    (tests/golden/batch4096_results.txt)."""
    import multiprocessing as mp
    import make_workload_golden as mk
    gold = mk.load("batch")
    assert len(gold) == 4096
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        specs = pool.map(_gen_batch_rows, range(4096), chunksize=32)
    graphs = [ctx.load_bitset(n, rows) for n, rows in specs]
    b = mce.Batch(ctx, graphs)
    res = b.run()
    bad = []
    for g, r in zip(gold, res):
        hist = {k: int(v) for k, v in enumerate(r["hist"]) if v}
        if (r["status"], r["count"], r["hash"], r["nodes"], r["internal"], r["dead_ends"], hist) != \
                (0, g["count"], g["hash"], g["nodes"], g["internal"], g["dead_ends"], g["hist"]):
            bad.append(g["index"])
    b.close()
    for g in graphs:
        g.free()
    assert not bad, bad[:20]
