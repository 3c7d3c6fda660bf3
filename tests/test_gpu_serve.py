"""GPU parity of the served form (continuous batching): requests submitted
while others run give exactly their alone results and the oracle's."""
from __future__ import annotations

import os
import sys
import time

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


def test_mix_equals_alone(mce):
    ctx = mce.Context(0)
    specs = [(n, synth.gnp(n, p, 300 + i)) for i, (n, p) in
             enumerate([(64, 0.6), (100, 0.5), (300, 0.25), (700, 0.1), (1500, 0.03), (2048, 0.02),
                        (45, 0.9), (128, 0.4), (900, 0.08), (200, 0.35)] * 4)]
    graphs = [ctx.load_edges(n, uv) for n, uv in specs]
    alone = [g.enumerate() for g in graphs]
    tickets = []
    for g in graphs:                         # arrive while earlier ones run
        tickets.append(ctx.submit(g))
        time.sleep(0.0005)
    got = [None] * len(tickets)
    deadline = time.time() + 120
    while any(x is None for x in got) and time.time() < deadline:
        for i, t in enumerate(tickets):
            if got[i] is None:
                got[i] = ctx.poll(t)
        time.sleep(0.001)
    for (n, uv), a, r in zip(specs, alone, got):
        assert r is not None and r["rc"] == 0
        assert (r["count"], r["hash"], r["nodes"], r["internal"], r["dead_ends"]) == \
            (a["count"], a["hash"], a["nodes"], a["internal"], a["dead_ends"])
        assert np.array_equal(r["hist"], a["hist"])
    for (n, uv), r in list(zip(specs, got))[:10]:
        ref = oracle.tomita(n, uv)
        assert (r["count"], r["hash"]) == (ref["count"], ref["hash"])
    for g in graphs:
        g.free()
    ctx.close()


def test_wait_and_small_budget(mce):
    # a budget that admits only a few requests at a time still serves all
    ctx = mce.Context(0, mem_budget=256 << 20)
    specs = [(n, synth.gnp(n, 0.3, 400 + n)) for n in (80, 160, 320, 640, 1000, 80, 160, 320)]
    graphs = [ctx.load_edges(n, uv) for n, uv in specs]
    tickets = [ctx.submit(g) for g in graphs]
    for (n, uv), t in zip(specs, tickets):
        r = ctx.wait(t, timeout_ns=60_000_000_000)
        ref = oracle.ordered(n, uv)
        assert r["rc"] == 0 and (r["count"], r["hash"], r["nodes"]) == (ref["count"], ref["hash"], ref["nodes"])
    for g in graphs:
        g.free()
    ctx.close()


@pytest.mark.parametrize("pivot", ["greedy", "tomita"])
def test_queued_requests_share_launches(mce, pivot):
    # many small requests submitted at once queue up and run as batched
    # launches (the scheduler's micro-batches); each result is its own
    ctx = mce.Context(0)
    specs = [(n, synth.gnp(n, p, 500 + i)) for i, (n, p) in
             enumerate([(40, 0.5), (90, 0.4), (150, 0.3), (33, 0.7), (250, 0.15), (64, 0.5)] * 12)]
    graphs = [ctx.load_edges(n, uv) for n, uv in specs]
    opts = mce.options(pivot=pivot)
    alone = [g.enumerate(opts) for g in graphs]
    tickets = [ctx.submit(g, None if pivot == "greedy" else opts) for g in graphs]
    got = [ctx.wait(t, timeout_ns=60_000_000_000) for t in tickets]
    for a, r in zip(alone, got):
        assert r["rc"] == 0
        assert (r["count"], r["hash"], r["nodes"], r["internal"], r["dead_ends"]) == \
            (a["count"], a["hash"], a["nodes"], a["internal"], a["dead_ends"])
        assert np.array_equal(r["hist"], a["hist"])
    for (n, uv), r in list(zip(specs, got))[:6]:
        ref = oracle.tomita(n, uv)
        assert (r["count"], r["hash"]) == (ref["count"], ref["hash"])
    for g in graphs:
        g.free()
    ctx.close()


def _gen_served_rows(r):
    g = synth.served_graph(r)
    return g.n, synth.to_bitset(g.n, g.uv)


def test_served_workload_matches_oracle(mce):
    """The first 2000 requests of the served workload (capped G(n, p), n
    log-uniform in [64, 2048]) submitted as a Poisson stream while earlier
    ones run, each against the oracle's stored count, hash, histogram and
    GreedyBB tree (tests/golden/served2000_results.txt)."""
    import multiprocessing as mp
    import make_workload_golden as mk
    gold = mk.load("served")
    assert len(gold) == 2000
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        specs = pool.map(_gen_served_rows, range(2000), chunksize=16)
    ctx = mce.Context(0)
    graphs = [ctx.load_bitset(n, rows) for n, rows in specs]
    gaps = np.diff(synth.served_arrivals(2000, 4000.0), prepend=0.0)
    t0 = time.perf_counter()
    due = np.cumsum(gaps)
    tickets = []
    for g, at in zip(graphs, due):           # arrive at about 4000 requests/s
        while time.perf_counter() - t0 < at:
            pass
        tickets.append(ctx.submit(g))
    got = [ctx.wait(t, timeout_ns=120_000_000_000) for t in tickets]
    bad = []
    for g, r in zip(gold, got):
        hist = {k: int(v) for k, v in enumerate(r["hist"]) if v}
        if (r["rc"], r["count"], r["hash"], r["nodes"], r["internal"], r["dead_ends"], hist) != \
                (0, g["count"], g["hash"], g["nodes"], g["internal"], g["dead_ends"], g["hist"]):
            bad.append(g["index"])
    for g in graphs:
        g.free()
    ctx.close()
    assert not bad, bad[:20]
