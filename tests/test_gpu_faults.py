"""Failure detection without a GPU fault: host-side injected failures
(mce_fault_inject) of device allocations, input copies and served
admission give their error code, release what the call had taken, and leave
the context usable (the next call is exact against the oracle); a queued
served request can be cancelled.  Nothing here makes a kernel fail."""
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


@pytest.fixture()
def ctx(mce):
    c = mce.Context(0)
    yield c
    for site in (mce.MCE_FAULT_ALLOC, mce.MCE_FAULT_COPY, mce.MCE_FAULT_ADMIT):
        mce.mce_fault_inject(site, 0, 0)
    c.close()


def _exact(r, n, uv):
    ref = oracle.tomita(n, uv)
    assert (r["count"], r["hash"]) == (ref["count"], ref["hash"])
    assert np.array_equal(r["hist"], ref["hist"])


@pytest.mark.parametrize("skip", [0, 1, 2])
def test_allocation_failure_while_loading(ctx, mce, skip):
    # loading an edge list allocates three device buffers; whichever fails,
    # the call returns MCE_ENOMEM and holds nothing afterwards
    n, uv = 120, synth.gnp(120, 0.4, 940)
    base = ctx.mem_used()
    assert mce.mce_fault_inject(mce.MCE_FAULT_ALLOC, skip, 1) == mce.MCE_OK
    with pytest.raises(mce.MceError) as e:
        ctx.load_edges(n, uv)
    assert e.value.code == mce.MCE_ENOMEM
    assert ctx.mem_used() == base
    g = ctx.load_edges(n, uv)
    try:
        _exact(g.enumerate(), n, uv)
    finally:
        g.free()
    assert ctx.mem_used() == base


def test_allocation_failure_while_enumerating(ctx, mce):
    n, uv = 200, synth.gnp(200, 0.3, 941)
    g = ctx.load_edges(n, uv)
    try:
        held = ctx.mem_used()
        mce.mce_fault_inject(mce.MCE_FAULT_ALLOC, 0, 1)
        r = g.enumerate(raise_on_error=False)
        assert r["rc"] == mce.MCE_ENOMEM
        assert ctx.mem_used() == held
        _exact(g.enumerate(), n, uv)
    finally:
        g.free()


def test_copy_failure_while_loading(ctx, mce):
    n, uv = 90, synth.gnp(90, 0.5, 942)
    base = ctx.mem_used()
    mce.mce_fault_inject(mce.MCE_FAULT_COPY, 0, 1)
    with pytest.raises(mce.MceError) as e:
        ctx.load_edges(n, uv)
    assert e.value.code == mce.MCE_ECUDA
    assert ctx.mem_used() == base
    rows = synth.to_bitset(n, uv)
    mce.mce_fault_inject(mce.MCE_FAULT_COPY, 0, 1)
    with pytest.raises(mce.MceError) as e:
        ctx.load_bitset(n, rows)
    assert e.value.code == mce.MCE_ECUDA
    g = ctx.load_bitset(n, rows)
    try:
        _exact(g.enumerate(), n, uv)
    finally:
        g.free()
    assert ctx.mem_used() == base


def test_admission_failures_delay_but_do_not_lose_requests(ctx, mce):
    specs = [(n, synth.gnp(n, 0.3, 950 + n)) for n in (60, 150, 300, 500)]
    graphs = [ctx.load_edges(n, uv) for n, uv in specs]
    try:
        mce.mce_fault_inject(mce.MCE_FAULT_ADMIT, 0, 25)
        tickets = [ctx.submit(g) for g in graphs]
        for (n, uv), t in zip(specs, tickets):
            r = ctx.wait(t, 60_000_000_000)
            assert r["rc"] == mce.MCE_OK
            _exact(r, n, uv)
    finally:
        for g in graphs:
            g.free()


def test_cancel_a_queued_request(ctx, mce):
    n, uv = 300, synth.gnp(300, 0.3, 960)
    g = ctx.load_edges(n, uv)
    try:
        # admission refused long enough for the request to be still queued
        mce.mce_fault_inject(mce.MCE_FAULT_ADMIT, 0, 1_000_000)
        t = ctx.submit(g)
        assert ctx.cancel(t) == mce.MCE_OK
        r = ctx.wait(t, 10_000_000_000)
        assert r["rc"] == mce.MCE_ECANCELED
        mce.mce_fault_inject(mce.MCE_FAULT_ADMIT, 0, 0)
        assert ctx.cancel(t) == mce.MCE_EINVAL  # delivered: the ticket is gone
        t2 = ctx.submit(g)
        r2 = ctx.wait(t2, 60_000_000_000)
        assert r2["rc"] == mce.MCE_OK
        _exact(r2, n, uv)
        assert ctx.cancel(t2) == mce.MCE_EINVAL
    finally:
        g.free()


def test_cancel_after_admission_is_refused(ctx, mce):
    import time
    n, uv = 80, synth.gnp(80, 0.4, 961)
    g = ctx.load_edges(n, uv)
    try:
        t = ctx.submit(g)
        time.sleep(0.05)  # admitted within microseconds, done within a millisecond
        assert ctx.cancel(t) == mce.MCE_EBUSY
        r = ctx.wait(t, 60_000_000_000)
        assert r["rc"] == mce.MCE_OK
        _exact(r, n, uv)
    finally:
        g.free()
