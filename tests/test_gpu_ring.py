"""The device-wide frame ring under pressure, on one GPU: a few small blocks
(a ring of 1,024 or 2,048 slots) and breadth-first splitting down to small candidate
sets, so that tens of thousands of frames pass through the ring, its tickets
wrap around many times, producers wait for slots and consumers hold tickets
ahead of the producers.  Results stay exact against the oracle (count, hash,
histogram, nodes, internal nodes, dead ends)."""
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


CASES = [
    # Moon-Moser on 36 vertices: 3^12 cliques; every level keeps all but three
    # vertices, so a split threshold of 9 publishes the top nine levels
    ("mm36", 36, synth.moon_moser(12), "greedy", dict(blocks=2, threads=64, lanes=1, words=2, split_min_p=9)),
    ("mm36_tx", 36, synth.moon_moser(12), "tx", dict(blocks=2, threads=64, lanes=1, words=2, split_min_p=9)),
    ("gnp150", 150, synth.gnp(150, 0.5, 930), "greedy", dict(blocks=3, threads=96, split_min_p=10)),
    ("gnp150_tomita", 150, synth.gnp(150, 0.5, 930), "tomita", dict(blocks=3, threads=96, split_min_p=10)),
    ("gnp400", 400, synth.gnp(400, 0.3, 931), "greedy", dict(blocks=2, threads=128, split_min_p=12)),
]


@pytest.mark.parametrize("name,n,uv,mode,kw", CASES, ids=[c[0] for c in CASES])
def test_ring_under_pressure_stays_exact(mce, name, n, uv, mode, kw):
    import torch
    dev = torch.device("cuda:0")
    s = torch.cuda.current_stream()
    W = (n + 31) // 32
    rows = torch.from_numpy(synth.to_bitset(n, uv).view(np.int32).reshape(-1)).to(dev)
    o = mce.options(pivot=mode, **kw)
    nb = mce.mce_scratch_bytes(n, o)
    scr = torch.empty(nb, dtype=torch.uint8, device=dev)
    out = torch.zeros(mce.MCE_OUT_WORDS(n), dtype=torch.int64, device=dev)
    assert mce.mce_enumerate_device(n, W, rows, o, scr, nb, out, s) == 0
    torch.cuda.synchronize()
    r = mce.decode_out(out, n)
    ref = oracle.tomita(n, uv)
    tree = oracle.ordered(n, uv, mode)
    assert r["status"] == 0
    assert (r["count"], r["hash"]) == (ref["count"], ref["hash"])
    assert np.array_equal(r["hist"], ref["hist"])
    assert (r["nodes"], r["internal"], r["dead_ends"]) == (tree["nodes"], tree["internal"], tree["dead_ends"])
    # every published frame was taken, and on the Moon-Moser cases (128
    # one-lane groups: a ring of 1,024 slots; about 2,000 to 4,000 frames
    # published, depending on the schedule) its tickets wrapped around
    assert r["global_steals"] >= r["global_pushes"]
    if name.startswith("mm"):
        assert r["global_pushes"] > 1024
