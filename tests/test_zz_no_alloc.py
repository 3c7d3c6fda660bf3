"""The no-allocation entry point (mce_enumerate_device_static).

Some callers may not allocate device memory at all: a plug-in whose host
framework owns every device allocation, or a request path that must not
allocate per call.  For them the library keeps one fixed scratch area per GPU
and this entry point uses it instead of a caller-provided scratch buffer.
The test calls it twice in a row through the C ABI and compares every output
word with the regular entry point's (the results are exact integers, so
equality is the tolerance), and checks that a call leaves the device's free
memory unchanged.  This file is collected last so that a stop-at-first-failure
run has already run every other test.
"""
from __future__ import annotations

import numpy as np
import pytest

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


@pytest.mark.parametrize("n,p,seed", [(100, 0.5, 0), (45, 0.9, 3), (700, 0.3, 2), (2048, 0.05, 5), (4096, 0.01, 6)])
def test_static_scratch_matches_regular_entry_point(mce, n, p, seed):
    import torch
    dev = torch.device("cuda:0")
    s = torch.cuda.current_stream()
    uv = synth.gnp(n, p, seed)
    W = (n + 31) // 32
    rows = torch.from_numpy(synth.to_bitset(n, uv).view(np.int32).reshape(-1)).to(dev)
    o = mce.options()
    nbytes = mce.mce_scratch_bytes(n, o)
    assert nbytes <= mce.MCE_STATIC_SCRATCH_BYTES
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    ref = torch.zeros(mce.MCE_OUT_WORDS(n), dtype=torch.int64, device=dev)
    assert mce.mce_enumerate_device(n, W, rows, o, scratch, nbytes, ref, s) == mce.MCE_OK
    torch.cuda.synchronize()
    want = mce.decode_out(ref, n)
    assert want["status"] == 0
    for call in range(2):                    # the area keeps the previous call's contents
        out = torch.full((mce.MCE_OUT_WORDS(n),), -1, dtype=torch.int64, device=dev)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        assert mce.mce_enumerate_device_static(n, W, rows, o, out, s) == mce.MCE_OK
        torch.cuda.synchronize()
        if call == 1:                        # the first call may load device code
            assert torch.cuda.mem_get_info()[0] == free0
        got = mce.decode_out(out, n)
        for key in ("status", "count", "nodes", "internal", "dead_ends", "hash", "max_size"):
            assert got[key] == want[key], key
        assert np.array_equal(got["hist"], want["hist"])


def test_static_scratch_rejects_oversized_options(mce):
    import torch
    n = 1000
    o = mce.options(queue_log2=22)           # a work queue far larger than the fixed area
    assert mce.mce_scratch_bytes(n, o) > mce.MCE_STATIC_SCRATCH_BYTES
    rows = torch.zeros(n * 32, dtype=torch.int32, device="cuda:0")
    out = torch.zeros(mce.MCE_OUT_WORDS(n), dtype=torch.int64, device="cuda:0")
    assert mce.mce_enumerate_device_static(n, 32, rows, o, out, torch.cuda.current_stream()) == mce.MCE_ENOMEM
