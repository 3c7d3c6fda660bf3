"""The roofline microbenchmarks (mce_measure_peaks) on one GPU: every rate is
measured (positive, finite) and sits in the range the SM's unit counts and
clock allow, so that a roofline fraction divides by a real figure."""
from __future__ import annotations

import math

import pytest

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


def test_peaks_are_measured_and_plausible(mce):
    pk = mce.mce_measure_peaks(0)
    for k in ("lop3_lane_ops_per_s", "popc_lane_ops_per_s", "lds_bytes_per_s", "ballot_warp_ops_per_s",
              "shfl_warp_ops_per_s", "redux_warp_ops_per_s"):
        assert math.isfinite(pk[k]) and pk[k] > 0, k
    clk = pk["sm_clock_max_khz"] * 1e3
    sms = pk["sm_count"]
    assert sms > 0 and clk > 0
    # per SM per clock: at most 128 lanes of one 32-bit logic op, 128 bytes of
    # shared-memory loads, 4 warp instructions of any kind (4 schedulers);
    # measured at a clock no higher than the maximum, so never above these
    assert pk["lop3_lane_ops_per_s"] <= 1.05 * 128 * sms * clk
    assert pk["lds_bytes_per_s"] <= 1.05 * 128 * sms * clk
    for k in ("ballot_warp_ops_per_s", "shfl_warp_ops_per_s", "redux_warp_ops_per_s"):
        assert pk[k] <= 1.05 * 4 * sms * clk, k
    # and none is absurdly low (a broken kernel or a timer of the wrong unit)
    assert pk["lop3_lane_ops_per_s"] >= 8 * sms * clk
    assert pk["lds_bytes_per_s"] >= 8 * sms * clk
