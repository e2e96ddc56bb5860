"""Host logic of bench.py's roofline report (no GPU): per-kernel aggregation of
the library's profile records, the choice of the binding roof from the
arithmetic intensity against the measured ridge point, the achieved fraction,
the shares of the timed region, and the DRAM traffic scaled from the committed
capture to a run's edges per launch."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _rec(launches, ms, flops, nbytes):
    return {"launches": launches, "ms": ms, "flops": flops, "bytes": nbytes}


def test_by_kernel_sums_the_maps_of_a_kernel():
    rep = {"gemm_tc/a:silu": _rec(2, 1.0, 10.0, 5.0), "gemm_tc/b:linear": _rec(3, 2.0, 20.0, 7.0),
           "row_bwd_mid": _rec(1, 0.5, 0.0, 3.0)}
    out = bench._by_kernel(rep)
    assert out["gemm_tc"] == _rec(5, 3.0, 30.0, 12.0)
    assert out["row_bwd_mid"] == _rec(1, 0.5, 0.0, 3.0)


def test_roofline_hbm_bound_below_the_ridge():
    peaks = bench._peaks()
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    tc = peaks["bf16_tflops_sustained"] if peaks else 1700.0
    ridge = tc * 1e12 / (hbm * 1e9)
    # one GEMM map: 2 ms, intensity half the ridge point
    nbytes = 1e10
    flops = 0.5 * ridge * nbytes
    rep = {"gemm_tc/x:silu": _rec(4, 2.0, flops, nbytes), "row_fwd_mid": _rec(1, 1.0, 0.0, 1e9)}
    r = bench._roofline(rep, step_ms_total=4.0, steps=1, n_edges=0)
    assert r["kernel"] == "gemm_tc" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(nbytes / 2e-3 / 1e9, rel=1e-6)
    assert r["frac"] == pytest.approx(r["achieved"] / hbm, abs=1e-4)
    assert r["tensor"]["arithmetic_intensity_flop_per_byte"] == pytest.approx(0.5 * ridge, abs=0.1)
    assert r["share_of_timed_region"] == {"gemm_tc": 0.5, "row_fwd_mid": 0.25}
    assert r["launches"] == 4 and r["ms_per_launch"] == pytest.approx(0.5)
    assert r["gemm_detail"]["x:silu"]["share"] == 0.5


def test_roofline_tensor_bound_above_the_ridge():
    peaks = bench._peaks()
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    tc = peaks["bf16_tflops_sustained"] if peaks else 1700.0
    ridge = tc * 1e12 / (hbm * 1e9)
    rep = {"gemm_tc/x:silu": _rec(1, 1.0, 4.0 * ridge * 1e9, 1e9)}
    r = bench._roofline(rep, step_ms_total=1.0)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s" and r["peak"] == tc


def test_dominant_kernel_is_the_largest_total_time():
    rep = {"gemm_tc/x:silu": _rec(1, 1.0, 1.0, 1.0), "row_bwd_mid": _rec(1, 3.0, 0.0, 1e9)}
    r = bench._roofline(rep, step_ms_total=4.0)
    assert r["kernel"] == "row_bwd_mid" and r["bound"] == "hbm" and r["traffic"] is None


def test_traffic_scales_the_committed_capture():
    ref = json.load(open(os.path.join(ROOT, "profiles", "gemm_tc_traffic.json")))
    per_edge = ref["dram_bytes_per_edge_per_gemm_launch"]
    # 6 chunks per step (60 GEMM launches in 1 step of 10 per chunk), 1.2 M edges per step
    detail = {"gemm_tc/a:silu": _rec(30, 1.0, 1.0, 1.0), "gemm_tc/b:silu": _rec(30, 1.0, 1.0, 1.0)}
    t = bench._traffic_per_launch(detail, steps=1, n_edges=1_200_000)
    # launches per step of the first map = 30 -> 30 chunks; edges per launch = 1.2 M / 30
    assert t == pytest.approx(per_edge * 1_200_000 / 30)
