"""Host logic of bench.py's roofline report (no GPU): per-kernel aggregation of
the library's profile records, the model's MLP FLOPs and the fused-activation
byte budget per edge from the architecture, the MLP GEMMs against the tensor
roof with the model's FLOPs per launch, other kernels against HBM, the shares
of the timed region, and the DRAM traffic scaled from the committed capture to
a run's edges per launch."""
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


def test_model_macs_follow_the_architecture():
    from synth import ARCHS
    # 2 layers, l_max 2, 64 channels, two-body 18->64->128->256, latent (256+64)->256->256,
    # embedding and env weights 256->192, edge 256->128->1
    assert bench.model_macs_per_edge(ARCHS["c2"]) == (18 * 64 + 64 * 128 + 128 * 256 + 256 * 192
                                                      + 2 * (256 * 192 + 320 * 256 + 256 * 256)
                                                      + 256 * 128 + 128) == 517_376
    # 1 layer, l_max 1, 8 channels: 12->32, 32->16, 32->16, (32+8)->32, 32->1
    assert bench.model_macs_per_edge(ARCHS["c1"]) == 12 * 32 + 32 * 16 + 32 * 16 + 40 * 32 + 32
    assert bench.model_flops_per_edge(ARCHS["c2"]) == 4 * 517_376


def test_step_bytes_per_edge():
    from synth import ARCHS
    # CSR 16 B + x^0, x^1, x^2 (256 bf16 each) written and read + 4 per-atom C S float32 arrays
    # shared by ~25 edges + g written and read
    b = bench.step_bytes_per_edge(ARCHS["c2"], 25.0)
    assert b == pytest.approx(16 + 3 * 2 * 512 + 4 * 64 * 9 * 4 / 25.0 + 24)


def test_gemm_roofline_is_tensor_bound_with_model_flops():
    from synth import ARCHS
    arch = ARCHS["c2"]
    peaks = bench._peaks()
    tc = peaks["bf16_tflops_sustained"] if peaks else 1700.0
    n_edges, n_atoms, steps = 1_000_000, 40_000, 2
    # 20 launches over 2 steps, 3 ms each; executed flops deliberately different from the model's
    rep = {"gemm_tc/x:silu": _rec(12, 36.0, 1e12, 1e10), "gemm_tc/y:head": _rec(8, 24.0, 5e11, 1e10),
           "row_fwd_mid": _rec(2, 10.0, 0.0, 1e9)}
    r = bench._roofline(rep, step_ms_total=100.0, steps=steps, n_edges=n_edges, arch=arch, n_atoms=n_atoms)
    assert r["kernel"] == "gemm_tc" and r["bound"] == "tensor" and r["unit"] == "TFLOP/s" and r["peak"] == tc
    flops_launch = bench.model_flops_per_edge(arch) * n_edges * steps / 20
    assert r["flops_per_launch"] == pytest.approx(flops_launch)
    assert r["ms_per_launch"] == pytest.approx(3.0)
    assert r["achieved"] == pytest.approx(flops_launch / 3e-3 / 1e12, rel=1e-4)
    assert r["frac"] == pytest.approx(r["achieved"] / tc, abs=1e-4)
    assert r["share_of_timed_region"] == {"gemm_tc": 0.6, "row_fwd_mid": 0.1}
    sb = bench.step_bytes_per_edge(arch, n_edges / n_atoms)
    assert r["step_hbm"]["achieved_gbs"] == pytest.approx(sb * n_edges / 50e-3 / 1e9, rel=1e-3)
    assert r["gemm_detail"]["x:silu"]["share"] == 0.36


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
