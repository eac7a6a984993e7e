"""Host-side arithmetic of bench.py's roofline objects (no GPU).

The bench reports, per distance-tile kernel, the algorithmic bytes of a
launch (every packed point read once: coordinates, norm, two thresholds and
the input index, plus 8 bytes per result pair), the algorithmic flops (d fused
multiply-adds per evaluated pair, or 2 K per pair for the tensor-core filters),
the achieved rate over the event-timed kernel duration, the peak it is divided
by and where that peak comes from.  These tests recompute those figures by
hand for fixed inputs.
"""
import importlib.util
import json
import os
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


W4 = types.SimpleNamespace(n=2_000_000, d=4, name="uniform4d")


def test_fp32_filter_is_bytes_bound(bench):
    r = {"n_evaluated": 450_000_000, "count": 121_473_756}
    ms = 0.9
    roof = bench.roofline("filter_f32", W4, r, ms)
    # binary32 rows of dp = 4: 4 (4 + 3) + 4 = 32 bytes a point, 8 a pair
    nbytes = W4.n * 32 + 8 * r["count"]
    assert roof["bytes_per_launch"] == nbytes
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert roof["achieved"] == pytest.approx(nbytes / (ms * 1e-3) / 1e9, rel=1e-3)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"], rel=1e-3)
    assert roof["peak"] == float(_peaks().get("hbm_gbs", 6800.0))
    assert "hbm_gbs" in roof["peak_source"] or "fallback" in roof["peak_source"]
    # the arithmetic side: 2 d flop per evaluated pair against the FP32 formula
    assert roof["flop_per_launch"] == 2.0 * 4 * r["n_evaluated"]
    assert roof["alu_frac"] == pytest.approx(
        roof["flop_per_launch"] / (ms * 1e-3) / 1e12 / bench.FP32_FMA_PEAK_TFLOPS, rel=1e-2)
    assert "formula" in roof["alu_peak_source"]


def test_fp64_tile_is_alu_bound_on_the_measured_dfma_peak(bench):
    r = {"n_evaluated": 920_300_447, "count": 121_473_756}
    ms = 7.08
    roof = bench.roofline("fp64_fma", W4, r, ms)
    assert roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    assert roof["peak"] == pytest.approx(bench.FP64_DFMA_TFLOPS)
    assert roof["achieved"] == pytest.approx(2.0 * 4 * r["n_evaluated"] / (ms * 1e-3) / 1e12, rel=1e-3)
    assert "fp64_peaks_gb300" in roof["peak_source"]
    # binary64 rows: 8 (4 + 3) + 4 = 60 bytes a point
    assert roof["bytes_per_launch"] == W4.n * 60 + 8 * r["count"]


def test_tensor_core_flops_count_the_split_row_length(bench):
    w = types.SimpleNamespace(n=131_072, d=16, name="brute16d")
    r = {"n_evaluated": 8_610_000_000, "count": 6_980_000}
    roof = bench.roofline("filter_fp16x2", w, r, 2.86)
    # FP16x2: 3 products per dim + 3 norm slots, padded to 16: K = 64
    assert roof["flop_per_launch"] == 2.0 * 64 * r["n_evaluated"]
    assert roof["bound"] == "tensor"
    assert "bf16_tflops" in roof["peak_source"] or "fallback" in roof["peak_source"]
    roof3 = bench.roofline("filter_bf16x3", w, r, 3.0)
    assert roof3["flop_per_launch"] == 2.0 * 112 * r["n_evaluated"]  # 6 x 16 + 3 -> 112


def test_batched_groups_use_the_sustained_tensor_peak(bench):
    groups = {4: {"ms": 10.0, "kernel": "filter_f32", "flops_2d": 2.0e11, "instances": 800, "evaluated": 2.5e10},
              32: {"ms": 60.0, "kernel": "filter_fp16x2", "flops_2d": 0.0, "instances": 800, "evaluated": 1.6e11}}
    out = bench.batch_rooflines({"groups": groups})
    assert out["d32"]["bound"] == "tensor"
    assert out["d32"]["peak"] == pytest.approx(float(_peaks().get("bf16_tflops_sustained", 1700.0)), abs=1e-3)
    kp = (3 * 32 + 3 + 15) // 16 * 16
    assert out["d32"]["achieved"] == pytest.approx(2.0 * kp * 1.6e11 / 60e-3 / 1e12, rel=1e-3)
    assert out["d4"]["bound"] == "alu" and "formula" in out["d4"]["peak_source"]
