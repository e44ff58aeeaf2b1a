"""The benchmark's detection roofline on CPU: per engine, which resources bound a launch, the
binding one is the slowest at its peak, and the peaks follow from the unit counts and clock."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_fp32_pipe_and_mufu_peaks_follow_from_unit_counts_and_clock():
    # 152 SMs x 128 FP32 lanes x 2 flop and 152 SMs x 32 ex2 per clock, at 2070 MHz
    assert bench.FP32_PEAK_TFLOPS == pytest.approx(80.54784)
    assert bench.MUFU_PEAK_PER_S == pytest.approx(10.06848e12)


@pytest.mark.parametrize("engine,resources", [("tf32x3", {"tensor", "alu", "mufu"}),
                                              ("half", {"tensor", "alu", "mufu"}),
                                              ("ffma", {"alu", "mufu"})])
def test_the_bound_is_the_slowest_resource_of_the_engine(engine, resources):
    w = dict(M=16, K=6, N=65536)
    r = bench.detect_roofline(w, 1024, 1e-3, engine)
    assert set(r["frac_by_resource"]) == resources
    assert r["bound"] == max(r["frac_by_resource"], key=r["frac_by_resource"].get)
    assert r["frac"] == pytest.approx(r["frac_by_resource"][r["bound"]], rel=1e-3)
    assert r["achieved"] / r["peak"] == pytest.approx(r["frac"], rel=1e-9)


def test_fp32_pipe_work_per_pair_by_engine():
    # the tensor engines leave 4K + 3 FMA per pair on the FP32 pipe, the FMA engine also the
    # Gram's 4M: at M = 64, K = 16 that is 67 against 323 FMA per pair
    w, pairs, s = dict(M=64, K=16, N=1000), 1000 * 4096, 1e-5  # fractions of order 1
    half = bench.detect_roofline(w, 4096, s, "half")["frac_by_resource"]["alu"]
    ffma = bench.detect_roofline(w, 4096, s, "ffma")["frac_by_resource"]["alu"]
    assert half == pytest.approx(round(2 * 67 * pairs / (bench.FP32_PEAK_TFLOPS * 1e12) / s, 4), abs=1e-4)
    assert ffma / half == pytest.approx(323 / 67, rel=1e-2)


def test_tf32x3_issues_three_products_against_the_scaled_bf16_peak():
    w, s = dict(M=16, K=6, N=1 << 20), 1e-4  # fractions of order 1
    peaks = bench.measured_peaks()
    bf16 = peaks.get("bf16_tflops", 1900.0)
    t3 = bench.detect_roofline(w, 1024, s, "tf32x3")["frac_by_resource"]["tensor"]
    t1 = bench.detect_roofline(w, 1024, s, "half")["frac_by_resource"]["tensor"]
    # three products at 1.1/2.25 of the BF16 rate against one product at the BF16 rate
    assert t3 / t1 == pytest.approx(3 * 2.25 / 1.1, rel=2e-3)
    assert t1 == pytest.approx(round(2 * 32 * 2 * (1 << 20) * 1024 / (bf16 * 1e12) / s, 4), abs=1e-4)
