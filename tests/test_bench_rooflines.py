"""The benchmark's per-stage roofline arithmetic on made-up stage counters (CPU only): the roof of
a stage is the larger of its flops at the stage's compute peak and its bytes at the HBM rate,
and the summed fraction leaves out the latency-bound float64 algebra."""
import argparse
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_stage_rooflines():
    sys.path.insert(0, ROOT)
    import bench
    peaks = {"bf16_tflops_sustained": 1800.0, "hbm_gbs": 6000.0}
    prof = {"gemm": (16, 2.0, 176e9, 1e9),             # 176 GFLOP at 880 TFLOP/s = 0.2 ms
            "response_density": (1, 1.0, 90e9, 12e9),  # 0.05 ms of flops, 2 ms of bytes
            "trace": (7, 0.5, 0.0, 0.6e9),             # 0.1 ms of bytes
            "small_fp64": (4, 0.4, 0.0, 0.0),
            "vector": (0, 0.0, 0.0, 0.0)}
    out, summed = bench.stage_rooflines(prof, peaks, argparse.Namespace(precision="mixed"))
    assert out["gemm"]["roof_ms"] == pytest.approx(0.2) and out["gemm"]["bound"] == "tensor"
    assert out["gemm"]["frac"] == pytest.approx(0.1)
    assert out["response_density"]["roof_ms"] == pytest.approx(2.0) and out["response_density"]["bound"] == "hbm"
    assert out["trace"]["roof_ms"] == pytest.approx(0.1)
    assert "small_fp64" not in out and "vector" not in out
    assert summed["roof_ms"] == pytest.approx(2.3) and summed["measured_ms"] == pytest.approx(3.5)
    assert summed["frac"] == pytest.approx(2.3 / 3.5, rel=1e-3)
    assert summed["small_fp64_ms_excluded"] == pytest.approx(0.4)
