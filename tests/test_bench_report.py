"""Arithmetic of bench.py's GEMM report (no GPU): the flop counts of the setup Gram K and of
the per-iteration Q1^T [Q1 A2], and the TF32 peak derived from the measured bf16 peak."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_gemm_report_counts():
    import bench
    m, n2, k = 19200, 380, 20
    peaks = {"bf16_tflops": 2250.0}
    rep = bench._gemm_report((0.5, 10), (0.2, 10), m, n2, k, peaks, 7000.0, "measured")
    assert abs(rep["peak_tf32_tflops"] - 1100.0) < 1e-9           # 2250 x 1.1 / 2.25
    kk = rep["a0_K"]
    # 128 x 64 blocks holding entries c1 <= c2 of a 380 x 380 K: block rows 0..2 against
    # 64-column blocks 2 bi .. 5, i.e. 6 + 4 + 2 = 12 blocks
    assert kk["tensor_flops"] == 3 * 2 * m * 12 * 128 * 64
    assert kk["algorithmic_flops"] == m * n2 * (n2 + 1)
    assert abs(kk["ms"] - 0.05) < 1e-12                             # 0.5 ms over 10 launches
    assert abs(kk["tflops"] - kk["algorithmic_flops"] / 0.05e-3 / 1e12) < 1e-6
    g = rep["a2_Q1tQ1A2"]
    assert g["algorithmic_flops"] == 2 * m * k * (k + n2)
    assert g["bytes"] == 4 * m * n2 + 8 * m * k        # FP32 A2 once + the Q1 pair
    assert abs(g["gbs"] - g["bytes"] / 0.02e-3 / 1e9) < 1e-6
    assert abs(g["hbm_frac"] - g["gbs"] / 7000.0) < 1e-12


def test_gemm_report_without_measured_peaks_says_fallback():
    import bench
    rep = bench._gemm_report(None, None, 100, 50, 5, {}, 6800.0, "fallback")
    assert "fallback" in rep["peak_source"] and "a0_K" not in rep and "a2_Q1tQ1A2" not in rep
