"""Host-side arithmetic of bench.py: the Zolo-PD flop model credited per matrix and
the roofline entry of the dominant kernel class (no GPU)."""
import os
import sys

import pytest

from conftest import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_model_flops_per_iteration_form():
    m, n = 300, 120
    assert bench.pd_model_flops(m, n, 4, []) == 2.0 * m * n * n                 # H only
    qr = bench.pd_model_flops(m, n, 4, [True]) - 2.0 * m * n * n
    assert qr == pytest.approx(5 * 4 * m * n * n)
    ch = bench.pd_model_flops(m, n, 4, [False]) - 2.0 * m * n * n
    assert ch == pytest.approx(m * n * n + 4 * (n ** 3 / 3 + 2 * m * n * n))
    # two iterations add
    both = bench.pd_model_flops(m, n, 4, [True, False])
    assert both == pytest.approx(2.0 * m * n * n + qr + ch)


def test_roofline_of_the_dominant_fp64_class():
    kstats = {"gemm_f64": {"launches": 10, "ms": 900.0, "flops": 1.08e12, "bytes": 0.0},
              "qr_panel": {"launches": 4, "ms": 50.0, "flops": 1e9, "bytes": 0.0},
              "jacobi_round": {"launches": 0, "ms": 0.0, "flops": 0.0, "bytes": 0.0}}
    roof = bench.roofline(kstats, 1000.0)
    assert roof["kernel"] == "gemm_f64" and roof["bound"] == "alu"
    assert roof["achieved"] == pytest.approx(1.2)
    assert roof["frac"] == pytest.approx(1.2 / bench.FP64_PEAK_TFLOPS)
    assert roof["share_of_step"] == pytest.approx(0.9)
    assert roof["avg_launch_ms"] == pytest.approx(90.0)


@pytest.mark.skipif(not os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")),
                    reason="measured peaks not written on this machine")
def test_roofline_of_the_split_class_counts_issued_pairs():
    kstats = {"gemm_split": {"launches": 2, "ms": 100.0, "flops": 1e12, "bytes": 0.0}}
    roof = bench.roofline(kstats, 200.0)
    assert roof["bound"] == "tensor"
    assert roof["fp64_equivalent_tflops"] == pytest.approx(10.0)
    assert roof["achieved"] == pytest.approx(530.0)            # 53 slice-pair products
    assert roof["frac"] == pytest.approx(530.0 / roof["peak"])


def test_roofline_shares_the_model_flops_between_classes():
    # the launches state 1.2e12 + 0.3e12 flops; the model credits 1.0e12 to the
    # step, so the dominant class is credited 0.8e12 over its 0.9 s
    kstats = {"gemm_f64": {"launches": 10, "ms": 900.0, "flops": 1.2e12, "bytes": 0.0},
              "qr_panel": {"launches": 4, "ms": 50.0, "flops": 0.3e12, "bytes": 0.0},
              "combine": {"launches": 2, "ms": 1.0, "flops": 0.0, "bytes": 1e6}}
    roof = bench.roofline(kstats, 1000.0, model_flops=1.0e12)
    assert roof["kernel"] == "gemm_f64"
    assert roof["achieved"] == pytest.approx(0.8e12 / 0.9 / 1e12)
    assert roof["issued_tflops"] == pytest.approx(1.2e12 / 0.9 / 1e12)
    assert "model" in roof["work_basis"]


def test_roofline_leaves_the_eigensolver_out_of_the_model_share():
    # Zolo-SVD: the Jacobi sweeps state flops the Zolo-PD model does not count,
    # so they must not dilute the share of the model's own classes
    kstats = {"gemm_f64": {"launches": 10, "ms": 900.0, "flops": 1.2e12, "bytes": 0.0},
              "qr_panel": {"launches": 4, "ms": 50.0, "flops": 0.3e12, "bytes": 0.0},
              "jacobi_round": {"launches": 4, "ms": 600.0, "flops": 2.0e12, "bytes": 0.0},
              "jacobi32_sweep": {"launches": 13, "ms": 600.0, "flops": 5.0e12, "bytes": 0.0}}
    roof = bench.roofline(kstats, 2200.0, model_flops=1.0e12)
    assert roof["kernel"] == "gemm_f64"
    assert roof["achieved"] == pytest.approx(0.8e12 / 0.9 / 1e12)


def test_oracle_sample_times_two_sizes_and_scales_by_the_model():
    w = dict(bench.WORKLOADS["pd256"], sample_n=96)
    v, spent, desc = bench.oracle_sample(w)
    assert v > 0 and spent > 0
    assert "256x96" not in desc and "96x96" in desc and "64x64" in desc


def test_roofline_traffic_scales_the_captured_ratio():
    kstats = {"qr_panel": {"launches": 4, "ms": 8.0, "flops": 4e9, "bytes": 8e6},
              "gemm_split": {"launches": 4, "ms": 2.0, "flops": 1e10, "bytes": 0.0}}
    roof = bench.roofline(kstats, 12.0, model_flops=1e10)
    assert roof["kernel"] == "qr_panel"
    assert roof["traffic"] == pytest.approx(bench.TRAFFIC_PER_STATED_BYTE["qr_panel"] * 2e6)
    assert roof["algorithmic_bytes_per_launch"] == pytest.approx(2e6)
