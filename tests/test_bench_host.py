"""Host-side arithmetic of bench.py (no GPU): the method's bytes per
angle-iteration, the roofline figures computed from kernel timings, the
ncu traffic table's fingerprint rule, and the workload both arms name."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
import paper_2402_05283_gb300 as cp  # noqa: E402  (constants only; no library load)


class FakePlan:
    """kernel_stats(kind) -> (total ms, launches), as the C ABI reports them."""

    def __init__(self, stats):
        self.stats = stats

    def kernel_stats(self, kind):
        return self.stats.get(kind, (0.0, 0))


def test_method_bytes_hand_value():
    # read and write the FP32 iterate (4 N^2 each), read the half-plane
    # amplitude (4 N (N/2 + 1)) and the support bits (N^2 / 8), N = 512
    assert bench.method_bytes_per_angle_iteration(512) == 1048576 + 1048576 + 526336 + 32768
    assert bench.method_bytes_per_angle_iteration(16) == 1024 + 1024 + 576 + 32


def test_roofline_from_kernel_times():
    # 220 iterations of 360 angles: column 56 ms, row 51 ms, 22 primes 5.5 ms
    stats = {cp.KERNEL_COLPASS: (56.0, 220), cp.KERNEL_ROWPASS: (51.0, 220),
             cp.KERNEL_PRIME: (5.5, 22), cp.KERNEL_ASSEMBLE: (3.8, 5)}
    roof, _ = bench.roofline_figures(FakePlan(stats), cp, {"hbm_gbs": 6796.5}, 360, 220)
    ms_per_iter = (56.0 + 51.0 + 5.5) / 220
    unit = 360 * bench.method_bytes_per_angle_iteration(512)
    achieved = unit / (ms_per_iter * 1e-3) / 1e9
    assert roof["ms_per_iteration"] == pytest.approx(ms_per_iter, abs=1e-5)
    assert roof["achieved"] == pytest.approx(achieved, abs=0.05)
    assert roof["frac"] == pytest.approx(achieved / 6796.5, abs=1e-4)
    assert roof["bytes_per_iteration"] == unit
    assert roof["kernel"].endswith("k_colpass + k_rowpass + k_prime")
    col = roof["per_kernel"]["k_colpass"]
    assert col["ms_per_launch"] == pytest.approx(56.0 / 220, abs=1e-4)
    # the column pass's own design bytes: Hp in and out, A_sym
    assert col["design_bytes_per_launch"] == 360 * (10 * 512 * 512 + 4 * 512)
    # assembly time is not iteration time
    assert "assembly" not in roof["per_kernel"]


def test_traffic_only_for_the_captured_sources(monkeypatch):
    stats = {cp.KERNEL_COLPASS: (56.0, 220), cp.KERNEL_ROWPASS: (51.0, 220), cp.KERNEL_PRIME: (5.5, 22)}
    key = (("k_colpass", "k_rowpass", "k_prime"), 512)
    per_ai, date, fp = bench.NCU_ITERATION_TRAFFIC[key]
    monkeypatch.setattr(bench, "kernel_fingerprint", lambda: fp)
    roof, _ = bench.roofline_figures(FakePlan(stats), cp, {"hbm_gbs": 6796.5}, 360, 220)
    assert roof["traffic"] == int(per_ai * 360) and date in roof["traffic_note"]
    monkeypatch.setattr(bench, "kernel_fingerprint", lambda: "0" * 16)
    roof, _ = bench.roofline_figures(FakePlan(stats), cp, {"hbm_gbs": 6796.5}, 360, 220)
    assert roof["traffic"] is None


def test_no_roofline_without_iteration_time():
    roof, _ = bench.roofline_figures(FakePlan({cp.KERNEL_ASSEMBLE: (3.8, 1)}), cp, {}, 360, 220)
    assert roof is None


def test_both_arms_name_the_same_workload():
    a, b = bench.bench_config(1), bench.bench_config(1)
    assert a == b and a["N"] == 512 and a["Np"] == 360 and a["iterations"] == 220
    assert bench.bench_config(4)["parallelism"] == "replicas x4"
