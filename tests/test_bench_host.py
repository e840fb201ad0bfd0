"""The benchmark's host arithmetic, on the CPU: the force sweep's and the
correction kernel's roofline figures, and the CPU baseline's fields."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _FakeSystem:
    n_tri = 2000


def test_correction_roofline_counts_the_documented_bytes():
    # 2 steps: 8 check passes visiting 9000 triangles, 4 flip rounds with 60
    # flips, 2 apply passes
    stage_raw = {"check": (0.8, 8), "repair": (0.0, 0), "flip": (0.2, 4), "apply": (0.1, 2),
                 "check_lists": (0.3, 6)}
    N, steps, visits, flips = 1000, 2, 4500.0, 30.0
    r = bench.correction_roofline(_FakeSystem(), stage_raw, steps, N, False, {"hbm_gbs": 5000.0},
                                  "measured", visits=visits, flips=flips)
    A = 1.0                                    # apply passes per launch
    per = 32 * visits + 25 * N + 200 * flips + A * 100 * N
    ms = (0.8 + 0.2 + 0.1) / steps             # check_lists is part of check
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(per)
    assert r["avg_launch_ms"] == pytest.approx(ms)
    assert r["achieved"] == pytest.approx(per / (ms / 1e3) / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 5000.0)
    assert r["bound"] == "hbm" and r["kernel"] == "k_triangulation" and r["traffic"] is None


@pytest.mark.parametrize("variant,periodic,lanes,executed", [
    (3, False, 5, 8),      # symmetric sweep: 16 flops in 10 lane ops per unordered pair
    (2, True, 5, 8),       # its periodic form counts the same
    (1, False, 8, 12),     # one-sided packed sweep
    (0, True, 12, 16),     # one-sided periodic sweep (exact near-pair vectors)
])
def test_force_roofline_counts_the_algorithmic_flops(variant, periodic, lanes, executed):
    N, t, sms, f = 1000, 2.0e-5, 152, 2.07e9
    r = bench.force_roofline(N, t, variant, periodic, sms, f, "measured", traffic=123)
    pairs = N * (N - 1)
    peak = sms * 128 * 2 * f / 1e12
    # achieved: 12 flops per ordered pair whatever the sweep executes
    assert r["achieved"] == pytest.approx(12 * pairs / t / 1e12)
    assert r["peak"] == pytest.approx(peak)
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
    assert r["frac_executed"] == pytest.approx(executed * pairs / t / 1e12 / peak)
    assert r["fp32_pipe_frac"] == pytest.approx(lanes * pairs / t / (sms * 128 * f))
    assert r["pair_interactions_per_s"] == pytest.approx(pairs / t)
    assert r["avg_launch_ms"] == pytest.approx(t * 1e3)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["traffic"] == 123
    # at a full FMA pipe (fp32_pipe_frac = 1) each fraction reaches its cap
    scale = r["fp32_pipe_frac"]
    assert r["frac"] / scale == pytest.approx(12 / (2 * lanes))
    assert r["frac_executed"] / scale == pytest.approx(executed / (2 * lanes))
    assert ("periodic" in r["kernel"] or "per" in r["kernel"]) == periodic


def test_cpu_baseline_fields():
    from paper_1703_02484_gb300 import workloads
    cfg = workloads.CONFIGS["c5"]          # long range, N = 4096: a second or two
    xy, sp, th = workloads.initial_state(cfg)
    r = bench.cpu_baseline(cfg, xy, sp, th)
    assert r["kind"] == "oracle" and r["unit"] == bench.UNIT and r["cores"] >= 1
    assert r["value"] > 0 and np.isfinite(r["value"])
    if r["cores"] > 1:
        assert 0 < r["value_1core"] < r["value"] * r["cores"] * 2
    assert "oracle step" in r["sample"]
