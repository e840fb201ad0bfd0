"""The benchmark's host arithmetic, on the CPU: the correction kernel's
algorithmic bytes and roofline fraction, and the CPU baseline's fields."""
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
