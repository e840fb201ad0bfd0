"""The library's start positions (bd_place_disks, used by bd_init when no
positions are given), on the CPU: random sequential addition and the paper's
lattice start (Sec. 4.1: a triangular lattice with N* >= n sites, n of them
chosen by reservoir sampling, each jittered within the spare gap)."""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

import paper_1703_02484_gb300 as bd
from paper_1703_02484_gb300 import workloads


def _check_valid(xy, n, L, a):
    assert xy.shape == (n, 2)
    assert np.all(xy >= a) and np.all(xy <= L - a)
    assert len(cKDTree(xy).query_pairs(2 * a * (1 - 1e-12))) == 0


@pytest.mark.parametrize("placement", [bd.PLACE_RSA, bd.PLACE_LATTICE])
@pytest.mark.parametrize("n,rho", [(1, 0.3), (7, 0.3), (2000, 0.3), (4000, 0.5)])
def test_placement_valid_and_deterministic(placement, n, rho):
    L = workloads.box_side(max(n, 16), rho)
    a = bd.place_disks(n, L, 1.0, placement, seed=5)
    _check_valid(a, n, L, 1.0)
    assert np.array_equal(a, bd.place_disks(n, L, 1.0, placement, seed=5))
    if n > 1:
        assert not np.array_equal(a, bd.place_disks(n, L, 1.0, placement, seed=6))


def test_lattice_reaches_densities_random_addition_cannot():
    # area fraction 0.8 of [0, L]^2: beyond random sequential addition's jamming
    # (about 0.547), within the triangular lattice's (0.907 in the limit)
    n = 1500
    L = math.sqrt(n * math.pi / 0.8)
    xy = bd.place_disks(n, L, 1.0, bd.PLACE_LATTICE, seed=1)
    _check_valid(xy, n, L, 1.0)
    # nearest neighbours sit near the lattice spacing: the set is lattice-like
    d = cKDTree(xy).query(xy, k=2)[0][:, 1]
    assert d.min() >= 2.0 and np.median(d) < 2.3
    with pytest.raises(bd.BDError):
        bd.place_disks(n, math.sqrt(n * math.pi / 0.97), 1.0, bd.PLACE_LATTICE, seed=1)


def test_lattice_reservoir_sampling_is_uniform():
    # every site is kept with probability n / N*: over many seeds the kept
    # disks cover the box evenly (quadrant shares within 4 standard errors),
    # and the jitter leaves the set in general position (distinct distances)
    n, L = 60, 40.0
    pts = np.concatenate([bd.place_disks(n, L, 1.0, bd.PLACE_LATTICE, seed=s) for s in range(300)])
    mid = 0.5 * L
    for frac in ((pts[:, 0] < mid).mean(), (pts[:, 1] < mid).mean()):
        assert abs(frac - 0.5) < 4 * math.sqrt(0.25 / len(pts)) + 0.02
    one = bd.place_disks(n, L, 1.0, bd.PLACE_LATTICE, seed=3)
    dd = np.round(np.sort(cKDTree(one).query(one, k=2)[0][:, 1]), 9)
    assert len(np.unique(dd)) > n // 3


def test_placement_argument_errors():
    for args in [(0, 50.0, 1.0, 0), (10, 1.5, 1.0, 0), (10, 50.0, -1.0, 0), (10, 50.0, 1.0, 2)]:
        with pytest.raises(bd.BDError) as e:
            bd.place_disks(*args, seed=0)
        assert e.value.code == -1
