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


def _lattice_sites(L, a):
    # the number of triangular-lattice sites of spacing 2a over [a, L - a]^2
    W = L - 2 * a
    s = 2 * a
    nx0 = int(math.floor(W / s)) + 1
    nx1 = int(math.floor((W - 0.5 * s) / s)) + 1
    ny = int(math.floor(W / (s * math.sqrt(3) / 2))) + 1
    return ((ny + 1) // 2) * nx0 + (ny // 2) * nx1


def test_lattice_at_its_packing_limit_is_refused():
    # a box whose width is a whole number of spacings 2a (W = 40) and exactly
    # as many disks as lattice sites of spacing 2a: any wider spacing has
    # fewer sites, so there is no room to jitter and the start would be a
    # perfect lattice (four sites on every circle)
    L = 42.0
    n = _lattice_sites(L, 1.0)
    with pytest.raises(bd.BDError) as e:
        bd.place_disks(n, L, 1.0, bd.PLACE_LATTICE, seed=2)
    assert e.value.code == -1


def test_lattice_near_its_limit_is_in_general_position():
    # a few sites to spare: every site, border rows included, is jittered, so
    # no four centres are cocircular (the Delaunay triangulation is unique)
    from oracle import geometry
    L = 41.3
    n = _lattice_sites(L, 1.0) - 3
    xy = bd.place_disks(n, L, 1.0, bd.PLACE_LATTICE, seed=2)
    _check_valid(xy, n, L, 1.0)
    tris = geometry.delaunay(xy, L, 1.0)
    assert geometry.general_position(geometry.with_ghosts(xy, L, 1.0), tris)
