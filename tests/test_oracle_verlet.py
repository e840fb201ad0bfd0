"""Pins for the oracle's Verlet lists (Sec. 2.1, Sec. 5)."""
import numpy as np
from scipy.spatial import cKDTree

from oracle import verlet


def test_verlet_matches_kdtree_ball_query():
    rng = np.random.default_rng(6)
    xy = rng.uniform(0, 80, size=(3000, 2))
    lists = verlet.build(xy, 5.0, 0.6)
    tree = cKDTree(xy)
    for i in range(0, 3000, 7):
        want = sorted(j for j in tree.query_ball_point(xy[i], 5.6 - 1e-9) if j != i)
        got = lists[i].tolist()
        # kd-tree uses <= and its own rounding; allow only boundary ties
        extra = set(got) ^ set(want)
        for j in extra:
            assert abs(np.hypot(*(xy[i] - xy[j])) - 5.6) < 1e-8
    assert all(np.all(np.diff(l) > 0) for l in lists)


def test_rebuild_trigger():
    xy = np.zeros((4, 2))
    moved = xy.copy()
    moved[2] = [0.29, 0.0]
    assert not verlet.needs_rebuild(moved, xy, 0.6)
    moved[2] = [0.31, 0.0]
    assert verlet.needs_rebuild(moved, xy, 0.6)
