"""Verlet neighbour lists -- oracle (test infrastructure).

Sec. 2.1 / Sec. 5: short-range forces are truncated, so each disk keeps the
list of disks within r_cut + skin; forces are summed over the list only, and
the list is rebuilt when some disk has moved more than skin/2 since the last
build (then no pair can have entered r_cut unseen).  The oracle builds the
list by brute force over all pairs; membership is decided in FP64 as
(x_i - x_j)*(x_i - x_j) + (y_i - y_j)*(y_i - y_j) < (r_cut + skin)^2, two
products and one sum, each rounded once.
"""
import numpy as np


def build(xy, r_cut, skin, L=None):
    """List of sorted neighbour index arrays, one per disk (brute force).
    L: periodic box side (minimum-image differences); None = walls."""
    xy = np.asarray(xy, dtype=np.float64)
    n = len(xy)
    rl2 = (r_cut + skin) * (r_cut + skin)
    out = []
    for c0 in range(0, n, 1024):
        dx = xy[c0:c0 + 1024, None, 0] - xy[None, :, 0]
        dy = xy[c0:c0 + 1024, None, 1] - xy[None, :, 1]
        if L is not None:
            dx = dx - L * np.round(dx / L)
            dy = dy - L * np.round(dy / L)
        d2 = dx * dx + dy * dy
        for r in range(d2.shape[0]):
            i = c0 + r
            nb = np.nonzero(d2[r] < rl2)[0]
            out.append(nb[nb != i])
    return out


def needs_rebuild(xy, xy_at_build, skin):
    d = np.asarray(xy) - np.asarray(xy_at_build)
    return float(np.max(np.sqrt(d[:, 0] ** 2 + d[:, 1] ** 2))) > 0.5 * skin
