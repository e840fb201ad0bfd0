"""Periodic box -- oracle (test infrastructure).

Sec. 2.1: the paper's box is periodic; pair vectors follow the minimum-image
convention (each component of r_j - r_i replaced by its image nearest zero),
and a disk leaving one side re-enters at the other.  Sec. 4.1: the
triangulation then lives on a flat torus of side L.

The oracle builds the torus triangulation from the Delaunay triangulation of
the 3 x 3 tiling of the points (the points plus their eight images shifted
by L in x, y or both), made by the oracle's own builder.  A triangle of the
torus is kept once: as the lifted triangle whose smallest disk id lies in
the central copy.  Each corner is reported as (disk id, integer shift s):
it sits at xy[id] + L s.  For boxes several disk spacings wide the lifted
triangles touching the central copy have circumcircles well inside the 3 x 3
tiling, so they are exactly the Delaunay triangles of the infinite periodic
point set.

Edges are keyed (u, w, s) with u < w and s the shift of w's image relative
to u's: the pair vector is xy[w] + L s - xy[u].
"""
import numpy as np

from . import geometry

SHIFTS = np.array([(sx, sy) for sy in (-1, 0, 1) for sx in (-1, 0, 1)], dtype=np.int64)


def wrap(xy, L):
    """Coordinates brought into [0, L) (a disk leaving one side re-enters at
    the other)."""
    y = np.asarray(xy, dtype=np.float64) - L * np.floor(np.asarray(xy, dtype=np.float64) / L)
    y = np.where(y >= L, y - L, y)
    return np.where(y < 0, y + L, y)


def min_image(d, L):
    """Minimum-image form of pair vectors d (any shape, last axis 2)."""
    d = np.asarray(d, dtype=np.float64)
    return d - L * np.round(d / L)


def delaunay_torus(xy, L):
    """The Delaunay triangulation of the periodic point set on the torus.
    Returns (tri (T, 3) disk ids counter-clockwise, shift (T, 3, 2) integer
    image shifts of the corners); T = 2n for a proper torus triangulation."""
    xy = np.asarray(xy, dtype=np.float64)
    n = len(xy)
    pts = np.concatenate([xy + L * s for s in SHIFTS], axis=0)
    src = np.tile(np.arange(n), len(SHIFTS))
    sh = np.repeat(SHIFTS, n, axis=0)
    F = 4.0 * L
    square = np.array([(-F, -F), (F + L, -F), (F + L, F + L), (-F, F + L)])
    tris = geometry.delaunay_generic(pts, square)
    tris = tris[np.all(tris < len(pts), axis=1)]
    s_id = src[tris]                                  # (T9, 3)
    s_sh = sh[tris]                                   # (T9, 3, 2)
    k0 = np.argmin(s_id, axis=1)
    anchor = s_sh[np.arange(len(tris)), k0]
    keep = np.all(anchor == 0, axis=1)
    return s_id[keep].copy(), s_sh[keep].copy()


def edge_keys(tri, shift):
    """Sorted unique edge keys (E, 4): (u, w, sx, sy), u < w, w's image at
    xy[w] + L s relative to u's position xy[u] (u at shift 0)."""
    out = []
    for a, b in ((0, 1), (1, 2), (2, 0)):
        u, w = tri[:, a], tri[:, b]
        s = shift[:, b] - shift[:, a]
        swap = u > w
        uu = np.where(swap, w, u)
        ww = np.where(swap, u, w)
        ss = np.where(swap[:, None], -s, s)
        out.append(np.concatenate([uu[:, None], ww[:, None], ss], axis=1))
    e = np.concatenate(out, axis=0)
    return np.unique(e, axis=0)


def edge_vectors(xy, keys, L):
    """Pair vectors r_w + L s - r_u of the edges."""
    xy = np.asarray(xy, dtype=np.float64)
    return xy[keys[:, 1]] + L * keys[:, 2:4] - xy[keys[:, 0]]


def is_torus_triangulation(tri, shift):
    """Counts of a closed torus triangulation: T = 2n triangles, 3n edges, each
    edge in exactly two triangles (Euler characteristic 0)."""
    n = int(tri.max()) + 1 if len(tri) else 0
    keys = []
    for a, b in ((0, 1), (1, 2), (2, 0)):
        u, w = tri[:, a], tri[:, b]
        s = shift[:, b] - shift[:, a]
        swap = u > w
        keys.append(np.concatenate([np.where(swap, w, u)[:, None], np.where(swap, u, w)[:, None],
                                    np.where(swap[:, None], -s, s)], axis=1))
    k = np.concatenate(keys, axis=0)
    _, counts = np.unique(k, axis=0, return_counts=True)
    return len(tri) == 2 * n and len(counts) == 3 * n and bool(np.all(counts == 2))


def lifted(xy, tri, shift, L):
    """Corner coordinates (T, 3, 2) of the triangles."""
    return np.asarray(xy, dtype=np.float64)[tri] + L * shift


def close_pairs(xy, sigma, L, chunk=512, radii=None):
    """Every pair i < j whose minimum-image distance is below sigma
    (polydisperse: below a_i + a_j), with the image shift of j: rows
    (i, j, sx, sy)."""
    xy = np.asarray(xy, dtype=np.float64)
    n = len(xy)
    out = []
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        d = xy[None, :, :] - xy[c0:c1, None, :]          # r_j - r_i
        s = -np.round(d / L)
        d = d + L * s
        r = np.sqrt(d[:, :, 0] ** 2 + d[:, :, 1] ** 2)
        lim = sigma if radii is None else radii[c0:c1, None] + radii[None, :]
        ii, jj = np.nonzero(r < lim)
        ii = ii + c0
        keep = jj > ii
        if keep.any():
            out.append(np.concatenate([ii[keep, None], jj[keep, None],
                                       s[ii[keep] - c0, jj[keep]].astype(np.int64)], axis=1))
    return np.concatenate(out) if out else np.zeros((0, 4), dtype=np.int64)
