"""Pair forces in FP64 -- oracle (test infrastructure).

Long range (Sec. 2.2): the force on disk i is the sum over every other disk
k of mu_i alpha_k f(r_i - r_k) with f(r) = r / |r|^3.  The charges enter only
through the product for the ordered species pair, so the oracle stores that
product as an n x n table A[s_i][s_k] (n species) ("force ON species s_i FROM species s_k");
a positive entry pushes i away from k.  The table need not factor as
mu_i alpha_k, nor be symmetric (non-reciprocal interactions).  With
reflecting walls there are no images; in a periodic box (Sec. 2.1) every
pair vector takes its minimum image.

Short range: the paper's r/r^7 law is replaced by a WCA core plus a Yukawa
tail, both truncated (not shifted) at r_cut as in Eq. (displacement) /
Fig. "cutoff":  U = 4 eps[(s/r)^12 - (s/r)^6] + eps for r < 2^(1/6) s, plus
-eps (s/r) exp(-kappa (r - s)), with s = 2a; the force on i is -U'(r) r_hat
with r_hat pointing from k to i.
"""
import ctypes
import math

import numpy as np

from . import _clib


def species_table(A):
    """The n x n table A[s_i][s_k] from its row-major entries (n^2 of them,
    n = 1 .. 4)."""
    A = np.asarray(A, dtype=np.float64).reshape(-1)
    n = int(round(len(A) ** 0.5))
    if n * n != len(A):
        raise ValueError("a square table is needed, got %d entries" % len(A))
    return A.reshape(n, n)


def long_range_numpy(xy, species, A, idx=None, L=None):
    """Direct O(N^2) sum, numpy, for moderate N.  Returns (n_idx, 2).
    L: periodic box side (minimum-image pair vectors, Sec. 2.1); None = walls."""
    xy = np.asarray(xy, dtype=np.float64)
    s = np.asarray(species, dtype=np.int64)
    A = species_table(A)
    n = len(xy)
    idx = np.arange(n) if idx is None else np.asarray(idx)
    out = np.zeros((len(idx), 2))
    for c0 in range(0, len(idx), 512):
        ii = idx[c0:c0 + 512]
        d = xy[ii, None, :] - xy[None, :, :]          # r_i - r_k
        if L is not None:
            d = d - L * np.round(d / L)
        r2 = np.einsum("ijk,ijk->ij", d, d)
        self_ = ii[:, None] == np.arange(n)[None, :]
        r2[self_] = 1.0
        coef = A[s[ii]][:, s] / (r2 * np.sqrt(r2))
        coef[self_] = 0.0
        out[c0:c0 + 512] = np.einsum("ij,ijk->ik", coef, d)
    return out


def long_range(xy, species, A, idx=None, threads=1, L=None):
    """Same sum in the oracle's plain C loop (OpenMP over i when threads > 1).
    idx must be a contiguous range (or None for all); L as long_range_numpy."""
    xy = np.ascontiguousarray(np.asarray(xy, dtype=np.float64))
    n = len(xy)
    x = np.ascontiguousarray(xy[:, 0])
    y = np.ascontiguousarray(xy[:, 1])
    s = np.ascontiguousarray(np.asarray(species, dtype=np.uint8))
    T = species_table(A)
    ns = len(T)
    A = np.ascontiguousarray(T.reshape(-1))
    if idx is None:
        i0, i1 = 0, n
    else:
        idx = np.asarray(idx)
        i0, i1 = int(idx[0]), int(idx[-1]) + 1
        assert np.array_equal(idx, np.arange(i0, i1)), "idx must be contiguous"
    fx = np.zeros(i1 - i0)
    fy = np.zeros(i1 - i0)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    if L is None:
        _clib.lib().oracle_force_long(n, p(x), p(y), p(s), p(A), ns, i0, i1, p(fx), p(fy), int(threads))
    else:
        _clib.lib().oracle_force_long_periodic(n, p(x), p(y), p(s), p(A), ns, float(L), i0, i1, p(fx),
                                               p(fy), int(threads))
    return np.stack([fx, fy], axis=1)


def short_range_magnitude(r, eps, kappa, sigma_c):
    """-U'(r) for the WCA + Yukawa pair potential (positive = repulsive)."""
    r = np.asarray(r, dtype=np.float64)
    sr6 = (sigma_c / r) ** 6
    wca = np.where(r < 2.0 ** (1.0 / 6.0) * sigma_c, 24.0 * eps / r * (2.0 * sr6 * sr6 - sr6), 0.0)
    yuk = -eps * sigma_c * np.exp(-kappa * (r - sigma_c)) * (1.0 / (r * r) + kappa / r)
    return wca + yuk


def short_range_potential(r, eps, kappa, sigma_c):
    r = np.asarray(r, dtype=np.float64)
    sr6 = (sigma_c / r) ** 6
    wca = np.where(r < 2.0 ** (1.0 / 6.0) * sigma_c, 4.0 * eps * (sr6 * sr6 - sr6) + eps, 0.0)
    yuk = -eps * (sigma_c / r) * np.exp(-kappa * (r - sigma_c))
    return wca + yuk


def short_range_pairs(xy, pairs_i, pairs_j, eps, kappa, sigma_c, r_cut, L=None, radii=None):
    """Force on each i from its listed partners j (one row per listed pair):
    returns (n, 2) accumulated over the given ordered pairs (i <- j).
    L: periodic box side (minimum image); None = walls.  radii: polydisperse
    disks, the pair's length scale is then a_i + a_j (additive mixing)."""
    xy = np.asarray(xy, dtype=np.float64)
    d = xy[pairs_i] - xy[pairs_j]
    if L is not None:
        d = d - L * np.round(d / L)
    r = np.sqrt(np.einsum("ij,ij->i", d, d))
    sc = sigma_c if radii is None else radii[pairs_i] + radii[pairs_j]
    mag = np.where(r < r_cut, short_range_magnitude(r, eps, kappa, sc), 0.0)
    f = d * (mag / r)[:, None]
    out = np.zeros_like(xy)
    np.add.at(out, pairs_i, f)
    return out


def short_range(xy, eps, kappa, sigma_c, r_cut, L=None, radii=None):
    """All-pairs evaluation of the truncated short-range force (candidate
    pairs from a k-d tree, periodic when L is given; the law is above)."""
    xy = np.asarray(xy, dtype=np.float64)
    n = len(xy)
    from scipy.spatial import cKDTree  # neighbour search only; the force is below
    tree = cKDTree(xy) if L is None else cKDTree(np.mod(xy, L), boxsize=L)
    pairs = np.array(sorted(tree.query_pairs(r_cut * (1 + 1e-9))), dtype=np.int64).reshape(-1, 2)
    pi = np.concatenate([pairs[:, 0], pairs[:, 1]])
    pj = np.concatenate([pairs[:, 1], pairs[:, 0]])
    return short_range_pairs(xy, pi, pj, eps, kappa, sigma_c, r_cut, L, radii)
