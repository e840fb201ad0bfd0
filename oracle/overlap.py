"""Overlap correction -- oracle (test infrastructure).

Eq. (overlaps), Sec. 2.3: an overlapping pair (r_12 < sigma) is pushed apart
along n = (r_2 - r_1)/|r_12|: r_1' = r_1 - delta* n, r_2' = r_2 + delta* n with
the "bounce" value delta* = sigma - |r_12| (each disk moves by the full
overlap depth).

Algorithm 2, Sec. 4.4, run on the Delaunay edges: every edge with r < sigma
adds -delta* n to its first disk's displacement and +delta* n to its second's;
the displacements are summed (Jacobi style, not Strating's sequential order),
then each disk moves by its sum, truncated to length sigma/4 (the heuristic
cap against the oscillating instability of Fig. "overlaps"; the cap scales
the summed vector), and is reflected at the walls.  The pass repeats until
no pair is closer than sigma.

Which triangulation each pass uses: Algorithm 1 updates the triangulation
before correcting, so its last pass sees a stale triangulation.  The stopping test is read
as "no Delaunay edge of the *current* positions is
shorter than sigma": the closest pair of a point set is a Delaunay edge, so
that certifies that no pair anywhere overlaps.  The oracle therefore rebuilds
the triangulation from scratch before every pass.
"""
import numpy as np

from . import dynamics, geometry, periodic


# why a step was rejected (0 = it was not): a pair passed through each other
# (Sec. 4.3), or Algorithm 2 ran out of passes
REJ_NONE, REJ_REVERSAL, REJ_NOT_CONVERGED = 0, 1, 2


def real_edges(tris, n):
    e = geometry.edges(tris)
    return e[(e[:, 0] < n) & (e[:, 1] < n)]


def contact(sigma, radii, i, j):
    """Contact distance of pairs (i, j): sigma for equal disks; a_i + a_j for
    polydisperse disks (Sec. 2.3's extension)."""
    return sigma if radii is None else radii[i] + radii[j]


def caps(sigma, radii, n):
    """Sec. 4.4's truncation, "sigma/4 (half the particle radius)": half of
    each disk's own radius for polydisperse disks."""
    return np.full(n, sigma / 4.0) if radii is None else 0.5 * np.asarray(radii, dtype=np.float64)


def correction_pass(xy, E, sigma, a, L, radii=None):
    """One pass of Algorithm 2 over the edge list E (pairs i < j).
    Returns (new xy, overlapping pairs (k,2), capped mask, raw displacement).
    radii: one radius per disk (polydisperse), else every disk has radius a."""
    xy = np.asarray(xy, dtype=np.float64)
    i, j = E[:, 0], E[:, 1]
    d = xy[j] - xy[i]                          # r_j - r_i
    r = np.sqrt(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1])
    sg = contact(sigma, radii, i, j)
    hit = r < sg
    pairs = E[hit]
    disp = np.zeros_like(xy)
    if hit.any():
        nhat = d[hit] / r[hit][:, None]
        delta = ((sg[hit] if radii is not None else sigma) - r[hit])[:, None]
        np.add.at(disp, pairs[:, 0], -delta * nhat)
        np.add.at(disp, pairs[:, 1], delta * nhat)
    mag = np.sqrt(disp[:, 0] ** 2 + disp[:, 1] ** 2)
    cap = caps(sigma, radii, len(xy))
    capped = mag > cap
    scale = np.where(capped, cap / np.where(mag > 0, mag, 1.0), 1.0)
    new = xy + disp * scale[:, None]
    new = dynamics.reflect(new, a if radii is None else radii, L)
    return new, pairs, capped, disp


def reversed_edges(xy0, xy1, E):
    """Sec. 4.3 first criterion: r0_ij . r1_ij < 0 (the pair passed through
    each other), evaluated on edges E with before/after positions."""
    r0 = xy0[E[:, 1]] - xy0[E[:, 0]]
    r1 = xy1[E[:, 1]] - xy1[E[:, 0]]
    dot = r0[:, 0] * r1[:, 0] + r0[:, 1] * r1[:, 1]
    return E[dot < 0]


def correct(xy, L, a, max_iters=10000, tris=None, record=None, radii=None):
    """Iterate Algorithm 2 until no Delaunay edge is shorter than sigma = 2a
    (polydisperse: than a_i + a_j; a is then the largest radius, which lays
    out the ghost points).
    Returns (xy, tris of final positions, iterations that moved disks,
    total overlapping edges seen, rejection reason REJ_*: false when none)."""
    sigma = 2.0 * a
    n = len(xy)
    xy = np.asarray(xy, dtype=np.float64)
    it = 0
    total = 0
    while True:
        if tris is None:
            tris = geometry.delaunay(xy, L, a)
        E = real_edges(tris, n)
        new, pairs, capped, disp = correction_pass(xy, E, sigma, a, L, radii)
        if len(pairs) == 0:
            return xy, tris, it, total, REJ_NONE
        if record is not None:
            record.append({"pairs": pairs, "capped": capped, "disp": disp, "xy": xy})
        if len(reversed_edges(xy, new, E)):
            return xy, tris, it, total, REJ_REVERSAL
        total += len(pairs)
        it += 1
        xy = new
        tris = None
        if it >= max_iters:
            return xy, geometry.delaunay(xy, L, a), it, total, REJ_NOT_CONVERGED


def close_pairs(xy, sigma, chunk=512, radii=None):
    """Every pair i < j with |r_j - r_i| < sigma (polydisperse: < a_i + a_j),
    by brute force (chunked)."""
    xy = np.asarray(xy, dtype=np.float64)
    n = len(xy)
    out = []
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        d = xy[None, :, :] - xy[c0:c1, None, :]          # r_j - r_i
        r = np.sqrt(d[:, :, 0] * d[:, :, 0] + d[:, :, 1] * d[:, :, 1])
        lim = sigma if radii is None else radii[c0:c1, None] + radii[None, :]
        ii, jj = np.nonzero(r < lim)
        ii = ii + c0
        keep = jj > ii
        if keep.any():
            out.append(np.stack([ii[keep], jj[keep]], axis=1))
    return np.concatenate(out) if out else np.zeros((0, 2), dtype=np.int64)


def correct_allpairs(xy, L, a, max_iters=10000, record=None, radii=None):
    """Algorithm 2 over every pair of disks (the short-range path of Sec. 5,
    where the neighbour lists, not a triangulation, supply the pairs): each
    pass takes every pair closer than sigma, sums the displacements Jacobi
    style, caps each at sigma/4 and reflects, until no pair is closer than
    sigma.  Returns (xy, passes that moved disks, overlapping pairs seen,
    rejected flag)."""
    sigma = 2.0 * a
    xy = np.asarray(xy, dtype=np.float64)
    it = 0
    total = 0
    while True:
        E = close_pairs(xy, sigma, radii=radii)
        if len(E) == 0:
            return xy, it, total, REJ_NONE
        new, pairs, capped, disp = correction_pass(xy, E, sigma, a, L, radii)
        if record is not None:
            record.append({"pairs": pairs, "capped": capped, "disp": disp, "xy": xy})
        total += len(pairs)
        it += 1
        xy = new
        if it >= max_iters:
            return xy, it, total, REJ_NOT_CONVERGED



# ------------------------------------------------------ periodic box (Sec. 2.1)
# Pairs are torus edges keyed (u, w, sx, sy) (oracle.periodic): the pair
# vector is r_w + L s - r_u.  A disk that leaves the box re-enters at the
# other side (Algorithm 2's apply step "applying the periodic boundary
# conditions").


def correction_pass_periodic(xy, K, sigma, L, radii=None):
    """One pass of Algorithm 2 over torus edges K.  Returns (new positions
    before wrapping, overlapping keys, capped mask, raw displacement)."""
    xy = np.asarray(xy, dtype=np.float64)
    d = periodic.edge_vectors(xy, K, L)
    r = np.sqrt(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1])
    sg = contact(sigma, radii, K[:, 0], K[:, 1])
    hit = r < sg
    pairs = K[hit]
    disp = np.zeros_like(xy)
    if hit.any():
        nhat = d[hit] / r[hit][:, None]
        delta = ((sg[hit] if radii is not None else sigma) - r[hit])[:, None]
        np.add.at(disp, pairs[:, 0], -delta * nhat)
        np.add.at(disp, pairs[:, 1], delta * nhat)
    mag = np.sqrt(disp[:, 0] ** 2 + disp[:, 1] ** 2)
    cap = caps(sigma, radii, len(xy))
    capped = mag > cap
    scale = np.where(capped, cap / np.where(mag > 0, mag, 1.0), 1.0)
    return xy + disp * scale[:, None], pairs, capped, disp


def reversed_keys(xy0, xy1, K, L):
    """Sec. 4.3 reversal test on torus edges: xy1 are the positions after the
    move *before* wrapping, so r1 = r0 + (move of w) - (move of u)."""
    r0 = periodic.edge_vectors(xy0, K, L)
    r1 = periodic.edge_vectors(xy1, K, L)
    dot = r0[:, 0] * r1[:, 0] + r0[:, 1] * r1[:, 1]
    return K[dot < 0]


def correct_periodic(xy, L, a, max_iters=10000, record=None, radii=None):
    """Algorithm 2 over the edges of the torus Delaunay triangulation of the
    current positions until none is shorter than sigma (as correct()).
    Returns (xy, (tri, shift) of the final positions, passes, overlapping
    edges seen, rejection reason)."""
    sigma = 2.0 * a
    xy = np.asarray(xy, dtype=np.float64)
    it = 0
    total = 0
    while True:
        tri, sh = periodic.delaunay_torus(xy, L)
        K = periodic.edge_keys(tri, sh)
        new, pairs, capped, disp = correction_pass_periodic(xy, K, sigma, L, radii)
        if len(pairs) == 0:
            return xy, (tri, sh), it, total, REJ_NONE
        if record is not None:
            record.append({"pairs": pairs, "capped": capped, "disp": disp, "xy": xy})
        if len(reversed_keys(xy, new, K, L)):
            return xy, (tri, sh), it, total, REJ_REVERSAL
        total += len(pairs)
        it += 1
        xy = periodic.wrap(new, L)
        if it >= max_iters:
            return xy, periodic.delaunay_torus(xy, L), it, total, REJ_NOT_CONVERGED


def correct_allpairs_periodic(xy, L, a, max_iters=10000, record=None, radii=None):
    """correct_allpairs() in a periodic box (minimum-image pairs)."""
    sigma = 2.0 * a
    xy = np.asarray(xy, dtype=np.float64)
    it = 0
    total = 0
    while True:
        K = periodic.close_pairs(xy, sigma, L, radii=radii)
        if len(K) == 0:
            return xy, it, total, REJ_NONE
        new, pairs, capped, disp = correction_pass_periodic(xy, K, sigma, L, radii)
        if record is not None:
            record.append({"pairs": pairs, "capped": capped, "disp": disp, "xy": xy})
        total += len(pairs)
        it += 1
        xy = periodic.wrap(new, L)
        if it >= max_iters:
            return xy, it, total, REJ_NOT_CONVERGED
