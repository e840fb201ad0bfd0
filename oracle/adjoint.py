"""Differentiated rollout -- oracle (test infrastructure; no counterpart in the paper).

The paper has no gradients.  This module states, in plain FP64, the function
whose gradient the GPU adjoint returns, and computes that gradient two
independent ways.

The function.  A rollout of T steps of oracle.step (forces, Sec. 2.2;
Euler-Maruyama + self-propulsion, Eq. (integration) and Sec. 7; walls;
overlap correction, Algorithm 2) is recorded with its random and discrete
choices: the Philox noise, which walls reflected each move, and for every
correction pass its overlapping pairs, which disks were capped at sigma/4 and
which walls reflected them.  With those frozen the rollout is a smooth map of
the parameters p = (A00, A01, A10, A11, v0):
  y     = Refl_0( x + dt (F(x; A) + v0 e(theta)) + amp xi )
  z'    = Refl_j( z + cap_j(d_j(z)) )   for each pass j of the step,
  d_j(z)_u = -sum (sigma - r) n,  d_j(z)_w = +sum (sigma - r) n  over the pass's
            pairs (u, w), n = (z_w - z_u)/r, r = |z_w - z_u|;
  cap(d) = d, or (sigma/4) d/|d| for a capped disk.
Two losses of the final positions x_T:
  MSD:  L = sum_s (MSD_s - target)^2 with MSD_s the mean of |x_T - x_0|^2
        over species s;
  HIST: L = sum_b (h_b(x_T) - h_b(x_0))^2, the pair-distance histogram of
        the final positions against that of the start, with 32 Gaussian
        bins of width a/4 centred over [2a, 10a]:
        h_b(x) = (1/n) sum_{i<j} exp(-(r_ij - c_b)^2 / (2 s^2)),
        c_b = 2a + (b + 1/2) a/4, s = a/4 (walls: no images).

The gradient, (a) by forward-mode tangents: T = dx/dp (n, 2, 5) carried
through every move and pass with the chain rule, and (b) by central finite
differences of the frozen replay.  (b) pins (a).
"""
import math

import numpy as np

from . import _clib, dynamics, forces, geometry, noise, overlap
from .step import LAW_LONG

NPARAM = 5


# ---------------------------------------------------------------- walls

def reflect_flags(y, a, L):
    """dynamics.reflect with the reflections it made: flags per disk,
    bit 1 x < a, bit 2 x > L - a (after the first mirror), bit 4 / 8 for y."""
    lo, hi = a, L - a
    y = np.array(y, dtype=np.float64, copy=True)
    f = np.zeros(len(y), dtype=np.uint8)
    for c, (blo, bhi) in enumerate(((1, 2), (4, 8))):
        m = y[:, c] < lo
        y[m, c] = 2.0 * lo - y[m, c]
        f[m] |= blo
        m = y[:, c] > hi
        y[m, c] = 2.0 * hi - y[m, c]
        f[m] |= bhi
    return y, f


def apply_flags(y, f, a, L):
    """The recorded reflections, applied in the same order."""
    lo, hi = a, L - a
    y = np.array(y, dtype=np.float64, copy=True)
    for c, (blo, bhi) in enumerate(((1, 2), (4, 8))):
        m = (f & blo) != 0
        y[m, c] = 2.0 * lo - y[m, c]
        m = (f & bhi) != 0
        y[m, c] = 2.0 * hi - y[m, c]
    return y


def flag_signs(f):
    """d Refl / dy per component: -1 for an odd number of mirrors."""
    sx = np.where(((f & 1) != 0) ^ ((f & 2) != 0), -1.0, 1.0)
    sy = np.where(((f & 4) != 0) ^ ((f & 8) != 0), -1.0, 1.0)
    return np.stack([sx, sy], axis=1)


# ---------------------------------------------------------------- forces

def force(xy, species, A, threads=1):
    if len(xy) <= 2048:
        return forces.long_range_numpy(xy, species, A)
    return forces.long_range(xy, species, A, threads=threads)


def _c(a):
    import ctypes
    return a.ctypes.data_as(ctypes.c_void_p)


def force_jvp(xy, species, A, Tm, threads=1):
    """(dF/dx) t for every direction t: Tm (n, 2, K) -> (n, 2, K)."""
    xy = np.ascontiguousarray(np.asarray(xy, dtype=np.float64))
    n, _, K = Tm.shape
    x = np.ascontiguousarray(xy[:, 0])
    y = np.ascontiguousarray(xy[:, 1])
    s = np.ascontiguousarray(np.asarray(species, dtype=np.uint8))
    Af = np.ascontiguousarray(np.asarray(A, dtype=np.float64).reshape(4))
    tx = np.ascontiguousarray(Tm[:, 0, :].T)
    ty = np.ascontiguousarray(Tm[:, 1, :].T)
    ox = np.zeros((K, n))
    oy = np.zeros((K, n))
    _clib.lib().oracle_force_long_jvp(n, _c(x), _c(y), _c(s), _c(Af), K, _c(tx), _c(ty), _c(ox), _c(oy),
                                      int(threads))
    return np.stack([ox.T, oy.T], axis=1)


def force_dA(xy, species, threads=1):
    """dF/dA: (n, 2, 4), column 2a + b = dF/dA[a][b]."""
    xy = np.ascontiguousarray(np.asarray(xy, dtype=np.float64))
    n = len(xy)
    x = np.ascontiguousarray(xy[:, 0])
    y = np.ascontiguousarray(xy[:, 1])
    s = np.ascontiguousarray(np.asarray(species, dtype=np.uint8))
    S = np.zeros((n, 4))
    _clib.lib().oracle_force_long_dA(n, _c(x), _c(y), _c(s), _c(S), int(threads))
    out = np.zeros((n, 2, 4))
    si = (s != 0).astype(int)
    for b in range(2):
        for a in range(2):
            m = si == a
            out[m, 0, 2 * a + b] = S[m, 2 * b]
            out[m, 1, 2 * a + b] = S[m, 2 * b + 1]
    return out


# ---------------------------------------------------------------- record / replay

def record(xy0, th0, species, p, nsteps, step0=0, threads=1):
    """FP64 rollout of oracle.step with its frozen choices.  Raises if a step
    is rejected (Sec. 4.3) or the correction does not converge."""
    assert p.law == LAW_LONG
    xy = np.asarray(xy0, dtype=np.float64).copy()
    th = np.asarray(th0, dtype=np.float64).copy()
    sp = np.asarray(species)
    n = len(xy)
    ids = np.arange(n)
    sigma = 2.0 * p.a
    steps = []
    tris = geometry.delaunay(xy, p.L, p.a)
    for t in range(nsteps):
        F = force(xy, sp, p.alpha, threads)
        y_raw, th_new = dynamics.em_move(xy, th, F, ids, step0 + t, p.seed, p.D, p.Dr, p.v0, p.dt,
                                         p.replica, p.literal_amp)
        y, f0 = reflect_flags(y_raw, p.a, p.L)
        assert np.array_equal(y, dynamics.reflect(y_raw, p.a, p.L))
        if len(overlap.reversed_edges(xy, y, overlap.real_edges(tris, n))):
            raise RuntimeError("step %d rejected (pair reversal)" % (step0 + t))
        rec = []
        z, tris, iters, _, rej = overlap.correct(y, p.L, p.a, p.max_corr_iters, record=rec)
        if rej:
            raise RuntimeError("step %d rejected" % (step0 + t))
        passes = []
        for k, r in enumerate(rec):
            mag = np.sqrt(r["disp"][:, 0] ** 2 + r["disp"][:, 1] ** 2)
            scale = np.where(r["capped"], (sigma / 4.0) / np.where(mag > 0, mag, 1.0), 1.0)
            _, fj = reflect_flags(r["xy"] + r["disp"] * scale[:, None], p.a, p.L)
            passes.append({"pairs": r["pairs"].copy(), "capped": r["capped"].copy(), "flags": fj})
        steps.append({"th": th.copy(), "flags": f0, "passes": passes})
        xy, th = z, th_new
    return {"x0": np.asarray(xy0, dtype=np.float64).copy(), "th0": np.asarray(th0, np.float64).copy(),
            "xT": xy, "steps": steps, "step0": step0}


def pass_disp(z, pairs, sigma):
    """d_j(z): the summed pair displacements of one pass (Algorithm 2)."""
    d = np.zeros_like(z)
    if len(pairs) == 0:
        return d
    u, w = pairs[:, 0], pairs[:, 1]
    v = z[w] - z[u]
    r = np.sqrt(v[:, 0] ** 2 + v[:, 1] ** 2)
    g = (sigma - r)[:, None] * v / r[:, None]
    np.add.at(d, u, -g)
    np.add.at(d, w, g)
    return d


def capped_move(d, capped, sigma):
    mag = np.sqrt(d[:, 0] ** 2 + d[:, 1] ** 2)
    scale = np.where(capped, (sigma / 4.0) / np.where(mag > 0, mag, 1.0), 1.0)
    return d * scale[:, None]


def replay(rec, species, p, alpha=None, v0=None, threads=1):
    """The frozen map: final positions for the force table `alpha` and speed
    `v0` (None = p's)."""
    A = p.alpha if alpha is None else alpha
    v = p.v0 if v0 is None else v0
    sigma = 2.0 * p.a
    x = rec["x0"].copy()
    n = len(x)
    ids = np.arange(n)
    for t, st in enumerate(rec["steps"]):
        F = force(x, species, A, threads)
        y_raw, _ = dynamics.em_move(x, st["th"], F, ids, rec["step0"] + t, p.seed, p.D, p.Dr, v, p.dt,
                                    p.replica, p.literal_amp)
        x = apply_flags(y_raw, st["flags"], p.a, p.L)
        for ps in st["passes"]:
            d = pass_disp(x, ps["pairs"], sigma)
            x = apply_flags(x + capped_move(d, ps["capped"], sigma), ps["flags"], p.a, p.L)
    return x


# ---------------------------------------------------------------- loss

def msd_loss(xT, x0, species, target):
    s = (np.asarray(species) != 0).astype(int)
    L = 0.0
    for k in (0, 1):
        m = s == k
        if m.any():
            msd = float(np.mean(np.sum((xT[m] - x0[m]) ** 2, axis=1)))
            L += (msd - target) ** 2
    return L


def msd_loss_grad(xT, x0, species, target):
    """dL/dx_T, (n, 2)."""
    s = (np.asarray(species) != 0).astype(int)
    g = np.zeros_like(xT)
    for k in (0, 1):
        m = s == k
        if m.any():
            nk = int(m.sum())
            msd = float(np.mean(np.sum((xT[m] - x0[m]) ** 2, axis=1)))
            g[m] = 2.0 * (msd - target) * 2.0 * (xT[m] - x0[m]) / nk
    return g


HIST_BINS = 32


def hist_centres(a):
    """c_b = 2a + (b + 1/2) a/4, b = 0..31: 32 bins of width a/4 covering [2a, 10a]."""
    return 2.0 * a + (np.arange(HIST_BINS) + 0.5) * (0.25 * a)


def pair_histogram(x, a):
    """h_b = (1/n) sum over pairs i < j of exp(-(r_ij - c_b)^2 / (2 s^2)), s = a/4."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    c = hist_centres(a)
    s2 = (0.25 * a) ** 2
    h = np.zeros(HIST_BINS)
    for i in range(n - 1):
        d = x[i + 1:] - x[i]
        r = np.sqrt(d[:, 0] ** 2 + d[:, 1] ** 2)
        u = r[:, None] - c[None, :]
        h += np.exp(-u * u / (2.0 * s2)).sum(axis=0)
    return h / n


def hist_loss(xT, x0, a):
    return float(np.sum((pair_histogram(xT, a) - pair_histogram(x0, a)) ** 2))


def hist_loss_grad(xT, x0, a):
    """dL/dx_T, (n, 2): dL/dr_ij = sum_b 2 (h_b - h0_b)/n * dK/du(r_ij - c_b),
    K(u) = exp(-u^2 / (2 s^2)), dK/du = -(u / s^2) K(u), and dr_ij/dx_i = (x_i - x_j)/r_ij."""
    xT = np.asarray(xT, dtype=np.float64)
    n = len(xT)
    c = hist_centres(a)
    s2 = (0.25 * a) ** 2
    wb = 2.0 * (pair_histogram(xT, a) - pair_histogram(x0, a)) / n
    g = np.zeros_like(xT)
    for i in range(n - 1):
        d = xT[i] - xT[i + 1:]
        r = np.sqrt(d[:, 0] ** 2 + d[:, 1] ** 2)
        u = r[:, None] - c[None, :]
        dLdr = (wb[None, :] * (-u / s2) * np.exp(-u * u / (2.0 * s2))).sum(axis=1)
        v = (dLdr / r)[:, None] * d
        g[i] += v.sum(axis=0)
        g[i + 1:] -= v
    return g


def loss_value(xT, x0, species, target, a, loss="msd"):
    if loss == "msd":
        return msd_loss(xT, x0, species, target)
    if loss == "hist":
        return hist_loss(xT, x0, a)
    raise ValueError(loss)


def loss_grad(xT, x0, species, target, a, loss="msd"):
    if loss == "msd":
        return msd_loss_grad(xT, x0, species, target)
    if loss == "hist":
        return hist_loss_grad(xT, x0, a)
    raise ValueError(loss)


# ---------------------------------------------------------------- gradients

def _pair_G(v, sigma):
    """d[(sigma - |v|) v/|v|]/dv = (sigma/r)(I - n n^T) - I, per pair: (m, 2, 2)."""
    r = np.sqrt(v[:, 0] ** 2 + v[:, 1] ** 2)
    nn = v / r[:, None]
    I = np.eye(2)[None]
    P = I - nn[:, :, None] * nn[:, None, :]
    return (sigma / r)[:, None, None] * P - I


def tangent_gradient(rec, species, p, target, threads=1, loss="msd"):
    """dL/dp, p = (A00, A01, A10, A11, v0), by forward-mode tangents along the
    frozen map.  Returns (grad (5,), final positions)."""
    Tm, x = tangent_map(rec, species, p, threads)
    g = loss_grad(x, rec["x0"], species, target, p.a, loss)
    return np.einsum("ia,iak->k", g, Tm), x


def tangent_map(rec, species, p, threads=1):
    """dx_T/dp, (n, 2, 5), carried forward through every move and pass of the
    frozen map; returns (dx_T/dp, x_T)."""
    sigma = 2.0 * p.a
    sp = np.asarray(species)
    x = rec["x0"].copy()
    n = len(x)
    ids = np.arange(n)
    Tm = np.zeros((n, 2, NPARAM))
    for t, st in enumerate(rec["steps"]):
        F = force(x, sp, p.alpha, threads)
        # move: dy = T + dt (dF/dx T + dF/dA [cols 0..3] + e(theta) [col 4])
        dT = force_jvp(x, sp, p.alpha, Tm, threads)
        dT[:, :, 0:4] += force_dA(x, sp, threads)
        th = st["th"]
        dT[:, 0, 4] += np.cos(th)
        dT[:, 1, 4] += np.sin(th)
        Tm = Tm + p.dt * dT
        y_raw, _ = dynamics.em_move(x, th, F, ids, rec["step0"] + t, p.seed, p.D, p.Dr, p.v0, p.dt,
                                    p.replica, p.literal_amp)
        x = apply_flags(y_raw, st["flags"], p.a, p.L)
        Tm = Tm * flag_signs(st["flags"])[:, :, None]
        for ps in st["passes"]:
            pairs = ps["pairs"]
            d = pass_disp(x, pairs, sigma)
            # tangent of d: (Dd T)_u = sum G (T_u - T_w), (Dd T)_w = sum G (T_w - T_u)
            Td = np.zeros_like(Tm)
            if len(pairs):
                u, w = pairs[:, 0], pairs[:, 1]
                G = _pair_G(x[w] - x[u], sigma)
                gt = np.einsum("mab,mbk->mak", G, Tm[u] - Tm[w])
                np.add.at(Td, u, gt)
                np.add.at(Td, w, -gt)
            # cap: (s/|d|)(I - dhat dhat^T) for capped disks
            c = ps["capped"]
            if c.any():
                dc = d[c]
                m = np.sqrt(dc[:, 0] ** 2 + dc[:, 1] ** 2)
                dh = dc / m[:, None]
                P = np.eye(2)[None] - dh[:, :, None] * dh[:, None, :]
                Td[c] = np.einsum("mab,mbk->mak", ((sigma / 4.0) / m)[:, None, None] * P, Td[c])
            x = apply_flags(x + capped_move(d, c, sigma), ps["flags"], p.a, p.L)
            Tm = (Tm + Td) * flag_signs(ps["flags"])[:, :, None]
    return Tm, x


def fd_gradient(rec, species, p, target, h=1e-4, threads=1, loss="msd"):
    """dL/dp by central differences of the frozen replay, step h."""
    base = np.array(list(p.alpha) + [p.v0], dtype=np.float64)
    out = np.zeros(NPARAM)
    for k in range(NPARAM):
        vals = []
        for sgn in (1.0, -1.0):
            q = base.copy()
            q[k] += sgn * h
            xT = replay(rec, species, p, alpha=tuple(q[:4]), v0=q[4], threads=threads)
            vals.append(loss_value(xT, rec["x0"], species, target, p.a, loss))
        out[k] = (vals[0] - vals[1]) / (2.0 * h)
    return out
