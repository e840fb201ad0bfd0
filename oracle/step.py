"""One full time step -- oracle (test infrastructure).

Algorithm 1 (Sec. 4.1) for one step t -> t + dt:
  1. forces at the step's start positions (Sec. 2.2; all pairs for the
     long-range law, truncated pairs for the short-range law);
  2. Euler-Maruyama + active self-propulsion + walls (Eq. (integration),
     Sec. 7), noise from the Philox stream of this step;
  3. the first validity criterion of Sec. 4.3: if any Delaunay edge of the
     start positions has r0 . r1 < 0 the step is rejected;
  4. overlap correction (Algorithm 2, Sec. 4.4) until no Delaunay edge of the
     current positions is shorter than sigma (see oracle.overlap).
Steps 3-4 need the Delaunay triangulation, which the oracle builds from
scratch; inverted-triangle repair and edge flips (Sec. 4.3) are how the GPU
*maintains* that triangulation, so they have no counterpart here beyond the
final triangulation itself.
"""
from dataclasses import dataclass

import numpy as np

from . import dynamics, forces, geometry, overlap

LAW_NONE, LAW_LONG, LAW_SHORT = 0, 1, 2


@dataclass
class Params:
    L: float
    a: float = 1.0
    law: int = LAW_LONG
    alpha: tuple = (0.0, 0.0, 0.0, 0.0)
    eps: float = 1.0
    kappa: float = 1.0
    r_cut: float = 5.0
    D: float = 1.0
    Dr: float = 0.0
    v0: float = 0.0
    dt: float = 1e-4
    seed: int = 0
    replica: int = 0
    max_corr_iters: int = 10000
    literal_amp: bool = False


def compute_forces(xy, species, p: Params, threads=1):
    if p.law == LAW_LONG:
        if len(xy) <= 4096:
            return forces.long_range_numpy(xy, species, p.alpha)
        return forces.long_range(xy, species, p.alpha, threads=threads)
    if p.law == LAW_SHORT:
        return forces.short_range(xy, p.eps, p.kappa, 2.0 * p.a, p.r_cut)
    return np.zeros_like(np.asarray(xy, dtype=np.float64))


def step(xy, theta, species, step_index, p: Params, ids=None, tris=None, F=None,
         threads=1, record=None, pairs_from="delaunay"):
    """Returns dict(xy, theta, tris, corr_iters, overlap_pairs, rejected, F).

    pairs_from="allpairs": the short-range path of Sec. 5, whose neighbour lists
    supply the pairs of Algorithm 2: every pair closer than sigma is corrected,
    no triangulation is involved (tris is None, no reversal test)."""
    xy = np.asarray(xy, dtype=np.float64)
    n = len(xy)
    ids = np.arange(n) if ids is None else np.asarray(ids)
    if F is None:
        F = compute_forces(xy, species, p, threads)
    new, th = dynamics.em_step(xy, theta, F, ids, step_index, p.seed, p.D, p.Dr, p.v0, p.dt,
                               p.a, p.L, p.replica, p.literal_amp)
    if pairs_from == "allpairs":
        out, iters, pairs, rej = overlap.correct_allpairs(new, p.L, p.a, p.max_corr_iters,
                                                              record=record)
        return dict(xy=out, theta=th, tris=None, corr_iters=iters, overlap_pairs=pairs,
                    rejected=rej, F=F, xy_em=new)
    if tris is None:
        tris = geometry.delaunay(xy, p.L)
    E0 = overlap.real_edges(tris, n)
    if len(overlap.reversed_edges(xy, new, E0)):
        return dict(xy=xy, theta=np.asarray(theta, np.float64), tris=tris, corr_iters=0,
                    overlap_pairs=0, rejected=True, F=F)
    out, tris1, iters, pairs, rej = overlap.correct(new, p.L, p.a, p.max_corr_iters,
                                                    record=record)
    return dict(xy=out, theta=th, tris=tris1, corr_iters=iters, overlap_pairs=pairs,
                rejected=rej, F=F, xy_em=new)
