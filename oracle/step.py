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

Periodic box (Params.periodic, Sec. 2.1): minimum-image forces, moves that
wrap, and the torus triangulation of oracle.periodic.

Polydisperse disks (Params.radii, Sec. 2.3 "radii [that] do not differ too
much"): a pair overlaps when closer than a_i + a_j, each disk of an
overlapping pair moves a_i + a_j - r, a disk's summed displacement is
truncated at half its own radius, centres are reflected a_i from the walls,
and the short-range law takes a_i + a_j as its length scale.

Rejected moves (Sec. 4.3): when a pair passes through each other "the last
positions are discarded and integration is repeated with a lower dt".  With
Params.max_halvings = H > 0 a rejected move is replaced by two moves of half
its length, each with forces at its own start and fresh noise (counter word
oracle.philox.substep_tag(node), pieces numbered as a binary heap from the
whole step, node 1); a half that is rejected in turn is halved again, down to
dt / 2^H.  If a piece of length dt / 2^H is rejected the whole step is
rejected and the state is left as it was.
"""
from dataclasses import dataclass

import numpy as np

from . import dynamics, forces, geometry, overlap, periodic, philox

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
    max_halvings: int = 0
    periodic: bool = False
    radii: object = None     # polydisperse disks: one radius per disk (a is then the largest)


def compute_forces(xy, species, p: Params, threads=1):
    Lp = p.L if p.periodic else None
    if p.law == LAW_LONG:
        if len(xy) <= 4096:
            return forces.long_range_numpy(xy, species, p.alpha, L=Lp)
        return forces.long_range(xy, species, p.alpha, threads=threads, L=Lp)
    if p.law == LAW_SHORT:
        return forces.short_range(xy, p.eps, p.kappa, 2.0 * p.a, p.r_cut, L=Lp, radii=_radii(p))
    return np.zeros_like(np.asarray(xy, dtype=np.float64))


def _radii(p):
    return None if p.radii is None else np.asarray(p.radii, dtype=np.float64)


def _piece(xy, theta, species, step_index, p: Params, ids, tris, F, threads, record, pairs_from,
           node):
    """One move of length dt / 2^level (level = depth of `node` in the heap
    numbering) from xy with the noise of that node, then the validity test and
    the overlap correction."""
    n = len(xy)
    if F is None:
        F = compute_forces(xy, species, p, threads)
    dt = p.dt / float(2 ** (int(node).bit_length() - 1))
    if p.periodic:
        return _piece_periodic(xy, theta, F, step_index, p, ids, tris, record, pairs_from, node, dt)
    rad = _radii(p)
    new, th = dynamics.em_step(xy, theta, F, ids, step_index, p.seed, p.D, p.Dr, p.v0, dt,
                               p.a if rad is None else rad, p.L, p.replica, p.literal_amp,
                               philox.substep_tag(node))
    if pairs_from == "allpairs":
        out, iters, pairs, rej = overlap.correct_allpairs(new, p.L, p.a, p.max_corr_iters,
                                                          record=record, radii=rad)
        return dict(xy=out, theta=th, tris=None, corr_iters=iters, overlap_pairs=pairs,
                    rejected=rej, F=F, xy_em=new)
    if tris is None:
        tris = geometry.delaunay(xy, p.L, p.a)
    E0 = overlap.real_edges(tris, n)
    if len(overlap.reversed_edges(xy, new, E0)):
        return dict(xy=xy, theta=np.asarray(theta, np.float64), tris=tris, corr_iters=0,
                    overlap_pairs=0, rejected=overlap.REJ_REVERSAL, F=F)
    out, tris1, iters, pairs, rej = overlap.correct(new, p.L, p.a, p.max_corr_iters,
                                                    record=record, radii=rad)
    return dict(xy=out, theta=th, tris=tris1, corr_iters=iters, overlap_pairs=pairs,
                rejected=rej, F=F, xy_em=new)


def _piece_periodic(xy, theta, F, step_index, p, ids, tris, record, pairs_from, node, dt):
    """_piece() in a periodic box (Sec. 2.1): the move wraps instead of
    reflecting, pair vectors take their minimum image, and the triangulation
    is the torus one (tris = (tri, shift), oracle.periodic)."""
    moved, th = dynamics.em_move(xy, theta, F, ids, step_index, p.seed, p.D, p.Dr, p.v0, dt,
                                 p.replica, p.literal_amp, philox.substep_tag(node))
    new = periodic.wrap(moved, p.L)
    rad = _radii(p)
    if pairs_from == "allpairs":
        out, iters, pairs, rej = overlap.correct_allpairs_periodic(new, p.L, p.a, p.max_corr_iters,
                                                                   record=record, radii=rad)
        return dict(xy=out, theta=th, tris=None, corr_iters=iters, overlap_pairs=pairs,
                    rejected=rej, F=F, xy_em=new)
    if tris is None:
        tris = periodic.delaunay_torus(xy, p.L)
    K0 = periodic.edge_keys(*tris)
    if len(overlap.reversed_keys(xy, moved, K0, p.L)):
        return dict(xy=xy, theta=np.asarray(theta, np.float64), tris=tris, corr_iters=0,
                    overlap_pairs=0, rejected=overlap.REJ_REVERSAL, F=F)
    out, tris1, iters, pairs, rej = overlap.correct_periodic(new, p.L, p.a, p.max_corr_iters,
                                                             record=record, radii=rad)
    return dict(xy=out, theta=th, tris=tris1, corr_iters=iters, overlap_pairs=pairs,
                rejected=rej, F=F, xy_em=new)


def step(xy, theta, species, step_index, p: Params, ids=None, tris=None, F=None,
         threads=1, record=None, pairs_from="delaunay"):
    """Returns dict(xy, theta, tris, corr_iters, overlap_pairs, rejected, F,
    substeps, halvings).

    pairs_from="allpairs": the short-range path of Sec. 5, whose neighbour lists
    supply the pairs of Algorithm 2: every pair closer than sigma is corrected,
    no triangulation is involved (tris is None, no reversal test).

    substeps: pieces shorter than dt that completed (0 when the whole step was
    accepted); halvings: rejected pieces that were replaced by their halves."""
    xy = np.asarray(xy, dtype=np.float64)
    ids = np.arange(len(xy)) if ids is None else np.asarray(ids)
    r = _piece(xy, theta, species, step_index, p, ids, tris, F, threads, record, pairs_from, 1)
    r["substeps"], r["halvings"] = 0, 0
    if r["rejected"] != overlap.REJ_REVERSAL or p.max_halvings <= 0:
        return r
    # Sec. 4.3: discard the move, integrate again with half the time step
    count = {"substeps": 0, "halvings": 0, "corr_iters": 0, "overlap_pairs": 0}

    def halves(x, th, tr, node, depth_left):
        count["halvings"] += 1
        for child in (2 * node, 2 * node + 1):
            q = _piece(x, th, species, step_index, p, ids, tr, None, threads, None, pairs_from, child)
            if q["rejected"] == overlap.REJ_REVERSAL and depth_left > 1:
                ok, x, th, tr = halves(x, th, tr, child, depth_left - 1)
                if not ok:
                    return False, x, th, tr
                continue
            if q["rejected"]:
                return False, x, th, tr
            count["substeps"] += 1
            count["corr_iters"] += q["corr_iters"]
            count["overlap_pairs"] += q["overlap_pairs"]
            x, th, tr = q["xy"], q["theta"], q["tris"]
        return True, x, th, tr

    ok, x, th, tr = halves(xy, np.asarray(theta, np.float64), tris, 1, p.max_halvings)
    if not ok:
        r.update(count)
        return r
    return dict(xy=x, theta=th, tris=tr, corr_iters=count["corr_iters"],
                overlap_pairs=count["overlap_pairs"], rejected=overlap.REJ_NONE, F=r["F"],
                substeps=count["substeps"], halvings=count["halvings"])
