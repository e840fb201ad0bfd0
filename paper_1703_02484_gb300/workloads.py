"""Seeded synthetic workloads: system sizes, parameters and initial states.

This module only *generates inputs*; it holds none of the time-stepping
arithmetic, so both the CUDA path and the CPU oracle can take their inputs
from it without sharing any of the method's code.

Sizes follow the paper's performance set-up (Sec. 6): the box side is chosen
from the number of disks N and the area fraction rho as
L(N) = sqrt(N * pi * (sigma/2)^2 / rho), with sigma = 2a the disk diameter.
The paper's own parameter table is not available, so five synthetic
configurations stand in for its c0..c4 workloads (all in a square box with
reflecting walls):

  c1      N=1024 passive disks, rho=0.30, one species, long-range alpha=0.1, FP64
  c2      N=16384 active disks, rho=0.30, two species, non-reciprocal 2x2 alpha
  c3      N=1048576 active disks, rho=0.50, WCA + Yukawa short-range law
  c4      256 replicas, N log-uniform in [512, 65536], rho in [0.30, 0.50]
  c5      N=4096 active disks, rho=0.35, c2's 2x2 alpha (rollout gradients)
  n1e5    N=100000, rho=0.30, c2's law (the throughput workload)

Initial states: non-overlapping centres in [a, L-a]^2 by random sequential
addition (RSA) at rho <= 0.35; at higher rho by the paper's own start
(Sec. 4.1): a triangular lattice with N* >= N sites from which N are
reservoir-sampled, each site jittered so the points are in general position.
Species are an exact 50/50 split by a seeded permutation; theta ~ U[0, 2*pi).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

LAW_NONE = 0
LAW_LONG = 1      # alpha * rhat / r^2, all pairs
LAW_SHORT = 2     # WCA + Yukawa, truncated at r_cut, Verlet lists


def box_side(n: int, rho: float, a: float = 1.0) -> float:
    """L(N) = sqrt(N pi (sigma/2)^2 / rho), paper Sec. 6 (sigma/2 = a)."""
    return math.sqrt(n * math.pi * a * a / rho)


@dataclass
class Config:
    name: str
    n: int
    rho: float
    law: int
    alpha: tuple = (0.0, 0.0, 0.0, 0.0)   # A[s_i][s_j] row-major: on s_i from s_j
    n_species: int = 1
    eps: float = 1.0
    kappa: float = 1.0
    r_cut: float = 5.0
    skin: float = 0.6
    D: float = 1.0
    Dr: float = 0.0
    v0: float = 0.0
    dt: float = 1e-4
    seed: int = 0
    precision: int = 0          # 0 = FP32 force/integration increments, 1 = FP64
    steps: int = 100
    a: float = 1.0
    extra: dict = field(default_factory=dict)

    @property
    def L(self) -> float:
        return box_side(self.n, self.rho, self.a)

    def with_n(self, n: int) -> "Config":
        return replace(self, n=n)


ALPHA_C2 = (0.05, 0.2, -0.1, 0.05)   # AA, AB (on A from B), BA (on B from A), BB

CONFIGS = {
    "c1": Config("c1", 1024, 0.30, LAW_LONG, alpha=(0.1, 0.1, 0.1, 0.1), n_species=1,
                 D=1.0, dt=1e-4, seed=0, precision=1, steps=100),
    "c2": Config("c2", 16384, 0.30, LAW_LONG, alpha=ALPHA_C2, n_species=2,
                 D=1.0, Dr=0.5, v0=1.0, dt=1e-4, seed=1, steps=1000),
    "c3": Config("c3", 1048576, 0.50, LAW_SHORT, n_species=1, eps=1.0, kappa=1.0,
                 r_cut=5.0, skin=0.6, D=1.0, Dr=0.2, v0=0.5, dt=5e-5, seed=2, steps=1000),
    "c5": Config("c5", 4096, 0.35, LAW_LONG, alpha=ALPHA_C2, n_species=2,
                 D=1.0, Dr=0.5, v0=1.0, dt=1e-4, seed=4, steps=200),
    "n1e5": Config("n1e5", 100000, 0.30, LAW_LONG, alpha=ALPHA_C2, n_species=2,
                   D=1.0, Dr=0.5, v0=1.0, dt=1e-4, seed=100, steps=100),
}


def _rsa(n: int, L: float, a: float, rng: np.random.Generator, max_tries: int = 200000):
    """Random sequential addition of n disks of radius a in [a, L-a]^2 (cell grid)."""
    lo, hi = a, L - a
    d2min = (2.0 * a) ** 2
    cs = 2.0 * a
    nc = max(1, int(math.floor(L / cs)))
    cs = L / nc
    cells = {}
    out = np.empty((n, 2), dtype=np.float64)
    k = 0
    batch = 4096
    buf = rng.uniform(lo, hi, size=(batch, 2))
    bi = 0
    tries = 0
    while k < n:
        if bi == batch:
            buf = rng.uniform(lo, hi, size=(batch, 2))
            bi = 0
        x, y = float(buf[bi, 0]), float(buf[bi, 1])
        bi += 1
        tries += 1
        if tries > max_tries + 50 * n:
            raise RuntimeError("RSA did not place %d disks (placed %d)" % (n, k))
        cx, cy = int(x / cs), int(y / cs)
        ok = True
        for gx in (cx - 1, cx, cx + 1):
            for gy in (cy - 1, cy, cy + 1):
                lst = cells.get((gx, gy))
                if lst is None:
                    continue
                for (px, py) in lst:
                    if (px - x) ** 2 + (py - y) ** 2 < d2min:
                        ok = False
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            cells.setdefault((cx, cy), []).append((x, y))
            out[k, 0] = x
            out[k, 1] = y
            k += 1
    return out


def _lattice(n: int, L: float, a: float, rng: np.random.Generator):
    """Jittered triangular lattice with N* >= n sites, n of them reservoir-sampled."""
    lo, hi = a, L - a
    W = hi - lo
    # spacing s so that a triangular lattice over [lo, hi]^2 has at least n sites
    s = math.sqrt(2.0 * W * W / (math.sqrt(3.0) * n))
    while True:
        nx = int(math.floor(W / s)) + 1
        ny = int(math.floor(W / (s * math.sqrt(3.0) / 2.0))) + 1
        xs, ys = [], []
        for r in range(ny):
            y = lo + r * s * math.sqrt(3.0) / 2.0
            off = 0.5 * s if (r % 2) else 0.0
            for c in range(nx):
                x = lo + off + c * s
                if x <= hi and y <= hi:
                    xs.append(x)
                    ys.append(y)
        if len(xs) >= n:
            break
        s *= 0.995
    if s < 2.0 * a * 1.01:
        raise RuntimeError("area fraction too high for the lattice start")
    pts = np.stack([np.array(xs), np.array(ys)], axis=1)
    # reservoir sampling (Vitter's algorithm R) of n of the N* sites
    res = np.arange(n)
    for i in range(n, len(pts)):
        j = int(rng.integers(0, i + 1))
        if j < n:
            res[j] = i
    pts = pts[np.sort(res)]
    # jitter inside a disk of radius jr so pairs stay >= 2a apart and the
    # points are in general position (no four cocircular)
    jr = 0.45 * (s - 2.0 * a)
    rr = jr * np.sqrt(rng.uniform(0.0, 1.0, size=n))
    ph = rng.uniform(0.0, 2.0 * math.pi, size=n)
    off = np.stack([rr * np.cos(ph), rr * np.sin(ph)], axis=1)
    # an offset that would leave the box is mirrored, so every site is jittered
    off = np.where((pts + off < lo) | (pts + off > hi), -off, off)
    return pts + off


def initial_positions(n: int, L: float, a: float, rho: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(np.random.PCG64([seed, 0x504C4143]))
    if rho <= 0.35:
        return _rsa(n, L, a, rng)
    return _lattice(n, L, a, rng)


def initial_state(cfg: Config, seed: int | None = None, n: int | None = None):
    """(xy (n,2) f64, species (n,) u8, theta (n,) f32) for a configuration."""
    seed = cfg.seed if seed is None else seed
    n = cfg.n if n is None else n
    L = box_side(n, cfg.rho, cfg.a)
    xy = initial_positions(n, L, cfg.a, cfg.rho, seed)
    rng = np.random.default_rng(np.random.PCG64([seed, 0x53504543]))
    species = np.zeros(n, dtype=np.uint8)
    if cfg.n_species == 2:
        perm = rng.permutation(n)
        species[perm[n // 2:]] = 1
    theta = rng.uniform(0.0, 2.0 * math.pi, size=n).astype(np.float32)
    return xy, species, theta


def replica_table(R: int = 256, seed: int = 3, n_lo: int = 512, n_hi: int = 65536):
    """Per-replica (n, rho, law) for the batched workload: N log-uniform in
    [n_lo, n_hi], rho ~ U[0.30, 0.50], law alternating long (even) / short (odd)."""
    rng = np.random.default_rng(np.random.PCG64([seed, 0x52455053]))
    ns = np.rint(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=R))).astype(np.int64)
    rhos = rng.uniform(0.30, 0.50, size=R)
    laws = np.where(np.arange(R) % 2 == 0, LAW_LONG, LAW_SHORT)
    return ns, rhos, laws


def near_contact_state(n: int, L: float, a: float, seed: int, gap: float = 0.02,
                       frac: float = 0.3, rho: float | None = None):
    """RSA start in which a fraction of disks is moved next to a neighbour,
    leaving a surface gap in (0, gap]: a start with many near-contacts, so the
    first step already has overlaps to correct (a stand-in for a state taken
    later in a run)."""
    rng = np.random.default_rng(np.random.PCG64([seed, 0x4E454152]))
    if rho is not None and rho > 0.35:
        xy = _lattice(n, L, a, rng)
    else:
        xy = _rsa(n, L, a, rng)
    cs = 6.0 * a
    nc = max(1, int(L // cs))
    cs = L / nc
    grid = {}

    def key(p):
        return (int(p[0] // cs), int(p[1] // cs))

    for k in range(n):
        grid.setdefault(key(xy[k]), set()).add(k)

    def near(p, rad):
        cx, cy = key(p)
        out = []
        for gx in (cx - 1, cx, cx + 1):
            for gy in (cy - 1, cy, cy + 1):
                for k in grid.get((gx, gy), ()):
                    d = math.hypot(xy[k, 0] - p[0], xy[k, 1] - p[1])
                    if d < rad:
                        out.append((d, k))
        return out

    for i in rng.permutation(n)[: int(frac * n)]:
        i = int(i)
        nb = [t for t in near(xy[i], cs) if t[1] != i]
        if not nb:
            continue
        _, j = min(nb)
        v = xy[i] - xy[j]
        r = math.hypot(v[0], v[1])
        cand = xy[j] + v / r * (2.0 * a + rng.uniform(0.1, 1.0) * gap)
        if not (a <= cand[0] <= L - a and a <= cand[1] <= L - a):
            continue
        if any(d < 2.0 * a for d, k in near(cand, 2.0 * a) if k != i):
            continue
        grid[key(xy[i])].discard(i)
        xy[i] = cand
        grid.setdefault(key(cand), set()).add(i)
    return xy


def batch_configs(R: int = 256, seed: int = 3, n_lo: int = 512, n_hi: int = 65536):
    """The batched workload: R replicas, N log-uniform in [n_lo, n_hi], area
    fraction U[0.30, 0.50]; even replicas take c1's long-range law (alpha 0.1,
    passive, dt 1e-4), odd replicas c3's short-range law (WCA + Yukawa, ABP
    v0 0.5, D_r 0.2, dt 5e-5); all FP32.  Replica r draws its noise from key
    (seed, r)."""
    ns, rhos, laws = replica_table(R, seed, n_lo, n_hi)
    out = []
    for r in range(R):
        base = CONFIGS["c1"] if laws[r] == LAW_LONG else CONFIGS["c3"]
        out.append(replace(base, name="c4r%d" % r, n=int(ns[r]), rho=float(rhos[r]), seed=seed,
                           precision=0, extra={"replica": r}))
    return out


# ---------------------------------------------------------------- polydisperse disks

def poly_radii(n: int, a_max: float = 1.0, ratio: float = 1.3, seed: int = 0) -> np.ndarray:
    """Radii drawn uniformly from [a_max / ratio, a_max] (slightly polydisperse
    disks, largest radius a_max)."""
    rng = np.random.default_rng(np.random.PCG64([seed, 0x52414449]))
    return rng.uniform(a_max / ratio, a_max, size=n)


def poly_positions(radii, L: float, seed: int, near_frac: float = 0.0, gap: float = 0.02):
    """Random sequential addition of disks with the given radii in the box
    [0, L]^2 (centre i in [a_i, L - a_i], pairs at least a_i + a_j apart); with
    near_frac > 0 that fraction of the disks is then moved next to its nearest
    neighbour, leaving a surface gap in (0, gap] (a start with overlaps to
    correct after the first move)."""
    radii = np.asarray(radii, dtype=np.float64)
    n = len(radii)
    rng = np.random.default_rng(np.random.PCG64([seed, 0x504F4C59]))
    amax = float(radii.max())
    cs = 2.0 * amax
    nc = max(1, int(L // cs))
    cs = L / nc
    grid = {}
    xy = np.empty((n, 2))

    def key(p):
        return (int(p[0] // cs), int(p[1] // cs))

    def conflicts(p, r, skip=-1):
        cx, cy = key(p)
        for gx in (cx - 1, cx, cx + 1):
            for gy in (cy - 1, cy, cy + 1):
                for k in grid.get((gx, gy), ()):
                    if k != skip and (xy[k, 0] - p[0]) ** 2 + (xy[k, 1] - p[1]) ** 2 < (r + radii[k]) ** 2:
                        return True
        return False

    for i in range(n):
        for _ in range(200000):
            p = rng.uniform(radii[i], L - radii[i], size=2)
            if not conflicts(p, radii[i]):
                break
        else:
            raise RuntimeError("random addition did not place disk %d" % i)
        xy[i] = p
        grid.setdefault(key(p), set()).add(i)
    for i in rng.permutation(n)[: int(near_frac * n)]:
        i = int(i)
        cx, cy = key(xy[i])
        best, bj = None, -1
        for gx in (cx - 1, cx, cx + 1):
            for gy in (cy - 1, cy, cy + 1):
                for k in grid.get((gx, gy), ()):
                    if k == i:
                        continue
                    dd = math.hypot(*(xy[k] - xy[i]))
                    if best is None or dd < best:
                        best, bj = dd, k
        if bj < 0:
            continue
        v = xy[i] - xy[bj]
        cand = xy[bj] + v / math.hypot(*v) * (radii[i] + radii[bj] + rng.uniform(0.1, 1.0) * gap)
        if not (radii[i] <= cand[0] <= L - radii[i] and radii[i] <= cand[1] <= L - radii[i]):
            continue
        if conflicts(cand, radii[i], skip=i):
            continue
        grid[key(xy[i])].discard(i)
        xy[i] = cand
        grid.setdefault(key(cand), set()).add(i)
    return xy
