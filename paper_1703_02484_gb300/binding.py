"""Thin ctypes binding of the C ABI in include/bd.h (argument marshalling only).

Every computation happens in libbd_gb300.so; if the library cannot be
loaded the binding raises -- there is no fallback implementation."""
import ctypes
import os

import numpy as np

from . import build as _build

BD_OK = 0
ERRORS = {
    -1: "BD_ERR_ARG", -2: "BD_ERR_CUDA", -3: "BD_ERR_INIT_OVERLAP", -4: "BD_ERR_STEP_REJECTED",
    -5: "BD_ERR_OVERLAP_NOT_CONVERGED", -6: "BD_ERR_FLIP_NOT_CONVERGED",
    -7: "BD_ERR_DEVICE_TIMEOUT", -8: "BD_ERR_NOMEM", -9: "BD_ERR_TRIANGULATION",
    -10: "BD_ERR_UNSUPPORTED",
}
LAW_NONE, LAW_LONG, LAW_SHORT = 0, 1, 2
BOUNDARY_WALLS, BOUNDARY_PERIODIC = 0, 1
PLACE_RSA, PLACE_LATTICE = 0, 1
LOSS_MSD = 0
LOSS_HIST = 1
OVERLAP_DELAUNAY, OVERLAP_VERLET = 0, 1


class bd_params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("n_species", ctypes.c_int32),
        ("a", ctypes.c_double), ("box_L", ctypes.c_double), ("area_fraction", ctypes.c_double),
        ("law", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("alpha", ctypes.c_double * 16),
        ("eps", ctypes.c_double), ("kappa", ctypes.c_double),
        ("r_cut", ctypes.c_double), ("skin", ctypes.c_double),
        ("D", ctypes.c_double), ("Dr", ctypes.c_double), ("v0", ctypes.c_double), ("dt", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("replica", ctypes.c_int32),
        ("max_corr_iters", ctypes.c_int32), ("max_flip_rounds", ctypes.c_int32),
        ("literal_noise", ctypes.c_int32), ("step0", ctypes.c_int64),
        ("overlap_mode", ctypes.c_int32), ("max_dt_halvings", ctypes.c_int32),
        ("boundary", ctypes.c_int32),
        ("placement", ctypes.c_int32),
    ]


class bd_step_stats(ctypes.Structure):
    _fields_ = [
        ("steps_done", ctypes.c_int64), ("corr_iters", ctypes.c_int64),
        ("overlap_pairs", ctypes.c_int64), ("flip_rounds", ctypes.c_int64),
        ("flips", ctypes.c_int64), ("repair_flips", ctypes.c_int64), ("inverted", ctypes.c_int64),
        ("max_corr_iters", ctypes.c_int32), ("rejected", ctypes.c_int32),
        ("verlet_rebuilds", ctypes.c_int32), ("fail_phase", ctypes.c_int32),
        ("max_overlap", ctypes.c_double),
        ("fail_item", ctypes.c_int32), ("fail_count", ctypes.c_int32),
        ("barriers", ctypes.c_int64),
        ("substeps", ctypes.c_int64), ("halvings", ctypes.c_int64),
        ("tri_visits", ctypes.c_int64), ("exact_tests", ctypes.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# entry points declared in include/bd.h: (name, restype, argtypes)
_P = ctypes.c_void_p
SIGNATURES = [
    ("bd_default_params", ctypes.c_int, [ctypes.POINTER(bd_params)]),
    ("bd_init", ctypes.c_int, [ctypes.POINTER(bd_params), _P, _P, _P, _P, ctypes.POINTER(_P)]),
    ("bd_init_radii", ctypes.c_int, [ctypes.POINTER(bd_params), _P, _P, _P, _P, _P, ctypes.POINTER(_P)]),
    ("bd_step", ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(bd_step_stats)]),
    ("bd_get_state", ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_int64)]),
    ("bd_set_state", ctypes.c_int, [_P, _P, _P]),
    ("bd_compute_forces", ctypes.c_int, [_P, _P]),
    ("bd_get_geometry", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    ("bd_force_timing", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_int64)]),
    ("bd_last_launch_count", ctypes.c_int64, [_P]),
    ("bd_triangulate", ctypes.c_int, [ctypes.c_int32, _P, ctypes.c_double, ctypes.c_double, _P, _P,
                                      ctypes.POINTER(ctypes.c_int32)]),
    ("bd_place_disks", ctypes.c_int, [ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                       ctypes.c_uint64, _P]),
    ("bd_ghost_points", ctypes.c_int, [ctypes.c_double, ctypes.c_double, _P,
                                       ctypes.POINTER(ctypes.c_int32)]),
    ("bd_forces_noalloc", ctypes.c_int, [ctypes.c_int32, _P, _P, ctypes.POINTER(ctypes.c_double),
                                         _P, _P]),
    ("bd_get_neighbors", ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    ("bd_batch_init", ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(bd_params), _P, _P, _P, _P,
                                     ctypes.POINTER(_P)]),
    ("bd_get_replica", ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]),
    ("bd_get_tuning", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_int32)]),
    ("bd_set_force_params", ctypes.c_int, [_P, _P, ctypes.c_double]),
    ("bd_set_step", ctypes.c_int, [_P, ctypes.c_int64]),
    ("bd_rollout", ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(bd_step_stats)]),
    ("bd_rollout_vjp", ctypes.c_int, [_P, _P]),
    ("bd_batch_step", ctypes.c_int, [_P, ctypes.c_int32, _P]),
    ("bd_rollout_replay", ctypes.c_int, [_P, _P, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
    ("bd_rollout_positions", ctypes.c_int, [_P, ctypes.c_int32, _P]),
    ("bd_rollout_log_size", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    ("bd_stage_times", ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    ("bd_get_tri_shifts", ctypes.c_int, [_P, ctypes.c_int32, _P]),
    ("bd_triangulate_periodic", ctypes.c_int, [ctypes.c_int32, _P, ctypes.c_double, _P, _P, _P,
                                               ctypes.POINTER(ctypes.c_int32)]),
    ("bd_struct_sizes", ctypes.c_int, [ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    ("bd_last_stats", ctypes.c_int, [_P, ctypes.POINTER(bd_step_stats)]),
    ("bd_set_wait_limit", ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int32]),
    ("bd_set_loop_caps", ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    ("bd_noise_sample", ctypes.c_int, [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P]),
    ("bd_set_force_shard", ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    ("bd_force_slots", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
    ("bd_step_begin", ctypes.c_int, [_P, _P]),
    ("bd_step_end", ctypes.c_int, [_P, _P, ctypes.POINTER(bd_step_stats)]),
    ("bd_free", None, [_P]),
    ("bd_strerror", ctypes.c_char_p, [ctypes.c_int]),
]

_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libbd_gb300.so (building it first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError("libbd_gb300.so is not built; run __graft_entry__.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    ps, ss = ctypes.c_int32(), ctypes.c_int32()
    lib.bd_struct_sizes(ctypes.byref(ps), ctypes.byref(ss))
    if (ps.value, ss.value) != (ctypes.sizeof(bd_params), ctypes.sizeof(bd_step_stats)):
        raise RuntimeError("libbd_gb300.so structure sizes (%d, %d) differ from the binding's (%d, %d)"
                           % (ps.value, ss.value, ctypes.sizeof(bd_params), ctypes.sizeof(bd_step_stats)))
    _lib = lib
    return lib


class BDError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = load().bd_strerror(code).decode()
        super().__init__("%s failed: %s (%s)" % (where, ERRORS.get(code, code), msg))


def _check(code, where):
    if code != BD_OK:
        raise BDError(code, where)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def make_params(n, L=None, rho=None, a=1.0, law=LAW_NONE, alpha=(0, 0, 0, 0), n_species=1,
                eps=1.0, kappa=1.0, r_cut=5.0, skin=0.6, D=1.0, Dr=0.0, v0=0.0, dt=1e-4,
                seed=0, replica=0, precision=0, max_corr_iters=1000, max_flip_rounds=4096,
                literal_noise=0, step0=0, max_dt_halvings=0, boundary=BOUNDARY_WALLS, placement=PLACE_RSA):
    p = bd_params()
    _check(load().bd_default_params(ctypes.byref(p)), "bd_default_params")
    p.n, p.n_species, p.a = int(n), int(n_species), float(a)
    p.box_L = float(L) if L is not None else 0.0
    p.area_fraction = float(rho) if rho is not None else 0.0
    p.law, p.precision = int(law), int(precision)
    if len(alpha) > 16:
        raise ValueError("alpha: at most a 4 x 4 table")
    for k in range(len(alpha)):
        p.alpha[k] = float(alpha[k])
    p.eps, p.kappa, p.r_cut, p.skin = float(eps), float(kappa), float(r_cut), float(skin)
    p.D, p.Dr, p.v0, p.dt = float(D), float(Dr), float(v0), float(dt)
    p.seed, p.replica = int(seed), int(replica)
    p.max_corr_iters, p.max_flip_rounds = int(max_corr_iters), int(max_flip_rounds)
    p.literal_noise, p.step0 = int(literal_noise), int(step0)
    p.max_dt_halvings = int(max_dt_halvings)
    p.boundary = int(boundary)
    p.placement = int(placement)
    return p


def params_from_config(cfg, n=None, seed=None):
    return make_params(n=cfg.n if n is None else n, rho=cfg.rho, a=cfg.a, law=cfg.law,
                       alpha=cfg.alpha, n_species=cfg.n_species, eps=cfg.eps, kappa=cfg.kappa,
                       r_cut=cfg.r_cut, skin=cfg.skin, D=cfg.D, Dr=cfg.Dr, v0=cfg.v0, dt=cfg.dt,
                       seed=cfg.seed if seed is None else seed, precision=cfg.precision)


class System:
    """One simulated system (or a batch of replicas) behind a bd_handle."""

    def __init__(self, params, xy=None, species=None, theta=None, stream=None, radii=None):
        lib = load()
        batch = isinstance(params, (list, tuple))
        plist = list(params) if batch else [params]
        self.R = len(plist)
        self.n = int(sum(p.n for p in plist))
        self._xy = None if xy is None else np.ascontiguousarray(xy, dtype=np.float64).reshape(-1)
        self._sp = None if species is None else np.ascontiguousarray(species, dtype=np.uint8)
        self._th = None if theta is None else np.ascontiguousarray(theta, dtype=np.float32)
        h = ctypes.c_void_p()
        st = None if stream is None else ctypes.c_void_p(int(stream))
        if batch:
            arr = (bd_params * self.R)(*plist)
            self._plist = arr
            _check(lib.bd_batch_init(self.R, arr, _ptr(self._xy), _ptr(self._sp), _ptr(self._th),
                                     st, ctypes.byref(h)), "bd_batch_init")
        elif radii is not None:
            self._rad = np.ascontiguousarray(radii, dtype=np.float64)
            _check(lib.bd_init_radii(ctypes.byref(params), _ptr(self._xy), _ptr(self._sp), _ptr(self._th),
                                     _ptr(self._rad), st, ctypes.byref(h)), "bd_init_radii")
        else:
            _check(lib.bd_init(ctypes.byref(params), _ptr(self._xy), _ptr(self._sp),
                               _ptr(self._th), st, ctypes.byref(h)), "bd_init")
        self.h = h
        self.params = params
        q, L = self.geometry()
        self.L = L
        self.n_tri = 0
        for r in range(self.R):
            nn, nt, LL = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
            _check(lib.bd_get_replica(self.h, r, None, None, None, ctypes.byref(nt), ctypes.byref(nn),
                                      ctypes.byref(LL)), "bd_get_replica")
            self.n_tri += nt.value
        self.ghosts = ghost_points(L, plist[0].a)

    def close(self):
        if self.h:
            load().bd_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, nsteps=1, raise_on_error=True):
        st = bd_step_stats()
        code = load().bd_step(self.h, int(nsteps), ctypes.byref(st))
        if raise_on_error:
            _check(code, "bd_step")
        return (st.as_dict(), code) if not raise_on_error else st.as_dict()

    def state(self, want_tri=True):
        n = self.n
        xy = np.zeros((n, 2), dtype=np.float64)
        th = np.zeros(n, dtype=np.float32)
        sp = np.zeros(n, dtype=np.uint8)
        tri = np.zeros((self.n_tri, 3), dtype=np.int32) if want_tri else None
        nt = ctypes.c_int32()
        stp = ctypes.c_int64()
        _check(load().bd_get_state(self.h, _ptr(xy), _ptr(th), _ptr(sp), _ptr(tri),
                                   ctypes.byref(nt), ctypes.byref(stp)), "bd_get_state")
        return dict(xy=xy, theta=th, species=sp, tri=tri, n_tri=nt.value, step=stp.value)

    def batch_step(self, nsteps=1):
        """bd_batch_step: the per-replica stats of the call, as dicts (R entries)."""
        arr = (bd_step_stats * self.R)()
        _check(load().bd_batch_step(self.h, int(nsteps), ctypes.cast(arr, ctypes.c_void_p)), "bd_batch_step")
        return [a.as_dict() for a in arr]

    def read_state(self, xy, theta=None, species=None):
        """Fill caller-owned arrays (C-contiguous; float64 (n, 2), float32 (n,), uint8 (n,))
        with the current positions, directions and species, without allocating."""
        n = self.n
        for a, dt, shape in ((xy, np.float64, (n, 2)), (theta, np.float32, (n,)), (species, np.uint8, (n,))):
            if a is not None and (a.dtype != dt or a.shape != shape or not a.flags.c_contiguous):
                raise ValueError("read_state: expected a C-contiguous %s array of shape %s" % (np.dtype(dt), shape))
        _check(load().bd_get_state(self.h, _ptr(xy), _ptr(theta), _ptr(species), None, None, None),
               "bd_get_state")

    def tri_shifts(self, replica=-1):
        """Corner image shifts (n_tri, 3, 2) of the triangulation (periodic box)."""
        nt = self.n_tri if replica < 0 else self.replica_sizes()[replica][1]
        sh = np.zeros((nt, 3, 2), dtype=np.int8)
        _check(load().bd_get_tri_shifts(self.h, int(replica), _ptr(sh)), "bd_get_tri_shifts")
        return sh.astype(np.int64)

    def replica_sizes(self):
        out = []
        for r in range(self.R):
            nn, nt, LL = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
            _check(load().bd_get_replica(self.h, r, None, None, None, ctypes.byref(nt), ctypes.byref(nn),
                                         ctypes.byref(LL)), "bd_get_replica")
            out.append((nn.value, nt.value, LL.value))
        return out

    def set_state(self, xy, theta=None):
        xy = np.ascontiguousarray(xy, dtype=np.float64)
        th = None if theta is None else np.ascontiguousarray(theta, dtype=np.float32)
        _check(load().bd_set_state(self.h, _ptr(xy), _ptr(th)), "bd_set_state")

    # ---- force sharding (one system on several ranks) ----
    def set_force_shard(self, rank, world):
        """bd_set_force_shard: compute this rank's share of the all-pairs sweep."""
        _check(load().bd_set_force_shard(self.h, int(rank), int(world)), "bd_set_force_shard")

    def force_slots(self):
        """Length (double2 entries) of the force buffer of bd_step_begin / bd_step_end."""
        k = ctypes.c_int32()
        _check(load().bd_force_slots(self.h, ctypes.byref(k)), "bd_force_slots")
        return k.value

    def step_begin(self, forces_dev_ptr):
        """bd_step_begin: this rank's partial forces into the device buffer."""
        _check(load().bd_step_begin(self.h, ctypes.c_void_p(int(forces_dev_ptr))), "bd_step_begin")

    def step_end(self, forces_dev_ptr):
        """bd_step_end: one step with the summed forces in the device buffer."""
        st = bd_step_stats()
        _check(load().bd_step_end(self.h, ctypes.c_void_p(int(forces_dev_ptr)), ctypes.byref(st)), "bd_step_end")
        return st.as_dict()

    def last_stats(self):
        """Counters of the last bd_step / bd_batch_step / bd_set_state call (bd_last_stats)."""
        st = bd_step_stats()
        _check(load().bd_last_stats(self.h, ctypes.byref(st)), "bd_last_stats")
        return st.as_dict()

    def set_loop_caps(self, max_corr_iters=1000, max_flip_rounds=4096):
        """bd_set_loop_caps: caps on correction passes and flip rounds of later steps."""
        _check(load().bd_set_loop_caps(self.h, int(max_corr_iters), int(max_flip_rounds)), "bd_set_loop_caps")

    def set_wait_limit(self, seconds=2.0, hold_barrier=0):
        """bd_set_wait_limit: time limit of the device-side barrier waits; hold_barrier > 0
        makes that barrier of every later launch run out (tests of the timeout path)."""
        _check(load().bd_set_wait_limit(self.h, float(seconds), int(hold_barrier)), "bd_set_wait_limit")

    def forces(self):
        F = np.zeros((self.n, 2), dtype=np.float64)
        _check(load().bd_compute_forces(self.h, _ptr(F)), "bd_compute_forces")
        return F

    def geometry(self):
        q, L = ctypes.c_double(), ctypes.c_double()
        _check(load().bd_get_geometry(self.h, ctypes.byref(q), ctypes.byref(L)), "bd_get_geometry")
        return q.value, L.value

    def force_timing(self, enable=True, reset=False):
        ms, k = ctypes.c_double(), ctypes.c_int64()
        _check(load().bd_force_timing(self.h, int(enable), int(reset), ctypes.byref(ms),
                                      ctypes.byref(k)), "bd_force_timing")
        return ms.value, k.value

    def replica(self, r):
        """State of replica r in its own numbering: dict(xy, theta, tri, n, L)."""
        lib = load()
        nn, nt, LL = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        _check(lib.bd_get_replica(self.h, int(r), None, None, None, ctypes.byref(nt),
                                  ctypes.byref(nn), ctypes.byref(LL)), "bd_get_replica")
        xy = np.zeros((nn.value, 2))
        th = np.zeros(nn.value, dtype=np.float32)
        tri = np.zeros((nt.value, 3), dtype=np.int32)
        _check(lib.bd_get_replica(self.h, int(r), _ptr(xy), _ptr(th), _ptr(tri), ctypes.byref(nt),
                                  ctypes.byref(nn), ctypes.byref(LL)), "bd_get_replica")
        return dict(xy=xy, theta=th, tri=tri, n=nn.value, L=LL.value)

    def tuning(self):
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(load().bd_get_tuning(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
               "bd_get_tuning")
        return dict(tiles_per_item=a.value, variant=b.value, n_items=c.value)

    def neighbors(self, max_per=64):
        n = self.n
        counts = np.zeros(n, dtype=np.int32)
        idx = np.zeros((n, max_per), dtype=np.int32)
        _check(load().bd_get_neighbors(self.h, int(max_per), _ptr(counts), _ptr(idx)),
               "bd_get_neighbors")
        return [idx[i, : counts[i]].copy() for i in range(n)]

    def last_launch_count(self):
        return int(load().bd_last_launch_count(self.h))

    def stage_times(self, reset=False):
        """Triangulation-kernel stage times (ms) and pass counts since the last
        reset: dict check/repair/flip/apply -> (ms, passes)."""
        ms = np.zeros(5, dtype=np.float64)
        n = np.zeros(5, dtype=np.int64)
        _check(load().bd_stage_times(self.h, int(reset), _ptr(ms), _ptr(n)), "bd_stage_times")
        return {k: (float(ms[i]), int(n[i]))
                for i, k in enumerate(("check", "repair", "flip", "apply", "check_lists"))}

    # ---- differentiated rollout ----
    def set_force_params(self, alpha=None, v0=None):
        A = None if alpha is None else np.ascontiguousarray(alpha, dtype=np.float64).reshape(4)
        _check(load().bd_set_force_params(self.h, _ptr(A), float("nan") if v0 is None else float(v0)),
               "bd_set_force_params")

    def set_step(self, step):
        _check(load().bd_set_step(self.h, int(step)), "bd_set_step")

    def rollout(self, nsteps, ckpt_every=20, target=0.1, loss_kind=LOSS_MSD):
        """Advance nsteps recording the frozen choices; returns (loss, stats)."""
        loss = ctypes.c_double()
        st = bd_step_stats()
        _check(load().bd_rollout(self.h, int(nsteps), int(ckpt_every), int(loss_kind), float(target),
                                 ctypes.byref(loss), ctypes.byref(st)), "bd_rollout")
        return loss.value, st.as_dict()

    def rollout_vjp(self):
        """dL/d(A00, A01, A10, A11, v0) of the last recorded rollout."""
        g = np.zeros(5, dtype=np.float64)
        _check(load().bd_rollout_vjp(self.h, _ptr(g)), "bd_rollout_vjp")
        return g

    def rollout_replay(self, alpha=None, v0=None):
        A = None if alpha is None else np.ascontiguousarray(alpha, dtype=np.float64).reshape(4)
        loss = ctypes.c_double()
        _check(load().bd_rollout_replay(self.h, _ptr(A), float("nan") if v0 is None else float(v0),
                                        ctypes.byref(loss)), "bd_rollout_replay")
        return loss.value

    def rollout_positions(self, which=0):
        xy = np.zeros((self.n, 2), dtype=np.float64)
        _check(load().bd_rollout_positions(self.h, int(which), _ptr(xy)), "bd_rollout_positions")
        return xy

    def rollout_log_size(self):
        a, b = ctypes.c_int32(), ctypes.c_int32()
        _check(load().bd_rollout_log_size(self.h, ctypes.byref(a), ctypes.byref(b)), "bd_rollout_log_size")
        return a.value, b.value


def rollout_loss(params, system, xy0, theta0, step0, nsteps, ckpt_every=20, target=0.1, loss_kind=LOSS_MSD):
    """Differentiable rollout loss: params is a torch tensor (5,) =
    (A00, A01, A10, A11, v0); the system is reset to (xy0, theta0) at step
    step0, advanced nsteps with bd_rollout, and the loss (LOSS_MSD or
    LOSS_HIST) returned as a 0-d float64 tensor whose backward runs
    bd_rollout_vjp."""
    return _rollout_fn().apply(params, system, xy0, theta0, step0, nsteps, ckpt_every, target, loss_kind)


_ROLLOUT_FN = None


def _rollout_fn():
    global _ROLLOUT_FN
    if _ROLLOUT_FN is None:
        import torch

        class RolloutLoss(torch.autograd.Function):
            @staticmethod
            def forward(ctx, params, system, xy0, theta0, step0, nsteps, ckpt_every, target, loss_kind):
                p = params.detach().to("cpu", torch.float64).numpy()
                system.set_force_params(p[:4], p[4])
                system.set_state(xy0, theta0)
                system.set_step(step0)
                loss, _ = system.rollout(nsteps, ckpt_every, target, loss_kind)
                ctx.system = system
                ctx.dev = params.device
                return torch.tensor(loss, dtype=torch.float64, device=params.device)

            @staticmethod
            def backward(ctx, g):
                grad = torch.from_numpy(ctx.system.rollout_vjp()).to(ctx.dev)
                return g * grad, None, None, None, None, None, None, None, None

        _ROLLOUT_FN = RolloutLoss
    return _ROLLOUT_FN


def noise_sample(seed, replica, counters):
    """bd_noise_sample: for counters (n, 4) uint32, the device's Philox words (n, 4) and
    clamped normals (n, 3) in the FP32 and the FP64 forms of the step."""
    c = np.ascontiguousarray(counters, dtype=np.uint32).reshape(-1, 4)
    n = len(c)
    words = np.zeros((n, 4), dtype=np.uint32)
    z32 = np.zeros((n, 3), dtype=np.float32)
    z64 = np.zeros((n, 3), dtype=np.float64)
    _check(load().bd_noise_sample(int(seed), int(replica), n, _ptr(c), _ptr(words), _ptr(z32), _ptr(z64)),
           "bd_noise_sample")
    return words, z32, z64


def place_disks(n, L, a=1.0, placement=PLACE_RSA, seed=0):
    """Start positions as bd_init draws them for xy = None (bd_place_disks): (n, 2)."""
    out = np.zeros((int(n), 2), dtype=np.float64)
    _check(load().bd_place_disks(int(n), float(L), float(a), int(placement), int(seed), _ptr(out)),
           "bd_place_disks")
    return out


def ghost_points(L, a=1.0):
    """The fixed ghost points closing the triangulation (bd_ghost_points)."""
    cnt = ctypes.c_int32(0)
    _check(load().bd_ghost_points(float(L), float(a), None, ctypes.byref(cnt)), "bd_ghost_points")
    out = np.zeros((cnt.value, 2), dtype=np.float64)
    _check(load().bd_ghost_points(float(L), float(a), _ptr(out), ctypes.byref(cnt)), "bd_ghost_points")
    return out


def triangulate(xy, L, a=1.0):
    """Host-side initial Delaunay triangulation (bd_triangulate): returns
    (triangles, centres rounded to the position grid)."""
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    n = len(xy)
    G = len(ghost_points(L, a))
    tri = np.zeros((2 * (n + G) - 6, 3), dtype=np.int32)
    grid = np.zeros_like(xy)
    nt = ctypes.c_int32()
    _check(load().bd_triangulate(n, _ptr(xy), float(L), float(a), _ptr(grid), _ptr(tri),
                                 ctypes.byref(nt)), "bd_triangulate")
    return tri[: nt.value], grid


def triangulate_periodic(xy, L):
    """Host-side torus triangulation (bd_triangulate_periodic): returns
    (triangles (2n, 3), corner shifts (2n, 3, 2), centres on the grid in [0, L))."""
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    n = len(xy)
    tri = np.zeros((2 * n, 3), dtype=np.int32)
    sh = np.zeros((2 * n, 3, 2), dtype=np.int8)
    grid = np.zeros_like(xy)
    nt = ctypes.c_int32()
    _check(load().bd_triangulate_periodic(n, _ptr(xy), float(L), _ptr(grid), _ptr(tri), _ptr(sh),
                                          ctypes.byref(nt)), "bd_triangulate_periodic")
    return tri[: nt.value], sh[: nt.value].astype(np.int64), grid


def forces_noalloc(n, xy_dev_ptr, species_dev_ptr, alpha, F_dev_ptr, stream=None):
    """bd_forces_noalloc on caller-owned device buffers (raw pointers)."""
    A = (ctypes.c_double * 4)(*[float(v) for v in alpha])
    st = None if stream is None else ctypes.c_void_p(int(stream))
    _check(load().bd_forces_noalloc(int(n), ctypes.c_void_p(int(xy_dev_ptr)),
                                    ctypes.c_void_p(int(species_dev_ptr)), A,
                                    ctypes.c_void_p(int(F_dev_ptr)), st), "bd_forces_noalloc")
