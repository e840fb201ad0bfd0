"""GPU tests of the state transfers: bd_set_state copies the caller's arrays to
the device as they are and checks, rounds and permutes them there; bd_get_state
permutes on the device and copies into the caller's arrays.  Checked in a batch
of walls and periodic replicas (the permutation spans replicas) against the
host's own rounding rules, bit for bit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1703_02484_gb300 as bd  # noqa: E402
from paper_1703_02484_gb300 import workloads  # noqa: E402
from oracle import periodic  # noqa: E402
from scipy.spatial import cKDTree  # noqa: E402


def stream():
    return torch.cuda.current_stream().cuda_stream


def mixed_batch(seed=31):
    cfgs = workloads.batch_configs(4, seed=seed, n_lo=300, n_hi=2000)
    params, xys, sps, ths = [], [], [], []
    for r, cfg in enumerate(cfgs):
        xy, sp, th = workloads.initial_state(cfg, seed=seed + 100 * r)
        p = bd.params_from_config(cfg)
        p.replica = r
        if r in (1, 3):
            L = float(np.float32(workloads.box_side(p.n, cfg.rho)))
            p.box_L = L
            p.boundary = bd.BOUNDARY_PERIODIC
            xy = periodic.wrap(xy + np.array([0.3 * L, 0.7 * L]), L)
        params.append(p)
        xys.append(xy)
        sps.append(sp)
        ths.append(th)
    b = bd.System(params, np.concatenate(xys), np.concatenate(sps), np.concatenate(ths), stream=stream())
    return b, params


def grid_round(x, L, a, q, is_periodic):
    # the host's rules at bd_init: round to the grid (half to even); walls clamp
    # to [ceil(a/q) q, floor((L-a)/q) q], a periodic box wraps into [0, L)
    inv_q = 1.0 / q
    if is_periodic:
        y = np.rint((x - L * np.floor(x / L)) * inv_q) * q
        y = np.where(y >= L, y - L, y)
        return np.where(y < 0.0, y + L, y)
    lo = np.ceil(a * inv_q) * q
    hi = np.floor((L - a) * inv_q) * q
    return np.minimum(hi, np.maximum(lo, np.rint(x * inv_q) * q))


def no_overlap(xy, L, is_periodic):
    # every pair farther than sigma = 2 (pairs at exactly sigma count as overlapping here)
    t = cKDTree(xy, boxsize=L) if is_periodic else cKDTree(xy)
    return len(t.query_pairs(2.0)) == 0


def test_read_state_matches_state():
    b, _ = mixed_batch()
    b.step(4)
    ref = b.state(want_tri=False)
    xy = np.empty((b.n, 2))
    th = np.empty(b.n, np.float32)
    sp = np.empty(b.n, np.uint8)
    b.read_state(xy, th, sp)
    assert np.array_equal(xy, ref["xy"]) and np.array_equal(th, ref["theta"])
    assert np.array_equal(sp, ref["species"])
    with pytest.raises(ValueError):
        b.read_state(xy.astype(np.float32))
    with pytest.raises(ValueError):
        b.read_state(np.empty((b.n + 1, 2)))
    b.close()


def test_set_state_rounds_wraps_and_permutes_on_the_device():
    b, params = mixed_batch()
    b.step(3)
    q, _ = b.geometry()
    cur = b.state(want_tri=False)
    rng = np.random.default_rng(7)
    new = cur["xy"] + rng.uniform(-3e-10, 3e-10, size=cur["xy"].shape)   # off the grid (q ~ 1e-13)
    th = rng.uniform(0.0, 6.0, size=b.n).astype(np.float32)
    expect = np.empty_like(new)
    off = 0
    for r, p in enumerate(params):
        n = p.n
        L = b.replica(r)["L"]
        seg = new[off:off + n]
        if p.boundary:
            seg[::7] += L * rng.integers(-3, 4, size=seg[::7].shape)   # the same point, other images
        else:
            # a disk set just below a (inside the 1e-9 L tolerance) is clamped to
            # the wall: the first of the disks nearest the wall that has room
            for k in np.argsort(seg[:, 0])[:8]:
                x0 = seg[k, 0]
                seg[k, 0] = p.a - 0.5e-9 * L
                if no_overlap(grid_round(seg, L, p.a, q, False), L, False):
                    break
                seg[k, 0] = x0
            else:
                pytest.fail("no disk near the wall has room")
        expect[off:off + n] = grid_round(seg, L, p.a, q, bool(p.boundary))
        assert no_overlap(expect[off:off + n], L, bool(p.boundary))
        off += n
    b.set_state(new, th)
    got = b.state(want_tri=False)
    assert np.array_equal(got["xy"], expect)
    assert np.array_equal(got["theta"], th)
    assert b.step(3)["steps_done"] == 3
    b.close()


def test_set_state_without_theta_keeps_directions():
    b, _ = mixed_batch()
    before = b.state(want_tri=False)
    b.set_state(before["xy"])
    after = b.state(want_tri=False)
    assert np.array_equal(after["theta"], before["theta"])
    assert np.array_equal(after["xy"], before["xy"])
    b.close()


@pytest.mark.parametrize("case", ["nan_walls", "outside_walls", "nan_periodic", "inf_walls"])
def test_set_state_rejects_bad_centres_and_keeps_state(case):
    b, params = mixed_batch()
    b.step(2)
    before = b.state()
    bad = before["xy"].copy()
    base = [0]
    for p in params:
        base.append(base[-1] + p.n)
    if case == "nan_walls":
        bad[base[2] + 5, 1] = np.nan
    elif case == "outside_walls":
        L = b.replica(2)["L"]
        bad[base[2] + 9, 0] = L - params[2].a + 1e-6 * L
    elif case == "nan_periodic":
        bad[base[3] + 4, 0] = np.nan
    else:
        bad[base[0], 0] = np.inf
    with pytest.raises(bd.BDError) as e:
        b.set_state(bad)
    assert e.value.code == -3
    after = b.state()
    assert np.array_equal(after["xy"], before["xy"]) and np.array_equal(after["tri"], before["tri"])
    assert np.array_equal(after["theta"], before["theta"])
    assert b.step(2)["steps_done"] == 2
    b.close()


@pytest.mark.parametrize("placement", [bd.PLACE_RSA, bd.PLACE_LATTICE])
def test_init_without_positions_uses_the_placement(placement):
    # bd_init with no positions: the start is bd_place_disks's, rounded to the
    # position grid (the lattice start at area fraction 0.5, Sec. 4.1)
    cfg = workloads.CONFIGS["c3"]
    n = 3000
    p = bd.params_from_config(cfg, n=n)
    p.placement = placement
    s = bd.System(p, stream=stream())
    q, L = s.geometry()
    want = bd.place_disks(n, L, cfg.a, placement, seed=cfg.seed)
    want = np.minimum(np.floor((L - cfg.a) / q) * q, np.maximum(np.ceil(cfg.a / q) * q, np.rint(want / q) * q))
    got = s.state(want_tri=False)["xy"]
    assert np.array_equal(got, want)
    assert s.step(5)["steps_done"] == 5
    s.close()
