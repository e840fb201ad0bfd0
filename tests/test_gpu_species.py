"""GPU parity with more than two species (up to four): the long-range table
A[s_i][s_j] of Sec. 2.2 (mu_i alpha_j for any number of species), through
the C ABI, against the FP64 oracle."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1703_02484_gb300 as bd  # noqa: E402
from paper_1703_02484_gb300 import workloads  # noqa: E402
from oracle import forces as oforces  # noqa: E402
from oracle import geometry  # noqa: E402
from oracle import step as ostep  # noqa: E402
from scipy.spatial import cKDTree  # noqa: E402

C2 = workloads.CONFIGS["c2"]


def stream():
    return torch.cuda.current_stream().cuda_stream


def table(ns, seed):
    # repulsive on the diagonal, mixed off it (non-reciprocal)
    rng = np.random.default_rng(seed)
    A = rng.uniform(-0.1, 0.2, (ns, ns))
    A[np.diag_indices(ns)] = 0.05
    return A.reshape(-1)


def setup(n, ns, seed, near_contact=False, precision=0):
    L = workloads.box_side(n, C2.rho)
    if near_contact:
        xy = workloads.near_contact_state(n, L, 1.0, seed=seed)
    else:
        xy = workloads.initial_positions(n, L, 1.0, C2.rho, seed=seed)
    rng = np.random.default_rng(seed + 7)
    sp = rng.integers(0, ns, n).astype(np.uint8)
    th = rng.uniform(0, 2 * math.pi, n).astype(np.float32)
    A = table(ns, seed)
    p = bd.make_params(n, L=L, law=bd.LAW_LONG, alpha=A, n_species=ns, D=C2.D, Dr=C2.Dr, v0=C2.v0,
                       dt=C2.dt, seed=seed, precision=precision)
    return p, xy, sp, th, A, L


def rel_err(F, ref):
    return float(np.max(np.linalg.norm(F - ref, axis=1))) / math.sqrt(float(np.mean(np.sum(ref ** 2, axis=1))))


@pytest.mark.parametrize("variant,tiles", [(0, 3), (1, 5), (2, 2), (3, 4)])
@pytest.mark.parametrize("ns", [3, 4])
def test_forces_more_species(monkeypatch, variant, tiles, ns):
    monkeypatch.setenv("BD_FORCE_VARIANT", str(variant))
    monkeypatch.setenv("BD_FORCE_TILES", str(tiles))
    p, xy, sp, th, A, L = setup(3001, ns, seed=ns)
    s = bd.System(p, xy, sp, th, stream=stream())
    F = s.forces()
    grid = s.state(want_tri=False)["xy"]
    assert s.tuning()["variant"] == variant
    assert rel_err(F, oforces.long_range_numpy(grid, sp, A)) <= 1e-5
    s.close()


def test_forces_more_species_fp64():
    p, xy, sp, th, A, L = setup(1500, 4, seed=9, precision=1)
    s = bd.System(p, xy, sp, th, stream=stream())
    F = s.forces()
    grid = s.state(want_tri=False)["xy"]
    assert rel_err(F, oforces.long_range_numpy(grid, sp, A)) <= 1e-12
    s.close()


@pytest.mark.parametrize("ns,seed", [(3, 21), (4, 22)])
def test_one_step_parity_more_species(ns, seed):
    p, xy, sp, th, A, L = setup(3000, ns, seed=seed, near_contact=True)
    s = bd.System(p, xy, sp, th, stream=stream())
    st = s.step(1)
    out = s.state()
    op = ostep.Params(L=L, law=ostep.LAW_LONG, alpha=tuple(A), D=C2.D, Dr=C2.Dr, v0=C2.v0, dt=C2.dt,
                      seed=seed)
    ref = ostep.step(xy, th.astype(np.float64), sp, 0, op)
    assert not ref["rejected"] and ref["corr_iters"] >= 1 and st["corr_iters"] == ref["corr_iters"]
    assert float(np.max(np.abs(out["xy"] - ref["xy"]))) <= 1e-5
    assert np.array_equal(geometry.edges(out["tri"]), geometry.edges(ref["tris"]))
    assert len(cKDTree(out["xy"]).query_pairs(2.0 * (1 - 1e-12))) == 0
    assert np.array_equal(out["species"], sp)
    s.close()


def test_batch_with_mixed_species_counts():
    specs = [setup(900 + 300 * k, ns, seed=30 + k) for k, ns in enumerate((1, 2, 3, 4))]
    params = []
    for r, (p, *_rest) in enumerate(specs):
        p.replica = r
        params.append(p)
    xy = np.concatenate([sp_[1] for sp_ in specs])
    sp = np.concatenate([sp_[2] for sp_ in specs])
    th = np.concatenate([sp_[3] for sp_ in specs])
    b = bd.System(params, xy, sp, th, stream=stream())
    F = b.forces()
    grid = b.state(want_tri=False)["xy"]
    off = 0
    for p, x, s_, t_, A, L in specs:
        n = len(x)
        ref = oforces.long_range_numpy(grid[off:off + n], s_, A if p.n_species > 1 else (A[0],) * 4)
        assert rel_err(F[off:off + n], ref) <= 1e-5
        off += n
    st = b.step(5)
    assert st["steps_done"] == 5
    b.close()


def test_two_by_two_entry_points_refuse_more_species():
    p, xy, sp, th, A, L = setup(600, 3, seed=40)
    s = bd.System(p, xy, sp, th, stream=stream())
    with pytest.raises(bd.BDError) as e:
        s.rollout(2)
    assert e.value.code == -10
    with pytest.raises(bd.BDError) as e:
        s.set_force_params(alpha=(0.1, 0.1, 0.1, 0.1))
    assert e.value.code == -10
    s.close()
