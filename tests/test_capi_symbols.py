"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/bd.h; host-only entry points run on the CPU."""
import os
import re

import numpy as np
import pytest

import paper_1703_02484_gb300 as bd
from paper_1703_02484_gb300 import binding, workloads
from oracle import geometry

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(bd_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    lib = bd.load()
    names = declared_functions()
    assert "bd_init" in names and "bd_step" in names and "bd_free" in names
    for name in names:
        assert hasattr(lib, name), name
    # the binding covers the same set
    assert {s[0] for s in binding.SIGNATURES} == names


def test_default_params_and_strerror():
    lib = bd.load()
    p = binding.bd_params()
    assert lib.bd_default_params(p) == 0
    assert p.a == 1.0 and p.max_corr_iters > 0
    assert b"overlap" in lib.bd_strerror(-3)
    assert lib.bd_default_params(None) == -1


def test_init_argument_errors_without_gpu():
    lib = bd.load()
    import ctypes
    p = binding.make_params(10, rho=0.3)
    p.n = 0
    h = ctypes.c_void_p()
    assert lib.bd_init(ctypes.byref(p), None, None, None, None, ctypes.byref(h)) == -1
    p = binding.make_params(10, rho=0.3, law=binding.LAW_LONG)
    p.n_species = 5                      # at most four species
    assert lib.bd_init(ctypes.byref(p), None, None, None, None, ctypes.byref(h)) == -1
    p.n_species = 3
    p.alpha[4] = float("nan")            # the 3 x 3 table is checked entry by entry
    assert lib.bd_init(ctypes.byref(p), None, None, None, None, ctypes.byref(h)) == -1


@pytest.mark.parametrize("n", [1, 2, 3, 7, 500, 20000])
def test_host_triangulation_equals_oracle_delaunay(n):
    cfg = workloads.CONFIGS["c5"]
    L = workloads.box_side(max(n, 4), cfg.rho)
    xy = workloads.initial_positions(n, L, 1.0, cfg.rho, seed=n)
    tri, grid = binding.triangulate(xy, L)
    G = len(geometry.ghost_points(L))
    assert len(tri) == 2 * (n + G) - 6
    assert np.max(np.abs(grid - xy)) <= 1e-11 * L
    ot = geometry.delaunay(grid, L)
    assert np.array_equal(geometry.edges(tri), geometry.edges(ot))
    P = geometry.with_ghosts(grid, L)
    for t in tri[: min(len(tri), 2000)]:
        assert geometry.orient(P[t[0]], P[t[1]], P[t[2]]) > 0


def test_ghost_points_match_oracle_definition():
    for L in (3.5, 12.9, 103.55, 1023.3, 2566.79):
        assert np.array_equal(binding.ghost_points(L, 1.0), geometry.ghost_points(L, 1.0))
    # ring points stay clear of the walls and inside the far corners
    g = geometry.ghost_points(100.0, 1.0)
    ring = g[4:]
    assert np.all((ring[:, 0] <= -2) | (ring[:, 0] >= 102) | (ring[:, 1] <= -2) | (ring[:, 1] >= 102))
    assert np.all(np.abs(ring) < np.abs(g[:4]).max())


def test_host_triangulation_lattice_start():
    # the jittered lattice start used at high area fraction
    cfg = workloads.CONFIGS["c3"]
    n = 4000
    L = workloads.box_side(n, cfg.rho)
    xy = workloads.initial_positions(n, L, 1.0, cfg.rho, seed=3)
    tri, grid = binding.triangulate(xy, L)
    ot = geometry.delaunay(grid, L)
    assert np.array_equal(geometry.edges(tri), geometry.edges(ot))


@pytest.mark.parametrize("n,rho,seed", [(16, 0.1, 1), (50, 0.3, 2), (777, 0.3, 3), (5000, 0.5, 4)])
def test_host_torus_triangulation_equals_oracle(n, rho, seed):
    # the periodic box's initial triangulation (built on the host, Sec. 4.1)
    # against the oracle's torus Delaunay triangulation of the 3 x 3 tiling
    from oracle import periodic
    L = workloads.box_side(n, rho)
    Lf = float(np.float32(L))
    xy = workloads.initial_positions(n, Lf, 1.0, rho, seed=seed)
    xy = xy + np.random.default_rng(seed).uniform(0, Lf, 2)       # straddle the box edges
    tri, sh, grid = binding.triangulate_periodic(xy, L)
    assert len(tri) == 2 * n
    assert np.all((grid >= 0) & (grid < Lf))
    assert np.max(np.abs(periodic.min_image(grid - xy, Lf))) <= 1e-11 * Lf
    assert np.all(sh[:, 0, :] == 0)
    assert periodic.is_torus_triangulation(tri, sh)
    ref = periodic.edge_keys(*periodic.delaunay_torus(grid, Lf))
    assert np.array_equal(periodic.edge_keys(tri, sh), ref)
    corners = periodic.lifted(grid, tri, sh, Lf)
    for a, b, c in corners[: min(len(corners), 3000)]:
        assert geometry.orient(a, b, c) > 0
