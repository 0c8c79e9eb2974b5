"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element
by element on every node of grids that span several transform tiles and
ragged bins, for both plan precisions.  Tolerances: see parity_util."""
import numpy as np
import pytest
import torch

import oracle
import paper_1112_3010_gb300 as pkg
from paper_1112_3010_gb300 import workloads as wl

from parity_util import check, oracle_ref, run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    pkg.load_library()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_circle_c1_full_grid(prec):
    """The 2D slice: 128^2 grid, 256 points on a circle, tau = 0.005: S, grad S
    and the winding-number sign on all 16384 nodes."""
    s = wl.config_c1()
    res = run(s, prec, outputs=("S", "dS", "sign"))
    ref = oracle_ref(s, want=("S", "dS", "mu", "R"))
    rep = check(s, res, ref, check_hess=False, label="c1-" + prec)
    assert rep["trusted"] > 4000
    assert rep["sign_checked"] > 10000


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_stars_2d_with_hessian_ragged(prec):
    """Non-power-of-two, non-square grid (ragged bins and a padded size
    above 2N), several star polygons, Hessian included."""
    s = wl.stars(N=256, K=3000, n_shapes=3, tau=0.006, seed=5)
    s.dims = (200, 168)
    s.points = s.points * np.array([200 / 256, 168 / 256])
    s.weights = s.weights * np.array([200 / 256, 168 / 256])
    res = run(s, prec, outputs=("S", "dS", "d2S", "sign"))
    ref = oracle_ref(s)
    check(s, res, ref, label="stars-" + prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sphere_3d(prec):
    """3D: points on a sphere with area-weighted normals, topological degree."""
    s = wl.sphere(N=40, K=3000, radius=0.3, tau=0.03, seed=8)
    res = run(s, prec, outputs=("S", "dS", "d2S", "sign"))
    ref = oracle_ref(s)
    check(s, res, ref, label="sphere-" + prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_torus_sphere_3d_small(prec):
    s = wl.torus_sphere(N=48, K=12000, tau=0.025, seed=9)
    res = run(s, prec, outputs=("S", "dS", "sign"))
    ref = oracle_ref(s, want=("S", "dS", "mu", "R"))
    check(s, res, ref, check_hess=False, label="torus-" + prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_unsigned_without_weights(prec):
    s = wl.random_points(2, 96, 50, tau=0.02, seed=3)
    res = run(s, prec, outputs=("S", "dS"), with_weights=False)
    assert "sign" not in res
    ref = oracle_ref(s, with_weights=False, want=("S", "dS", "R"))
    check(s, res, ref, check_sign=False, label="unsigned-" + prec)


def test_single_point_and_multiplicity():
    """One node holding 5 coincident points: S = r - tau log 5 (closed form)."""
    N, tau = 64, 0.05
    P = np.tile([[0.25, 0.5]], (5, 1))
    s = wl.Shape(2, (N, N), 1.0 / N, tau, P, None)
    res = run(s, "fp64", outputs=("S", "dS"), with_weights=False)
    X = oracle.grid_nodes(s.dims, s.h)
    r = np.linalg.norm(X - np.array([16 / 64, 32 / 64]), axis=1)
    ok = (res["flags"].ravel() & pkg.SDF_FLAG_CAPPED) == 0
    err = np.abs(res["S"].ravel()[ok] - (r[ok] - tau * np.log(5)))
    assert err.max() <= 1e-3 * tau
    assert res["flags"].ravel()[16 + 64 * 32] & pkg.SDF_FLAG_SOURCE


def test_points_on_grid_corners():
    """Points on the first and last nodes of every axis (the grid's edges)."""
    N = 33
    h = 1.0 / N
    P = np.array([[0.0, 0.0], [(N - 1) * h, 0.0], [0.0, (N - 1) * h], [(N - 1) * h, (N - 1) * h]])
    s = wl.Shape(2, (N, N), h, 0.05, P, None)
    for prec in ("fp64", "fp32"):
        res = run(s, prec, outputs=("S", "dS"), with_weights=False)
        ref = oracle_ref(s, with_weights=False, want=("S", "dS", "R"))
        check(s, res, ref, check_sign=False, label="corners-" + prec)


def test_out_of_grid_point_reported():
    N = 32
    P = np.array([[0.5, 0.5], [1.5, 0.5]])
    plan = pkg.Plan(2, (N, N), 1.0 / N, 0.05, precision="fp32", outputs=("S",))
    with pytest.raises(pkg.SDFError) as ei:
        plan.execute(torch.from_numpy(P).cuda())
    assert ei.value.code == 3
    # the plan stays usable after the error
    out = plan.execute(torch.from_numpy(P[:1]).cuda())
    assert torch.isfinite(out["S"]).all()


def test_deterministic_bitwise():
    s = wl.stars(N=256, K=4000, n_shapes=2, tau=0.008, seed=12)
    for prec in ("fp64", "fp32"):
        a = run(s, prec, outputs=("S", "dS", "d2S", "sign"))
        b = run(s, prec, outputs=("S", "dS", "d2S", "sign"))
        for k in ("S", "dS", "d2S", "sign", "flags"):
            assert np.array_equal(a[k], b[k]), (prec, k)


def test_execute_host_matches_device():
    s = wl.config_c1()
    plan = pkg.Plan(2, s.dims, s.h, s.tau, precision="fp32", outputs=("S", "dS", "sign"))
    dev = plan.execute(torch.from_numpy(s.points).cuda(), torch.from_numpy(s.weights).cuda())
    shp = (s.dims[1], s.dims[0])
    out = {"S": torch.empty(shp, dtype=torch.float32).pin_memory(),
           "dS": torch.empty((2,) + shp, dtype=torch.float32).pin_memory(),
           "sign": torch.empty(shp, dtype=torch.int8).pin_memory()}
    plan.execute_host(torch.from_numpy(s.points).pin_memory(), torch.from_numpy(s.weights).pin_memory(), out)
    for k in out:
        assert torch.equal(out[k], dev[k].cpu()), k


@pytest.mark.parametrize("pinned", [True, False])
def test_execute_host_fixup_outputs(pinned):
    # a small tau so that the fix-up rewrites many nodes: with pinned buffers
    # S, dS and d2S are written by the kernels straight into host memory,
    # with pageable ones they are staged on the device and copied
    s = wl.stars(N=256, K=3000, n_shapes=2, tau=0.004, seed=21)
    plan = pkg.Plan(2, s.dims, s.h, s.tau, precision="fp32", outputs=("S", "dS", "d2S", "sign"))
    dev = plan.execute(torch.from_numpy(s.points).cuda(), torch.from_numpy(s.weights).cuda())
    assert plan.stats().n_fixup_nodes > 0
    shp = (s.dims[1], s.dims[0])

    def host(shape, dtype):
        t = torch.empty(shape, dtype=dtype)
        return t.pin_memory() if pinned else t

    out = {"S": host(shp, torch.float32), "dS": host((2,) + shp, torch.float32),
           "d2S": host((3,) + shp, torch.float32), "sign": host(shp, torch.int8), "flags": host(shp, torch.uint8)}
    plan.execute_host(torch.from_numpy(s.points), torch.from_numpy(s.weights), out)
    for k in out:
        assert torch.equal(out[k], dev[k].cpu()), k


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_stats_match_flags(prec):
    """n_capped counts the nodes flagged CAPPED and n_fixup_nodes those the
    fix-up wrote (FIXUP without CAPPED), whichever kernel set the flag."""
    s = wl.stars(N=256, K=3000, n_shapes=2, tau=0.004, seed=21)
    res = run(s, prec, outputs=("S", "dS", "sign"))
    fl = res["flags"]
    st = res["stats"]
    capped = (fl & pkg.SDF_FLAG_CAPPED) != 0
    fixed = ((fl & pkg.SDF_FLAG_FIXUP) != 0) & ~capped
    assert capped.sum() > 0
    assert int(capped.sum()) == st.n_capped
    assert int(fixed.sum()) == st.n_fixup_nodes
    if prec == "fp32":
        assert st.n_fixup_nodes > 0
