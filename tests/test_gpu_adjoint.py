"""GPU parity of the adjoint (sdf_backward) against the oracle's analytic
gradient of L = sum_X w(X) S(X), and the autograd wrapper.

Loss weights: seeded N(0, 1) per node, zeroed outside a band around the
surface chosen a priori from the geometry (so that phi there is far above
the float transform's trust threshold; a = w/phi stays moderate).  Points are
snapped before use, so the forward values agree with the oracle's continuous
definition evaluated at the same positions.

Tolerances: max |dL/dY - oracle| <= 2e-3 * max |oracle| (float plan),
1e-6 * max |oracle| (double plan); |dL/dtau - oracle| <= 2e-3 |oracle| (float),
1e-6 (double)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1112_3010_gb300 as pkg
from paper_1112_3010_gb300 import workloads as wl
from paper_1112_3010_gb300.autograd import sdf

pytestmark = pytest.mark.gpu

TOL = {"fp32": 2e-3, "fp64": 1e-6}


def _snapped(s):
    idx, inside = oracle.snap(s.points, s.h, s.dims)
    assert inside.all()
    return idx.astype(np.float64) * s.h


def _band_weights(s, center, radius, half_width, seed):
    X = oracle.grid_nodes(s.dims, s.h)
    d = np.abs(np.linalg.norm(X - np.asarray(center), axis=1) - radius)
    w = wl.loss_weights(s.n_nodes, seed=seed)
    w[d > half_width] = 0.0
    return w


def _run(s, prec, Y, w, tune=False):
    plan = pkg.Plan(s.D, s.dims, s.h, s.tau, precision=prec, outputs=("S", "dS"))
    pts = torch.from_numpy(Y).cuda()
    if tune:
        pkg.sdf_plan_autotune(plan.handle, pts.shape[0], pts, None, 2)
    out = plan.execute(pts, None)
    dt = torch.float64 if prec == "fp64" else torch.float32
    wt = torch.from_numpy(w).to(dt).cuda().reshape(out["S"].shape)
    dY, dtau = plan.backward(pts, wt, out["S"], out["flags"])
    flags = out["flags"].cpu().numpy().ravel()
    plan.close()
    return dY.cpu().numpy(), float(dtau.item()), flags


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_adjoint_3d_small_all_points(prec):
    s = wl.jittered_sphere(N=40, K=1500, radius=0.3, sigma=0.01, tau=0.03, seed=21)
    Y = _snapped(s)
    s.points = Y
    w = _band_weights(s, (0.5, 0.5, 0.5), 0.3, 0.03, seed=51)
    dY, dtau, flags = _run(s, prec, Y, w)
    assert not np.any((flags != 0) & (flags != pkg.SDF_FLAG_SOURCE) & (w != 0)), "weights on untrusted nodes"
    X = oracle.grid_nodes(s.dims, s.h)
    keep = w != 0
    rY, rt = oracle.adjoint(Y, X[keep], w[keep], s.tau)
    tol = TOL[prec]
    assert np.abs(dY - rY).max() <= tol * np.abs(rY).max()
    assert abs(dtau - rt) <= tol * abs(rt)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_adjoint_2d_circle(prec):
    s = wl.circle(N=96, K=200, radius=0.3, center=(0.5, 0.5), tau=0.02)
    Y = _snapped(s)
    s.points = Y
    w = _band_weights(s, (0.5, 0.5), 0.3, 0.04, seed=52)
    dY, dtau, flags = _run(s, prec, Y, w)
    X = oracle.grid_nodes(s.dims, s.h)
    keep = w != 0
    rY, rt = oracle.adjoint(Y, X[keep], w[keep], s.tau)
    tol = TOL[prec]
    assert np.abs(dY - rY).max() <= tol * np.abs(rY).max()
    assert abs(dtau - rt) <= tol * abs(rt)


@pytest.mark.parametrize("tune", [False, True])
def test_adjoint_differentiation_workload_full_size(tune, tmp_path, monkeypatch):
    """The 3D differentiation workload: 128^3 grid, K = 20000 jittered sphere
    points (sigma 0.01), tau = 0.01, float plan; every point's gradient, with
    the default tile schedule and with the autotuner's (as the bench runs it)."""
    monkeypatch.setenv("SDF_AUTOTUNE_CACHE", str(tmp_path / "autotune.tsv"))
    s = wl.config_c5()
    Y = _snapped(s)
    s.points = Y
    w = _band_weights(s, (0.5, 0.5, 0.5), 0.3, 0.01, seed=50)
    dY, dtau, _ = _run(s, "fp32", Y, w, tune=tune)
    X = oracle.grid_nodes(s.dims, s.h)
    keep = w != 0
    rY, rt = oracle.adjoint(Y, X[keep], w[keep], s.tau)
    scale = np.abs(rY).max()
    err = np.abs(dY - rY).max()
    print("c5 adjoint: max|err|/max|ref| = %.3g, dtau rel err = %.3g" % (err / scale, abs(dtau - rt) / abs(rt)))
    assert err <= TOL["fp32"] * scale
    assert abs(dtau - rt) <= TOL["fp32"] * abs(rt)


def test_autograd_function_matches_backward():
    s = wl.jittered_sphere(N=32, K=800, radius=0.3, sigma=0.01, tau=0.04, seed=23)
    Y = _snapped(s)
    w = _band_weights(s, (0.5, 0.5, 0.5), 0.3, 0.04, seed=53)
    plan = pkg.Plan(3, s.dims, s.h, s.tau, precision="fp64", outputs=("S", "dS"))
    pts = torch.from_numpy(Y).cuda().requires_grad_(True)
    tau = torch.tensor(s.tau, dtype=torch.float64, requires_grad=True)
    S = sdf(pts, tau, plan)
    wt = torch.from_numpy(w).cuda().reshape(S.shape)
    loss = (wt * S).sum()
    loss.backward()
    X = oracle.grid_nodes(s.dims, s.h)
    keep = w != 0
    rY, rt = oracle.adjoint(Y, X[keep], w[keep], s.tau)
    g = pts.grad.cpu().numpy()
    assert np.abs(g - rY).max() <= 1e-6 * np.abs(rY).max()
    assert abs(float(tau.grad) - rt) <= 1e-6 * abs(rt)
    plan.close()
