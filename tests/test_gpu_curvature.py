"""Curvature fields (sdf_curvature) against the oracle.

Two checks per case:
  * the kernel's arithmetic: GPU curvature vs oracle.curvature applied to the
    GPU's own grad S and Hessian (FP64 plans: 1e-9 relative; FP32 plans:
    1e-4 relative to each field's largest value);
  * end to end: GPU curvature vs oracle.curvature of the oracle's derivatives
    at sampled trusted nodes, with a tolerance carried from the derivative
    tolerances (|d grad S| <= 1e-3, |d Hess| <= 1e-3/tau) through the
    formulas.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1112_3010_gb300 as pkg
from paper_1112_3010_gb300 import workloads as wl

from parity_util import oracle_ref

pytestmark = pytest.mark.gpu


def _gpu(shape, precision):
    plan = pkg.Plan(shape.D, shape.dims, shape.h, shape.tau, precision=precision, outputs=("S", "dS", "d2S"))
    out = plan.execute(torch.from_numpy(shape.points).cuda())
    curv = plan.curvature(out)
    n = int(np.prod(shape.dims))
    D = shape.D
    res = {"dS": out["dS"].reshape(D, n).T.double().cpu().numpy(),
           "d2S": out["d2S"].reshape(D * (D + 1) // 2, n).T.double().cpu().numpy(),
           "flags": out["flags"].reshape(n).cpu().numpy(),
           "curv": curv.reshape(4, n).T.double().cpu().numpy()}
    plan.close()
    return res


CASES = [("2d", lambda: wl.stars(N=128, K=2000, n_shapes=2, tau=0.01, seed=31)),
         ("3d", lambda: wl.torus_sphere(N=32, K=3000, tau=0.04, seed=32))]


@pytest.mark.parametrize("name,make", CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_curvature_kernel_arithmetic(name, make, precision):
    s = make()
    r = _gpu(s, precision)
    ok = (r["flags"] & pkg.SDF_FLAG_CAPPED) == 0
    assert ok.sum() > 100
    want = oracle.curvature(r["dS"][ok], r["d2S"][ok])
    got = r["curv"][ok]
    if s.D == 3:
        # level surfaces: 1/|grad S| amplifies rounding where grad S is small
        keep = np.linalg.norm(r["dS"][ok], axis=1) > 0.2
        want, got = want[keep], got[keep]
    for c in range(4):
        scale = max(1.0, float(np.abs(want[:, c]).max()))
        tol = 1e-9 if precision == "fp64" else 1e-4
        err = float(np.abs(got[:, c] - want[:, c]).max())
        assert err <= tol * scale, (name, precision, c, err, scale)
    # capped nodes get zeros
    assert np.all(r["curv"][~ok] == 0)


@pytest.mark.parametrize("name,make", CASES)
def test_curvature_end_to_end_fp64(name, make):
    s = make()
    r = _gpu(s, "fp64")
    n = int(np.prod(s.dims))
    rng = np.random.default_rng(7)
    trusted = np.flatnonzero((r["flags"] & pkg.SDF_FLAG_CAPPED) == 0)
    sel = rng.choice(trusted, size=min(400, trusted.size), replace=False)
    ref = oracle_ref(s, sel=sel, with_weights=False, want=("S", "dS", "d2S"))
    want = oracle.curvature(ref["dS"], ref["d2S"])
    got = r["curv"][sel]
    tau = s.tau
    hmax = float(np.abs(ref["d2S"]).max())
    if s.D == 2:
        # H is linear in the Hessian with coefficients <= 2, plus gradient
        # terms times the Hessian; K is quadratic in the Hessian
        tol_H = 4e-3 / tau + 4e-3 * hmax
        tol_K = 6e-3 / tau * hmax + 1e-5 / tau ** 2
        keep = np.ones(len(sel), bool)
    else:
        keep = np.linalg.norm(ref["dS"], axis=1) > 0.5
        tol_H = 1e-2 / tau + 1e-2 * hmax
        tol_K = 2e-2 / tau * hmax + 1e-5 / tau ** 2
    assert keep.sum() > 50
    eH = float(np.abs(got[keep, 1] - want[keep, 1]).max())
    eK = float(np.abs(got[keep, 0] - want[keep, 0]).max())
    assert eH <= tol_H, (name, eH, tol_H)
    assert eK <= tol_K, (name, eK, tol_K)


def test_curvature_rejects_null_planes():
    s = wl.config_c1()
    plan = pkg.Plan(2, s.dims, s.h, s.tau, precision="fp32", outputs=("S", "dS", "d2S"))
    with pytest.raises(pkg.SDFError):
        pkg.sdf_curvature(plan.handle, None, None, None, None)
    plan.close()
