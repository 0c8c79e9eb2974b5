"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and compare it with the FP64 oracle on the same seeded inputs.

Tolerances (over the FP64 trust region, i.e. nodes not flagged CAPPED):
  |S - S_oracle|          <= 1e-3 tau
  |dS - dS_oracle|        <= 1e-3
  |d2S - d2S_oracle|      <= 1e-3 / tau
Trust-mask consistency: a node is capped only if the oracle's phi is below
theta_64 up to a 1% margin, and trusted only if above it up to the same margin.
Sign: exact off the boundary band -- nodes farther than 2 max|weight| + h sqrt(D)
from every snapped point and with ||mu_oracle| - 1/2| >= 0.05.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
import paper_1112_3010_gb300 as pkg

TOL_S = 1e-3      # times tau
TOL_G = 1e-3
TOL_H = 1e-3      # divided by tau


def run(shape, precision="fp64", outputs=("S", "dS", "d2S", "sign"), with_weights=True):
    D = shape.D
    plan = pkg.Plan(D, shape.dims, shape.h, shape.tau, precision=precision, outputs=outputs)
    pts = torch.from_numpy(shape.points).cuda()
    w = torch.from_numpy(shape.weights).cuda() if (with_weights and shape.weights is not None) else None
    out = plan.execute(pts, w)
    st = plan.stats()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["stats"] = st
    res["plan"] = plan
    return res


def oracle_ref(shape, sel=None, with_weights=True, want=("S", "dS", "d2S", "mu", "R")):
    idx, inside = oracle.snap(shape.points, shape.h, shape.dims)
    Y = idx[inside].astype(np.float64) * shape.h
    W = shape.weights[inside] if (with_weights and shape.weights is not None) else None
    X = oracle.grid_nodes(shape.dims, shape.h, sel)
    ref = oracle.evaluate(Y, X, shape.tau, weights=W, want=want)
    ref["Y"] = Y
    ref["W"] = W
    ref["X"] = X
    return ref


def sample_nodes(s, n_uniform=1000, n_near=2000, seed=7, reach=40.0):
    """Seeded node sample of a workload, from its input geometry only:
    uniform random nodes plus nodes at random distances 0..reach*tau from
    random points, so the near band, the fix-up band and the capped far field
    are all represented.  Returns sorted unique flat node indices."""
    rng = np.random.default_rng(seed)
    D = s.D
    uni = rng.integers(0, s.n_nodes, n_uniform)
    k = rng.integers(0, s.K, n_near)
    d = rng.uniform(0.0, reach * s.tau, n_near)
    v = rng.normal(size=(n_near, D))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    P = s.points[k] + d[:, None] * v
    idx = np.floor(P / s.h + 0.5).astype(np.int64)
    dims = np.asarray(s.dims)
    ok = np.all((idx >= 0) & (idx < dims), axis=1)
    idx = idx[ok]
    flat_idx = idx[:, 0] + dims[0] * (idx[:, 1] + (dims[1] * idx[:, 2] if D == 3 else 0))
    return np.unique(np.concatenate([uni, flat_idx]))


def flat(a, D, planes=False):
    if planes:
        return a.reshape(a.shape[0], -1)
    return a.reshape(-1)


def check(shape, res, ref, sel=None, check_hess=True, check_sign=True, label=""):
    D = shape.D
    tau = shape.tau
    n = int(np.prod(shape.dims))
    sel = np.arange(n) if sel is None else np.asarray(sel)
    flags = flat(res["flags"], D)[sel]
    capped = (flags & pkg.SDF_FLAG_CAPPED) != 0
    ok = ~capped
    sign = flat(res["sign"], D)[sel].astype(np.float64) if "sign" in res else np.ones(len(sel))
    S = flat(res["S"], D)[sel].astype(np.float64) * sign
    st = res["stats"]
    report = {"n": len(sel), "trusted": int(ok.sum()), "capped": int(capped.sum())}
    # trust-mask consistency
    scap = st.s_cap
    margin = tau * np.log(1.01)
    assert np.all(ref["S"][capped] > scap - margin), (label, "capped a node inside the trust region")
    assert np.all(ref["S"][ok] < scap + margin), (label, "trusted a node outside the trust region")
    if capped.any():
        np.testing.assert_allclose(S[capped], scap, rtol=1e-6, err_msg=label + " capped S")
    eS = np.abs(S[ok] - ref["S"][ok])
    report["max_dS"] = float(eS.max()) if eS.size else 0.0
    assert report["max_dS"] <= TOL_S * tau, (label, "S", report["max_dS"] / tau)
    if "dS" in res:
        G = flat(res["dS"], D, planes=True)[:, sel].T.astype(np.float64)
        eG = np.abs(G[ok] - ref["dS"][ok]).max() if ok.any() else 0.0
        report["max_dG"] = float(eG)
        assert eG <= TOL_G, (label, "grad", eG)
        assert np.all(G[capped] == 0)
    if check_hess and "d2S" in res:
        H = flat(res["d2S"], D, planes=True)[:, sel].T.astype(np.float64)
        eH = np.abs(H[ok] - ref["d2S"][ok]).max() if ok.any() else 0.0
        report["max_dH_tau"] = float(eH * tau)
        assert eH <= TOL_H / tau, (label, "hess", eH * tau)
    if check_sign and "sign" in res and ref.get("mu") is not None:
        band = 2 * np.linalg.norm(ref["W"], axis=1).max() + shape.h * np.sqrt(D)
        d = ref["R"]
        mu = ref["mu"]
        off = (d > band) & (np.abs(np.abs(mu) - 0.5) >= 0.05)
        mism = int((flat(res["sign"], D)[sel][off] != oracle.sign_from_mu(mu[off])).sum())
        report["sign_checked"] = int(off.sum())
        report["sign_mismatch"] = mism
        assert mism == 0, (label, "sign mismatches", mism)
    return report
