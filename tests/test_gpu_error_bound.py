"""The per-result error report of sdf_get_stats (err_bound_S, err_bound_dS,
err_bound_d2S, trusted_frac): every bound must hold, and must not be vacuous
(at most 100 times the error actually measured).

* The 128^2 circle in both precisions, against the oracle at every node.
* The 2048^2 star workload at both tau: the mixed path against the plain FP64
  path over the whole grid (|S_32 - S_64| <= bound_32 + bound_64 where neither
  is capped), and each path against the oracle on sampled nodes."""
import numpy as np
import pytest
import torch

import paper_1112_3010_gb300 as pkg
from paper_1112_3010_gb300 import workloads as wl

from parity_util import oracle_ref

pytestmark = pytest.mark.gpu

RATIO = 100.0  # a bound at most this many times the measured error is not vacuous


def _run(s, prec, outs):
    plan = pkg.Plan(s.D, s.dims, s.h, s.tau, precision=prec, outputs=outs)
    res = plan.execute(torch.from_numpy(s.points).cuda(), torch.from_numpy(s.weights).cuda())
    st = plan.stats()
    plan.close()
    return res, st


def _unsigned(res):
    return (res["S"].double() * res["sign"].double()).cpu().numpy().ravel()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_bound_holds_against_oracle_circle(prec):
    s = wl.config_c1()
    res, st = _run(s, prec, ("S", "dS", "sign"))
    ref = oracle_ref(s, want=("S", "dS"))
    ok = (res["flags"].cpu().numpy().ravel() & pkg.SDF_FLAG_CAPPED) == 0
    assert abs(st.trusted_frac - ok.mean()) < 1e-12
    eS = np.abs(_unsigned(res)[ok] - ref["S"][ok]).max()
    G = res["dS"].double().cpu().numpy().reshape(2, -1).T
    eG = np.abs(G[ok] - ref["dS"][ok]).max()
    print("circle %s: |dS| %.3g <= %.3g, |dG| %.3g <= %.3g, trusted %.3f"
          % (prec, eS / s.tau, st.err_bound_S / s.tau, eG, st.err_bound_dS, st.trusted_frac))
    assert eS <= st.err_bound_S and st.err_bound_S <= RATIO * max(eS, 1e-300)
    assert eG <= st.err_bound_dS and st.err_bound_dS <= RATIO * max(eG, 1e-300)
    assert st.err_bound_d2S == 0.0   # not requested


def _sample(s, n_uniform=1500, n_near=1500, seed=21):
    rng = np.random.default_rng(seed)
    uni = rng.integers(0, s.n_nodes, n_uniform)
    k = rng.integers(0, s.K, n_near)
    d = rng.uniform(0.0, 30.0 * s.tau, n_near)
    v = rng.normal(size=(n_near, 2))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    idx = np.floor((s.points[k] + d[:, None] * v) / s.h + 0.5).astype(np.int64)
    ok = np.all((idx >= 0) & (idx < np.asarray(s.dims)), axis=1)
    idx = idx[ok]
    return np.unique(np.concatenate([uni, idx[:, 0] + s.dims[0] * idx[:, 1]]))


@pytest.mark.parametrize("tau", [0.002, 0.0005])
def test_bound_holds_mixed_against_fp64_stars_2048(tau):
    s = wl.config_c2(tau=tau)
    outs = ("S", "dS", "d2S", "sign")
    r32, s32 = _run(s, "fp32", outs)
    r64, s64 = _run(s, "fp64", outs)
    ok = ((r32["flags"] & pkg.SDF_FLAG_CAPPED) == 0) & ((r64["flags"] & pkg.SDF_FLAG_CAPPED) == 0)
    ok = ok.reshape(-1)
    # whole grid: mixed against FP64
    u32 = r32["S"].double() * r32["sign"].double()   # unsigned S (a sign may flip in the boundary band)
    u64 = r64["S"].double() * r64["sign"].double()
    d = {"S": ((u32 - u64).reshape(-1)[ok].abs().max().item(),
               s32.err_bound_S + s64.err_bound_S),
         "dS": ((r32["dS"].double() - r64["dS"].double()).reshape(2, -1)[:, ok].abs().max().item(),
                s32.err_bound_dS + s64.err_bound_dS),
         "d2S": ((r32["d2S"].double() - r64["d2S"].double()).reshape(3, -1)[:, ok].abs().max().item(),
                 s32.err_bound_d2S + s64.err_bound_d2S)}
    for k, (meas, bound) in d.items():
        print("stars %g %s: |32-64| %.3g <= bound %.3g (ratio %.1f)" % (tau, k, meas, bound, bound / meas))
        assert meas <= bound, k
        assert bound <= RATIO * meas, k
    assert abs(s32.trusted_frac - ((r32["flags"] & pkg.SDF_FLAG_CAPPED) == 0).double().mean().item()) < 1e-9
    # sampled nodes: each path against the oracle
    sel = _sample(s)
    ref = oracle_ref(s, sel=sel, want=("S", "dS", "d2S"))
    for res, st, name in ((r32, s32, "fp32"), (r64, s64, "fp64")):
        fl = res["flags"].cpu().numpy().ravel()[sel]
        keep = (fl & pkg.SDF_FLAG_CAPPED) == 0
        eS = np.abs(_unsigned(res)[sel][keep] - ref["S"][keep]).max()
        G = res["dS"].double().cpu().numpy().reshape(2, -1)[:, sel].T
        H = res["d2S"].double().cpu().numpy().reshape(3, -1)[:, sel].T
        eG = np.abs(G[keep] - ref["dS"][keep]).max()
        eH = np.abs(H[keep] - ref["d2S"][keep]).max()
        print("stars %g %s vs oracle: S %.3g/%.3g  dS %.3g/%.3g  d2S %.3g/%.3g"
              % (tau, name, eS, st.err_bound_S, eG, st.err_bound_dS, eH, st.err_bound_d2S))
        assert eS <= st.err_bound_S
        assert eG <= st.err_bound_dS
        assert eH <= st.err_bound_d2S
