"""GPU parity of the 1D path (D = 1 plans, one CTA per execute) against the
FP64 oracle: every node of lines that span several radix-16 stages and a
ragged end (N not a power of two), both precisions, the FP32 fix-up and full
range, the exact Green's function set, and the edges (smallest and largest
lines, all points on one node, points off the grid)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import green
import paper_1112_3010_gb300 as pkg
from paper_1112_3010_gb300 import workloads as wl

from parity_util import TOL_G, TOL_H, TOL_S, check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    pkg.load_library()


def line(N, K, tau_over_h, seed, lo=0.3, hi=0.7):
    """K points uniform in [lo, hi) of the line [0, 1) with N nodes (h = 1/N)."""
    rng = np.random.default_rng(seed)
    h = 1.0 / N
    P = rng.uniform(lo, hi, (K, 1))
    return wl.Shape(1, (N,), h, tau_over_h * h, P, None)


def run(s, prec, full=False, kernel="exp", outputs=("S", "dS", "d2S")):
    plan = pkg.Plan(1, s.dims, s.h, s.tau, precision=prec, outputs=outputs, full_range=full, kernel=kernel)
    out = plan.execute(torch.from_numpy(s.points).cuda())
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["stats"] = plan.stats()
    res["plan"] = plan
    return res


def ref_of(s, kernel="exp"):
    idx, inside = oracle.snap(s.points, s.h, s.dims)
    Y = idx[inside].astype(np.float64) * s.h
    X = oracle.grid_nodes(s.dims, s.h)
    if kernel == "green":
        ref = green.evaluate(Y, X, s.tau)
    else:
        ref = oracle.evaluate(Y, X, s.tau, want=("S", "dS", "d2S", "R"))
    ref["X"], ref["Y"] = X, Y
    return ref


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("N,K,th", [(1000, 300, 1.5), (2048, 2000, 0.75), (37, 5, 2.0)])
def test_line_matches_oracle(prec, N, K, th):
    s = line(N, K, th, seed=N + K)
    res = run(s, prec)
    rep = check(s, res, ref_of(s), check_sign=False, label="1d-%s-%d" % (prec, N))
    assert rep["trusted"] > 0


def test_fp32_fixup_is_exercised():
    """tau = h: far nodes fall below theta_32; the direct sum recomputes them,
    caps those below theta_64 and matches the oracle on the rest."""
    s = line(1500, 40, 1.0, seed=3, lo=0.45, hi=0.55)
    res = run(s, "fp32")
    st = res["stats"]
    assert st.n_fixup_nodes > 0 and st.n_capped > 0
    fix = (res["flags"] & pkg.SDF_FLAG_FIXUP) != 0
    # recomputed nodes keep FIXUP unless the exact sum put them below theta_64
    assert 0 < fix.sum() == st.n_fixup_nodes
    assert ((res["flags"] & pkg.SDF_FLAG_CAPPED) != 0).sum() == st.n_capped
    check(s, res, ref_of(s), check_sign=False, label="1d-fixup")


def test_full_range_every_node():
    s = line(1024, 20, 0.5, seed=4, lo=0.4, hi=0.6)
    res = run(s, "fp32", full=True)
    assert res["stats"].n_capped == 0
    assert ((res["flags"] & pkg.SDF_FLAG_CAPPED) == 0).all()
    ref = ref_of(s)
    assert np.abs(res["S"].astype(np.float64) - ref["S"]).max() <= TOL_S * s.tau
    assert np.abs(res["dS"][0].astype(np.float64) - ref["dS"][:, 0]).max() <= TOL_G
    assert np.abs(res["d2S"][0].astype(np.float64) - ref["d2S"][:, 0]).max() <= TOL_H / s.tau


def test_green_set():
    s = line(1200, 400, 1.2, seed=6)
    res = run(s, "fp64", kernel="green")
    check(s, res, ref_of(s, "green"), check_sign=False, label="1d-green")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_smallest_line_and_one_node(prec):
    """N = 2 (a 16-point transform, one thread) and all points on one node."""
    s = wl.Shape(1, (2,), 0.5, 0.3, np.array([[0.0], [0.0], [0.1]]), None)
    res = run(s, prec)
    check(s, res, ref_of(s), check_sign=False, label="1d-n2")
    assert res["flags"][0] & pkg.SDF_FLAG_SOURCE


def test_points_off_the_grid_reported():
    s = line(256, 10, 1.0, seed=8)
    plan = pkg.Plan(1, s.dims, s.h, s.tau, precision="fp32", outputs=("S",))
    bad = np.concatenate([s.points, [[1.5]]])
    with pytest.raises(pkg.SDFError) as ei:
        plan.execute(torch.from_numpy(bad).cuda())
    assert ei.value.code == 3
    out = plan.execute(torch.from_numpy(s.points).cuda())
    assert torch.isfinite(out["S"]).all()


def test_execute_host_matches_device():
    s = line(900, 200, 1.0, seed=9)
    plan = pkg.Plan(1, s.dims, s.h, s.tau, precision="fp32", outputs=("S", "dS", "d2S"))
    dev = plan.execute(torch.from_numpy(s.points).cuda())
    out = {"S": torch.empty(900, dtype=torch.float32).pin_memory(),
           "dS": torch.empty((1, 900), dtype=torch.float32).pin_memory(),
           "d2S": torch.empty((1, 900), dtype=torch.float32)}
    plan.execute_host(torch.from_numpy(s.points), None, out)
    for k in out:
        assert torch.equal(out[k], dev[k].cpu()), k


def test_unsupported_in_1d():
    with pytest.raises(pkg.SDFError) as ei:
        pkg.Plan(1, (64,), 1 / 64, 0.02, precision="fp32", outputs=("S", "sign"))
    assert ei.value.code == 2
    with pytest.raises(pkg.SDFError) as ei:
        pkg.Plan(1, (4096,), 1 / 4096, 0.001, precision="fp32", outputs=("S",))
    assert ei.value.code == 2
    s = line(128, 10, 1.0, seed=1)
    p = pkg.Plan(1, s.dims, s.h, s.tau, precision="fp64", outputs=("S", "dS"))
    x = torch.from_numpy(s.points).cuda()
    out = p.execute(x)
    with pytest.raises(pkg.SDFError) as ei:
        p.backward(x, torch.ones_like(out["S"]), out["S"], out["flags"])
    assert ei.value.code == 2
