"""GPU parity of the exact Green's function kernel set (sdf_plan_set_kernel with
SDF_KERNEL_GREEN, SDF_FP64 plans) against oracle/green.py, element by element
over the FP64 trust region, with the tolerances of parity_util (S within
1e-3 tau, grad S within 1e-3, Hessian within 1e-3/tau).  The sign does not
depend on the kernel set and is checked against the oracle's mu."""
import numpy as np
import pytest
import torch

import oracle
from oracle import green
import paper_1112_3010_gb300 as pkg
from paper_1112_3010_gb300 import workloads as wl

from parity_util import check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    pkg.load_library()


def run_green(s, outputs=("S", "dS", "d2S", "sign")):
    plan = pkg.Plan(s.D, s.dims, s.h, s.tau, precision="fp64", outputs=outputs, kernel="green")
    out = plan.execute(torch.from_numpy(s.points).cuda(),
                       torch.from_numpy(s.weights).cuda() if s.weights is not None else None)
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["stats"] = plan.stats()
    res["plan"] = plan
    return res


def green_ref(s, sel=None, want=("S", "dS", "d2S")):
    idx, inside = oracle.snap(s.points, s.h, s.dims)
    Y = idx[inside].astype(np.float64) * s.h
    X = oracle.grid_nodes(s.dims, s.h, sel)
    ref = green.evaluate(Y, X, s.tau, want=want)
    if s.weights is not None:
        W = s.weights[inside]
        geo = oracle.evaluate(Y, X, s.tau, weights=W, want=("mu", "R"))
        ref["mu"], ref["R"], ref["W"] = geo["mu"], geo["R"], W
    ref["X"], ref["Y"] = X, Y
    return ref


def test_stars_2d_ragged_with_hessian():
    """Non-square grid (ragged bins, padded size above 2N), three star polygons."""
    s = wl.stars(N=256, K=2000, n_shapes=3, tau=0.006, seed=5)
    s.dims = (200, 168)
    s.points = s.points * np.array([200 / 256, 168 / 256])
    s.weights = s.weights * np.array([200 / 256, 168 / 256])
    res = run_green(s)
    ref = green_ref(s)
    rep = check(s, res, ref, label="green-stars")
    assert rep["trusted"] > 0.3 * rep["n"]


def test_circle_c1_green():
    s = wl.config_c1()
    res = run_green(s, outputs=("S", "dS", "sign"))
    ref = green_ref(s, want=("S", "dS"))
    check(s, res, ref, check_hess=False, label="green-c1")


def test_sphere_3d():
    s = wl.sphere(N=32, K=2000, radius=0.3, tau=0.04, seed=8)
    res = run_green(s)
    ref = green_ref(s)
    check(s, res, ref, label="green-sphere")


def test_isolated_source_node_closed_form():
    """A single point on a node: phi there is tau^-D/2 c_D A_D (the box
    integral of Sec. 2.2), so S = -tau log(tau^-D/2 c_D A_D); with m coincident
    points, minus tau log m."""
    for D, N in ((2, 64), (3, 24)):
        tau, h = 0.05, 1.0 / N
        c = [N // 2] * D
        P = np.tile(np.array(c, dtype=np.float64) * h, (3, 1))
        s = wl.Shape(D, (N,) * D, h, tau, P, None)
        res = run_green(s, outputs=("S", "dS"))
        A = pkg.sdf_green_profile(D, [0.0])[0][0]
        ref = -tau * np.log(tau ** (-D / 2) * green.C_D[D] * A) - tau * np.log(3)
        # the grid's value at the source node (x fastest: reversed axes)
        S = res["S"][tuple(reversed(c))]
        assert abs(S - ref) <= 1e-9 * tau
        assert np.all(np.abs(res["dS"][(slice(None),) + tuple(reversed(c))]) < 1e-9)


def test_fullsize_2048_sampled_nodes():
    """The 2048^2 star workload (K = 40000, tau = 0.002) with the Green set, on
    sampled nodes the oracle sums one by one: half near the curves, half
    uniform."""
    s = wl.config_c2(tau=0.002)
    res = run_green(s, outputs=("S", "dS", "sign"))
    rng = np.random.default_rng(17)
    n = int(np.prod(s.dims))
    flags = res["flags"].reshape(-1)
    trusted = np.flatnonzero((flags & pkg.SDF_FLAG_CAPPED) == 0)
    sel = np.sort(np.concatenate([rng.choice(trusted, 192, replace=False), rng.choice(n, 64, replace=False)]))
    ref = green_ref(s, sel=sel, want=("S", "dS"))
    check(s, res, ref, sel=sel, check_hess=False, label="green-2048")


def test_switching_sets_restores_exp_bitwise():
    s = wl.stars(N=128, K=1500, n_shapes=2, tau=0.01, seed=3)
    a = pkg.Plan(2, s.dims, s.h, s.tau, precision="fp64", outputs=("S", "dS", "d2S", "sign"))
    x, w = torch.from_numpy(s.points).cuda(), torch.from_numpy(s.weights).cuda()
    ref = {k: v.clone() for k, v in a.execute(x, w).items()}
    a.set_kernel("green")
    g = a.execute(x, w)
    assert not torch.equal(g["S"], ref["S"])
    a.set_kernel("exp")
    back = a.execute(x, w)
    for k in ref:
        assert torch.equal(back[k], ref[k]), k


def test_unsupported_combinations():
    s = wl.config_c1()
    p32 = pkg.Plan(2, s.dims, s.h, s.tau, precision="fp32", outputs=("S", "dS"))
    with pytest.raises(pkg.SDFError) as ei:
        p32.set_kernel("green")
    assert ei.value.code == 2
    p = pkg.Plan(2, s.dims, s.h, s.tau, precision="fp64", outputs=("S", "dS"), kernel="green")
    x = torch.from_numpy(s.points).cuda()
    out = p.execute(x)
    w = torch.ones_like(out["S"])
    with pytest.raises(pkg.SDFError) as ei:
        p.backward(x, w, out["S"], out["flags"])
    assert ei.value.code == 2
