"""Edge cases of the CUDA path against the oracle: the largest 2D grid the
library accepts (4096^2, 8192-point lines), the smallest grids (2 nodes per
axis, 16-point lines), ragged non-cubic 3D grids, tau far above the domain,
all-zero tangents, and the sizes the library refuses."""
import numpy as np
import pytest
import torch

import oracle
import paper_1112_3010_gb300 as pkg
from paper_1112_3010_gb300 import workloads as wl

from parity_util import check, oracle_ref, run

pytestmark = pytest.mark.gpu


def test_largest_2d_grid_sampled():
    # N = 4096 (padded 8192: the run-time-length FFT path), FP32 with the fix-up
    s = wl.stars(N=4096, K=40000, n_shapes=8, tau=0.001, seed=51)
    res = run(s, "fp32", outputs=("S", "dS", "d2S", "sign"))
    rng = np.random.default_rng(52)
    n = int(np.prod(s.dims))
    sel = rng.choice(n, 1500, replace=False)
    ref = oracle_ref(s, sel=sel)
    check(s, res, ref, sel=sel, label="4096-fp32")
    assert res["stats"].n_fixup_nodes > 0
    res["plan"].close()


def test_largest_3d_grid_sampled():
    # N = 512 per axis (padded 1024^3, ~70 GB at the plan-time peak), FP32
    # with the fix-up, sign from the degree of a sampled sphere
    s = wl.sphere(N=512, K=4000, radius=0.3, tau=2.0 / 512, seed=57)
    res = run(s, "fp32", outputs=("S", "dS", "sign"))
    rng = np.random.default_rng(58)
    n = int(np.prod(s.dims))
    sel = rng.choice(n, 1000, replace=False)
    ref = oracle_ref(s, sel=sel, want=("S", "dS", "mu", "R"))
    check(s, res, ref, sel=sel, check_hess=False, label="512^3-fp32")
    assert res["stats"].n_fixup_nodes > 0
    res["plan"].close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("D", [2, 3])
def test_smallest_grids(D, prec):
    # 2 (and 3) nodes per axis: padded to 16, one radix-16 stage per line
    for N in (2, 3):
        dims = (N,) * D
        h = 0.5
        P = np.array([[0.0] * D, [h * (N - 1)] + [0.0] * (D - 1)])
        s = wl.Shape(D, dims, h, 0.3, P, None)
        res = run(s, prec, outputs=("S", "dS", "d2S"), with_weights=False)
        ref = oracle_ref(s, with_weights=False, want=("S", "dS", "d2S", "R"))
        check(s, res, ref, check_sign=False, label="N%d-%dD-%s" % (N, D, prec))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ragged_3d_dims(prec):
    dims = (20, 33, 17)
    h = 1.0 / 33
    rng = np.random.default_rng(53)
    P = rng.uniform(0, 1, size=(400, 3)) * (np.array(dims) - 1) * h
    W = rng.normal(size=(400, 3)) * 1e-3
    s = wl.Shape(3, dims, h, 1.2 * h, P, W)
    res = run(s, prec, outputs=("S", "dS", "d2S", "sign"))
    ref = oracle_ref(s)
    check(s, res, ref, label="ragged3d-" + prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tau_far_above_the_domain(prec):
    # phi nearly constant: S ~ R - tau log K, all trusted
    s = wl.stars(N=96, K=800, n_shapes=2, tau=2.0, seed=54)
    res = run(s, prec, outputs=("S", "dS", "d2S", "sign"))
    assert ((res["flags"] & pkg.SDF_FLAG_CAPPED) == 0).all()
    ref = oracle_ref(s)
    check(s, res, ref, label="bigtau-" + prec)


def test_zero_tangents_give_outside_everywhere():
    s = wl.stars(N=96, K=800, n_shapes=2, tau=0.02, seed=55)
    s = wl.Shape(2, s.dims, s.h, s.tau, s.points, np.zeros_like(s.weights))
    res = run(s, "fp32", outputs=("S", "dS", "sign"))
    src = (res["flags"] & pkg.SDF_FLAG_SOURCE) != 0
    assert np.all(res["sign"][~src] == -1)


def test_refused_sizes():
    for D, dims in ((2, (4097, 16)), (2, (1, 16)), (3, (513, 8, 8)), (4, (8, 8, 8, 8))):
        with pytest.raises(pkg.SDFError):
            pkg.Plan(D, dims, 0.01, 0.02, precision="fp32", outputs=("S",))
    s = wl.config_c1()
    plan = pkg.Plan(2, s.dims, s.h, s.tau, precision="fp32", outputs=("S",))
    with pytest.raises(pkg.SDFError):  # K = 0
        pkg.sdf_execute(plan.handle, 0, torch.zeros((1, 2), dtype=torch.float64, device="cuda"), None,
                        torch.zeros(s.dims, device="cuda"), None, None, None, None)
    plan.close()
