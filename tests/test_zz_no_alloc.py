"""sdf_execute_noalloc: the whole path with no device allocation, for callers
that cannot call cudaMalloc (their device memory belongs to another
allocator, or their host forbids allocation after start-up).  Its scratch is a
static array inside the library.

Checked through the C ABI against the plan-based entry point (sdf_plan_create
+ sdf_execute) on the same inputs, within the parity tolerances the other GPU
tests use, on two calls in a row (the array keeps the previous call's
contents, so the second call shows that everything that must start at zero is
cleared).  This file is collected last so that a run stopping at the first
failure has already run every other test; it also passes alone."""
import numpy as np
import pytest
import torch

import paper_1112_3010_gb300 as pkg
from paper_1112_3010_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL_S, TOL_G, TOL_H = 1e-3, 1e-3, 1e-3   # S: x tau, grad: absolute, Hessian: / tau


def _outputs(dims, D, dtype, hess):
    shp = tuple(reversed(dims))
    o = {"S": torch.empty(shp, dtype=dtype, device="cuda"),
         "dS": torch.empty((D,) + shp, dtype=dtype, device="cuda"),
         "sign": torch.empty(shp, dtype=torch.int8, device="cuda"),
         "flags": torch.empty(shp, dtype=torch.uint8, device="cuda")}
    if hess:
        o["d2S"] = torch.empty((D * (D + 1) // 2,) + shp, dtype=dtype, device="cuda")
    return o


def _compare(a, b, tau):
    assert torch.equal(a["flags"], b["flags"])
    assert torch.equal(a["sign"], b["sign"])
    assert (a["S"].double() - b["S"].double()).abs().max().item() <= TOL_S * tau
    assert (a["dS"].double() - b["dS"].double()).abs().max().item() <= TOL_G
    if "d2S" in a:
        assert (a["d2S"].double() - b["d2S"].double()).abs().max().item() <= TOL_H / tau


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["circle2d", "stars2d_hessian", "sphere3d"])
def test_noalloc_matches_plan_execute(case, prec):
    if case == "circle2d":
        s, outs, hess = wl.config_c1(), ("S", "dS", "sign"), False
    elif case == "stars2d_hessian":
        s, outs, hess = wl.stars(N=200, K=3000, n_shapes=3, tau=0.008, seed=15), ("S", "dS", "d2S", "sign"), True
    else:
        s, outs, hess = wl.sphere(N=32, K=2000, radius=0.3, tau=0.04, seed=16), ("S", "dS", "sign"), False
    pts = torch.from_numpy(s.points).cuda()
    w = torch.from_numpy(s.weights).cuda()
    dtype = torch.float64 if prec == "fp64" else torch.float32
    plan = pkg.Plan(s.D, s.dims, s.h, s.tau, precision=prec, outputs=outs)
    ref = _outputs(s.dims, s.D, dtype, hess)
    pkg.sdf_execute(plan.handle, s.K, pts, w, ref["S"], ref["dS"], ref.get("d2S"), ref["sign"], ref["flags"])
    plan.sync()
    mask = 0
    for o in outs:
        mask |= {"S": 1, "dS": 2, "d2S": 4, "sign": 8}[o]
    p = pkg.SDF_FP64 if prec == "fp64" else pkg.SDF_FP32
    stream = torch.cuda.current_stream().cuda_stream
    gots = [_outputs(s.dims, s.D, dtype, hess) for _ in range(2)]
    for call, got in enumerate(gots):
        for t in got.values():
            t.fill_(0x5A if t.dtype in (torch.int8, torch.uint8) else 7.0)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        pkg.sdf_execute_noalloc(s.D, s.dims, s.h, s.tau, p, mask, s.K, pts, w, got["S"], got["dS"],
                                got.get("d2S"), got["sign"], got["flags"], stream)
        torch.cuda.synchronize()
        if call > 0:
            # no device memory was taken by the call (the first call may still
            # load the library's kernels; the array itself exists from load)
            assert torch.cuda.mem_get_info()[0] == free0
        _compare(got, ref, s.tau)
    plan.close()


def test_noalloc_stream_of_the_current_device_only():
    """A stream handle is checked against the current device; the default
    stream passes."""
    pts = torch.tensor([[0.5, 0.5]], dtype=torch.float64, device="cuda")
    S = torch.empty((16, 16), dtype=torch.float32, device="cuda")
    pkg.sdf_execute_noalloc(2, (16, 16), 1.0 / 16, 0.1, pkg.SDF_FP32, 1, 1, pts, None, S, None, None, None,
                            None, 0)
    torch.cuda.synchronize()
    assert torch.isfinite(S).all()


def test_noalloc_rejects_problems_beyond_its_scratch():
    """A 1024^2 grid needs far more than the static array: SDF_ERR_CAPACITY,
    reported before any device work."""
    pts = torch.tensor([[0.5, 0.5]], dtype=torch.float64, device="cuda")
    S = torch.empty((1024, 1024), dtype=torch.float32, device="cuda")
    with pytest.raises(pkg.SDFError) as ei:
        pkg.sdf_execute_noalloc(2, (1024, 1024), 1.0 / 1024, 0.01, pkg.SDF_FP32, 1, 1, pts, None, S, None,
                                None, None, None, torch.cuda.current_stream().cuda_stream)
    assert ei.value.code == 7
    assert b"scratch" in pkg._lib().sdf_last_error()
