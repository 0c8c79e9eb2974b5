"""Failure paths, made on purpose without faulting or hanging the GPU
(sdf_debug_hook):

* a device allocation that fails (as an exhausted device would): plan creation
  and the first execute report SDF_ERR_OOM, release what they allocated, and
  the library works again afterwards;
* the epilogue's TMA waits poll a barrier that nothing completes and so
  expire on their first group while its copy is in flight: each CTA lets its
  copy land (a bounded wait), the execute reports SDF_ERR_TIMEOUT through
  sdf_sync, and the same plan then produces the normal result."""
import pytest
import torch

import paper_1112_3010_gb300 as pkg
from paper_1112_3010_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _reset_hooks():
    pkg.load_library()
    yield
    pkg.sdf_debug_hook(pkg.SDF_HOOK_FAIL_ALLOC, 0)
    pkg.sdf_debug_hook(pkg.SDF_HOOK_TMA_WAIT_POLLS, 0)


def _shape():
    return wl.stars(N=256, K=3000, n_shapes=3, tau=0.004, seed=61)


@pytest.mark.parametrize("nth", [1, 3, 7, 12])
def test_allocation_failure_in_plan_creation(nth):
    s = _shape()
    # the same plan once first: its kernels are loaded (module loading takes
    # device memory too, and must not count as a leak below)
    warm = pkg.Plan(2, s.dims, s.h, s.tau, precision="fp32", outputs=("S", "dS", "d2S", "sign"))
    warm.execute(torch.from_numpy(s.points).cuda(), torch.from_numpy(s.weights).cuda())
    warm.close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    pkg.sdf_debug_hook(pkg.SDF_HOOK_FAIL_ALLOC, nth)
    with pytest.raises(pkg.SDFError) as ei:
        pkg.Plan(2, s.dims, s.h, s.tau, precision="fp32", outputs=("S", "dS", "d2S", "sign"))
    assert ei.value.code == 4   # SDF_ERR_OOM
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0   # everything allocated was released
    plan = pkg.Plan(2, s.dims, s.h, s.tau, precision="fp32", outputs=("S", "dS", "d2S", "sign"))
    out = plan.execute(torch.from_numpy(s.points).cuda(), torch.from_numpy(s.weights).cuda())
    assert torch.isfinite(out["S"]).all()
    plan.close()


def test_allocation_failure_in_first_execute_leaves_plan_usable():
    s = _shape()
    plan = pkg.Plan(2, s.dims, s.h, s.tau, precision="fp32", outputs=("S", "sign"))
    pts = torch.from_numpy(s.points).cuda()
    w = torch.from_numpy(s.weights).cuda()
    pkg.sdf_debug_hook(pkg.SDF_HOOK_FAIL_ALLOC, 2)   # among the point buffers of the first execute
    with pytest.raises(pkg.SDFError) as ei:
        plan.execute(pts, w)
    assert ei.value.code == 4
    out = plan.execute(pts, w)
    ref = pkg.Plan(2, s.dims, s.h, s.tau, precision="fp32", outputs=("S", "sign"))
    r = ref.execute(pts, w)
    assert torch.equal(out["S"], r["S"]) and torch.equal(out["sign"], r["sign"])
    plan.close()
    ref.close()


def test_tma_wait_expiry_reports_timeout_and_plan_recovers():
    s = _shape()   # 256^2 padded to 512^2: the TMA epilogue applies (16 lines per CTA)
    pts = torch.from_numpy(s.points).cuda()
    w = torch.from_numpy(s.weights).cuda()
    plan = pkg.Plan(2, s.dims, s.h, s.tau, precision="fp32", outputs=("S", "dS", "sign"))
    ref = plan.execute(pts, w)
    ref = {k: v.clone() for k, v in ref.items()}
    pkg.sdf_debug_hook(pkg.SDF_HOOK_TMA_WAIT_POLLS, 1)
    with pytest.raises(pkg.SDFError) as ei:
        plan.execute(pts, w)
    assert ei.value.code == 6   # SDF_ERR_TIMEOUT, read back by sdf_sync
    pkg.sdf_debug_hook(pkg.SDF_HOOK_TMA_WAIT_POLLS, 0)
    again = plan.execute(pts, w)
    for k in ref:
        assert torch.equal(again[k], ref[k]), k
    # per-thread loads never wait on a barrier: the hook does not touch them
    pkg.sdf_debug_hook(pkg.SDF_HOOK_TMA_WAIT_POLLS, 1)
    pkg.sdf_plan_set_epilogue_loads(plan.handle, 1)
    plain = plan.execute(pts, w)
    for k in ref:
        assert torch.equal(plain[k], ref[k]), k
    plan.close()
