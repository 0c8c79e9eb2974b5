"""Device-side consistency checks (sdf_set_debug_checks): with them on, the
usual executes pass every check and give bitwise the same outputs; a bin
count broken on purpose (SDF_HOOK_CORRUPT_BINS, which keeps every kernel
inside its buffers) is reported as SDF_ERR_INTERNAL naming the check, and the
plan works again once the hook is off."""
import numpy as np
import pytest
import torch

import paper_1112_3010_gb300 as pkg
from paper_1112_3010_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _reset():
    pkg.load_library()
    yield
    pkg.sdf_debug_hook(pkg.SDF_HOOK_CORRUPT_BINS, 0)
    pkg.sdf_set_debug_checks(False)


def _cases():
    rng = np.random.default_rng(81)
    line = wl.Shape(1, (500,), 1 / 500, 2 / 500, rng.uniform(0.3, 0.7, (80, 1)), None)
    return {
        "2d_fp32": (wl.stars(N=256, K=3000, n_shapes=3, tau=0.004, seed=82), "fp32", ("S", "dS", "d2S", "sign")),
        "2d_fp64": (wl.stars(N=200, K=2000, n_shapes=2, tau=0.006, seed=83), "fp64", ("S", "dS", "sign")),
        "3d_fp32": (wl.sphere(N=48, K=3000, radius=0.3, tau=0.03, seed=84), "fp32", ("S", "dS", "d2S", "sign")),
        "1d_fp32": (line, "fp32", ("S", "dS", "d2S")),
    }


def _run(s, prec, outs):
    plan = pkg.Plan(s.D, s.dims, s.h, s.tau, precision=prec, outputs=outs)
    w = torch.from_numpy(s.weights).cuda() if (s.weights is not None and "sign" in outs) else None
    out = plan.execute(torch.from_numpy(s.points).cuda(), w)
    out = {k: v.clone() for k, v in out.items()}
    plan.close()
    return out


@pytest.mark.parametrize("name", list(_cases()))
def test_checks_pass_and_change_nothing(name):
    s, prec, outs = _cases()[name]
    ref = _run(s, prec, outs)
    pkg.sdf_set_debug_checks(True)
    assert pkg.sdf_get_debug_checks()
    got = _run(s, prec, outs)
    for k in ref:
        assert torch.equal(ref[k], got[k]), k


def test_multi_execute_passes_checks():
    s = wl.stars(N=256, K=3000, n_shapes=2, tau=0.004, seed=85)
    pkg.sdf_set_debug_checks(True)
    plans = [pkg.Plan(2, s.dims, s.h, t, precision="fp32", outputs=("S", "dS", "d2S", "sign"))
             for t in (0.004, 0.002)]
    outs = pkg.execute_multi(plans, torch.from_numpy(s.points).cuda(), torch.from_numpy(s.weights).cuda())
    torch.cuda.synchronize()
    assert all(torch.isfinite(o["S"]).all() for o in outs)
    for p in plans:
        p.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_broken_bin_count_is_reported(prec):
    s = wl.stars(N=256, K=3000, n_shapes=3, tau=0.004, seed=86)
    outs = ("S", "dS", "sign")
    ref = _run(s, prec, outs)
    plan = pkg.Plan(2, s.dims, s.h, s.tau, precision=prec, outputs=outs)
    x = torch.from_numpy(s.points).cuda()
    w = torch.from_numpy(s.weights).cuda()
    pkg.sdf_set_debug_checks(True)
    pkg.sdf_debug_hook(pkg.SDF_HOOK_CORRUPT_BINS, 1)
    with pytest.raises(pkg.SDFError) as ei:
        plan.execute(x, w)
    assert ei.value.code == 8   # SDF_ERR_INTERNAL
    assert "check 3" in str(ei.value)   # a bin's unique-node count beyond its points
    pkg.sdf_debug_hook(pkg.SDF_HOOK_CORRUPT_BINS, 0)
    again = plan.execute(x, w)
    for k in ref:
        assert torch.equal(again[k], ref[k]), k
    plan.close()


def test_checks_off_by_default_leave_the_broken_count_unreported():
    s = wl.stars(N=256, K=3000, n_shapes=3, tau=0.004, seed=86)
    pkg.sdf_set_debug_checks(False)
    pkg.sdf_debug_hook(pkg.SDF_HOOK_CORRUPT_BINS, 1)
    plan = pkg.Plan(2, s.dims, s.h, s.tau, precision="fp32", outputs=("S", "sign"))
    out = plan.execute(torch.from_numpy(s.points).cuda(), torch.from_numpy(s.weights).cuda())
    assert torch.isfinite(out["S"]).all()
    plan.close()
