"""The epilogue's two ways of reading its transposed input
(sdf_plan_set_epilogue_loads): TMA tensor copies staged in shared memory
(mode 0, used where the plan qualifies) and per-thread loads (mode 1).  The
transforms see the same numbers either way, so every output must agree bit
for bit; the staged plans are also checked against the oracle."""
import numpy as np
import pytest
import torch

import paper_1112_3010_gb300 as pkg
from paper_1112_3010_gb300 import workloads as wl

from parity_util import check, oracle_ref, sample_nodes

pytestmark = pytest.mark.gpu

CASES = {
    "stars2048": (lambda: wl.config_c2(tau=0.002), ("S", "dS", "d2S", "sign"), None),
    "stars256": (lambda: wl.stars(N=256, K=3000, n_shapes=3, tau=0.004, seed=61), ("S", "dS", "d2S", "sign"), None),
    "stars384_M768": (lambda: wl.stars(N=384, K=6000, n_shapes=1, tau=2.0 / 384, seed=63, r_lo=0.15, r_hi=0.4,
                                       center=(0.5, 0.5)), ("S", "dS", "sign"), (768, 768)),
    "sphere64": (lambda: wl.sphere(N=64, K=4000, radius=0.3, tau=0.02, seed=71), ("S", "dS", "sign"), None),
    # 3D at a compiled line length (256): the TMA epilogue applies
    "sphere128": (lambda: wl.sphere(N=128, K=12000, radius=0.3, tau=0.01, seed=73), ("S", "dS", "d2S", "sign"),
                  None),
}


def _run(s, outs, mode, padded):
    plan = pkg.Plan(s.D, s.dims, s.h, s.tau, precision="fp32", outputs=outs)
    if padded:
        plan.set_padding(padded)
    pkg.sdf_plan_set_epilogue_loads(plan.handle, mode)
    out = plan.execute(torch.from_numpy(s.points).cuda(), torch.from_numpy(s.weights).cuda())
    st = plan.stats()
    plan.close()
    return out, st


@pytest.mark.parametrize("name", list(CASES))
def test_tma_and_plain_loads_agree_bitwise(name):
    make, outs, padded = CASES[name]
    s = make()
    a, sa = _run(s, outs, 0, padded)
    b, sb = _run(s, outs, 1, padded)
    for k in a:
        assert torch.equal(a[k], b[k]), (name, k)
    assert sa.n_capped == sb.n_capped and sa.n_fixup_nodes == sb.n_fixup_nodes
    res = {k: v.cpu().numpy() for k, v in a.items()}
    res["stats"] = sa
    sel = None if s.n_nodes <= 70000 else sample_nodes(s, n_uniform=1000, n_near=1500, seed=72)
    ref = oracle_ref(s, sel=sel, want=("S", "dS", "d2S", "mu", "R") if "d2S" in outs else ("S", "dS", "mu", "R"))
    check(s, res, ref, sel=sel, check_hess="d2S" in outs, label="tma-" + name)


def test_epilogue_loads_rejects_unknown_mode():
    plan = pkg.Plan(2, (64, 64), 1 / 64, 0.02, precision="fp32", outputs=("S",))
    with pytest.raises(pkg.SDFError):
        pkg.sdf_plan_set_epilogue_loads(plan.handle, 2)
    plan.close()
