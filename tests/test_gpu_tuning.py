"""Tile schedules (sdf_plan_set_tuning): every variant of the transposed and
fused passes meets the oracle parity bar on the same inputs -- including the
one the autotuner picks for the bench workload."""
import numpy as np
import pytest
import torch

import paper_1112_3010_gb300 as pkg
from paper_1112_3010_gb300 import workloads as wl

from parity_util import check, oracle_ref

pytestmark = pytest.mark.gpu

# (lines_T, lines_F, fused_variant)
SCHEDULES = [(0, 0, 0), (1, 0, 1), (2, 1, 2), (4, 0, 2), (16, 0, 2), (8, 2, 3), (4, 0, 3), (2, 4, 1)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    pkg.load_library()


def _run(s, prec, sched, outputs):
    plan = pkg.Plan(s.D, s.dims, s.h, s.tau, precision=prec, outputs=outputs)
    pkg.sdf_plan_set_tuning(plan.handle, *sched)
    out = plan.execute(torch.from_numpy(s.points).cuda(), torch.from_numpy(s.weights).cuda())
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["stats"] = plan.stats()
    return res


def test_2d_schedules_fp32():
    s = wl.stars(N=256, K=3000, n_shapes=3, tau=0.004, seed=61)
    ref = oracle_ref(s)
    for sched in SCHEDULES:
        res = _run(s, "fp32", sched, ("S", "dS", "d2S", "sign"))
        check(s, res, ref, label="2d-%s" % (sched,))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_3d_schedules(prec):
    s = wl.sphere(N=40, K=3000, radius=0.3, tau=0.03, seed=62)
    ref = oracle_ref(s, want=("S", "dS", "mu", "R"))
    for sched in SCHEDULES[:5]:
        res = _run(s, prec, sched, ("S", "dS", "sign"))
        check(s, res, ref, check_hess=False, label="3d-%s-%s" % (prec, sched))
