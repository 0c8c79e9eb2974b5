"""Batched execution (one graph launch for many problems of uneven size)
against per-problem plans: identical outputs, replay, and re-capture when the
arguments change."""
import numpy as np
import pytest
import torch

import paper_1112_3010_gb300 as pkg
from paper_1112_3010_gb300 import workloads as wl

from parity_util import check, oracle_ref

pytestmark = pytest.mark.gpu


def _shapes():
    return wl.batch_stars(n=7, seed=41, sides=(48, 64, 100), k_lo=200, k_hi=2500)


def _single(s):
    plan = pkg.Plan(2, s.dims, s.h, s.tau, precision="fp32", outputs=("S", "sign"))
    out = plan.execute(torch.from_numpy(s.points).cuda(), torch.from_numpy(s.weights).cuda())
    plan.close()
    return out


def test_batch_matches_single_plans_and_replays():
    shapes = _shapes()
    b = pkg.Batch(2, [s.dims for s in shapes], [s.h for s in shapes], [s.tau for s in shapes],
                  precision="fp32", outputs=("S", "sign"), n_streams=3)
    pts = [torch.from_numpy(s.points).cuda() for s in shapes]
    wts = [torch.from_numpy(s.weights).cuda() for s in shapes]
    outs = b.alloc_outputs()
    for rep in range(3):
        for o in outs:
            o["S"].fill_(-7.0)
        b.execute(pts, wts, outs)
        b.sync()
        for s, o in zip(shapes, outs):
            ref = _single(s)
            for k in ("S", "sign", "flags"):
                assert torch.equal(o[k], ref[k]), (rep, s.dims, k)
    # changed point counts: the batch re-captures
    pts2 = [p[: max(10, p.shape[0] // 2)].contiguous() for p in pts]
    wts2 = [w[: p.shape[0]].contiguous() for w, p in zip(wts, pts2)]
    b.execute(pts2, wts2, outs)
    b.sync()
    for s, o, p, w in zip(shapes, outs, pts2, wts2):
        s2 = wl.Shape(2, s.dims, s.h, s.tau, p.cpu().numpy(), w.cpu().numpy())
        ref = _single(s2)
        assert torch.equal(o["S"], ref["S"])
    b.close()


def test_batch_parity_with_oracle():
    shapes = _shapes()[:3]
    b = pkg.Batch(2, [s.dims for s in shapes], [s.h for s in shapes], [s.tau for s in shapes],
                  precision="fp32", outputs=("S", "sign"), n_streams=2)
    outs = b.alloc_outputs()
    b.execute([torch.from_numpy(s.points).cuda() for s in shapes],
              [torch.from_numpy(s.weights).cuda() for s in shapes], outs)
    b.sync()
    for i, (s, o) in enumerate(zip(shapes, outs)):
        res = {k: v.cpu().numpy() for k, v in o.items()}
        res["stats"] = pkg.sdf_get_stats(pkg.sdf_batch_plan(b.handle, i))
        ref = oracle_ref(s, want=("S", "mu", "R"))
        check(s, res, ref, check_hess=False, label="batch%d" % i)
    b.close()
