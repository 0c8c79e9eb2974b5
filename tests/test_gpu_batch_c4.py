"""The batch at its full size: the 96 seeded shapes of the batched
configuration (sides uniform over {256, 384, 512, 768, 1024}, K from 500 to
20000 points on one star polygon each, tau = 2h), FP32, outputs S and sign,
one graph launch -- the launch bench.py times.  Every shape is checked
against the FP64 oracle on sampled nodes (uniform plus near-band), at the
parity tolerances, after a replay of the captured graph."""
import numpy as np
import pytest
import torch

import paper_1112_3010_gb300 as pkg
from paper_1112_3010_gb300 import workloads as wl

from parity_util import check, oracle_ref, sample_nodes

pytestmark = pytest.mark.gpu


def _execute(b, pts, wts, outs):
    for _ in range(2):   # the plain run and capture, then a graph replay
        for o in outs:
            o["S"].fill_(-7.0)
        b.execute(pts, wts, outs)
        b.sync()


def test_batch_96_shapes_full_size_against_oracle():
    """The default padding (powers of two), then the padded sizes and tile
    schedules sdf_batch_autotune chooses (3 * 2^k where that times faster):
    both against the oracle on the same sampled nodes."""
    shapes = wl.batch_stars(n=96, seed=4)
    sides = sorted(set(s.dims[0] for s in shapes))
    assert sides == [256, 384, 512, 768, 1024]
    b = pkg.Batch(2, [s.dims for s in shapes], [s.h for s in shapes], [s.tau for s in shapes],
                  precision="fp32", outputs=("S", "sign"), n_streams=16)
    pts = [torch.from_numpy(s.points).cuda() for s in shapes]
    wts = [torch.from_numpy(s.weights).cuda() for s in shapes]
    outs = b.alloc_outputs()
    refs = []
    for i, s in enumerate(shapes):
        sel = sample_nodes(s, n_uniform=150, n_near=250, seed=100 + i, reach=20.0)
        refs.append((sel, oracle_ref(s, sel=sel, want=("S", "mu", "R"))))
    for stage in ("default", "autotuned"):
        if stage == "autotuned":
            b.autotune(pts, wts, reps=2)
        _execute(b, pts, wts, outs)
        worst, padded = {}, {}
        for i, (s, o) in enumerate(zip(shapes, outs)):
            res = {k: v.cpu().numpy() for k, v in o.items()}
            plan = pkg.sdf_batch_plan(b.handle, i)
            res["stats"] = pkg.sdf_get_stats(plan)
            padded.setdefault(s.dims[0], set()).add(pkg.sdf_plan_get_info(plan).padded[0])
            sel, ref = refs[i]
            rep = check(s, res, ref, sel=sel, check_hess=False,
                        label="c4 %s shape %d (N=%d)" % (stage, i, s.dims[0]))
            w = worst.setdefault(s.dims[0], [0, 0.0])
            w[0] += 1
            w[1] = max(w[1], rep["max_dS"] / s.tau)
        print("c4", stage, "padded per side", {k: sorted(v) for k, v in padded.items()},
              "shapes and worst |S - S_oracle|/tau per side:", worst)
        for side, ms in padded.items():
            assert len(ms) == 1   # every shape of a side takes its owner's sizes
    b.close()
