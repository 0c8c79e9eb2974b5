"""Parity of the exact call the headline number measures: bench.py's
C2Problem (one FP32 plan per tau on its own stream, the tile schedule chosen
by sdf_plan_autotune on the workload, both tau through one sdf_execute_multi
forked from and joined to the timing stream), stepped as the timed loop steps
it, then every output checked against the FP64 oracle on sampled nodes at the
parity tolerances (S, grad S, Hessian, sign exact off the boundary band, trust
mask consistent with the oracle's phi)."""
import numpy as np
import pytest
import torch

import bench
import paper_1112_3010_gb300 as pkg

from parity_util import check, oracle_ref, sample_nodes

pytestmark = pytest.mark.gpu


def test_benchmarked_multi_execute_matches_oracle():
    pkg.load_library()
    prob = bench.C2Problem(torch, pkg, tune=True, reps=2)
    try:
        # two steps, as the timed loop runs them back to back
        for _ in range(2):
            with torch.cuda.stream(prob.stream):
                prob.step()
        torch.cuda.synchronize()
        for p in prob.plans:
            p.sync()
        print("tile schedule", prob.tuning)
        for i, (s, o, p) in enumerate(zip(prob.shapes, prob.outs, prob.plans)):
            res = {k: v.cpu().numpy() for k, v in o.items()}
            res["stats"] = p.stats()
            sel = sample_nodes(s, n_uniform=1500, n_near=2500, seed=30 + i)
            ref = oracle_ref(s, sel=sel)
            rep = check(s, res, ref, sel=sel, label="bench-call tau=%g" % s.tau)
            print("bench call", s.tau, rep)
            assert rep["trusted"] > 500 and rep["sign_checked"] > 500
    finally:
        prob.close()
