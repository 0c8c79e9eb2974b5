"""Parity at full workload sizes, on sampled nodes the oracle computes one by
one.  Samples come from the input geometry only (seeded): uniform random nodes
plus nodes at random distances 0..40 tau from random points, so the near band,
the fix-up band and the capped far field are all represented."""
import numpy as np
import pytest
import torch

import oracle
import paper_1112_3010_gb300 as pkg
from paper_1112_3010_gb300 import workloads as wl

from parity_util import check, oracle_ref, run, sample_nodes

pytestmark = pytest.mark.gpu


def _sample(s, n_uniform=1000, n_near=2000, seed=7):
    return sample_nodes(s, n_uniform=n_uniform, n_near=n_near, seed=seed)


@pytest.mark.parametrize("tau", [0.002, 0.0005])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_stars_2048(tau, prec):
    s = wl.config_c2(tau=tau)
    res = run(s, prec, outputs=("S", "dS", "d2S", "sign"))
    sel = _sample(s)
    ref = oracle_ref(s, sel=sel)
    rep = check(s, res, ref, sel=sel, label="c2-%s-%g" % (prec, tau))
    print("c2", prec, tau, rep)
    assert rep["trusted"] > 500


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_torus_sphere_256(prec):
    s = wl.config_c3()
    res = run(s, prec, outputs=("S", "dS", "sign"))
    sel = _sample(s, n_uniform=600, n_near=1400)
    ref = oracle_ref(s, sel=sel, want=("S", "dS", "mu", "R"))
    rep = check(s, res, ref, sel=sel, check_hess=False, label="c3-" + prec)
    print("c3", prec, rep)
    assert rep["trusted"] > 300


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_torus_sphere_256_autotuned(prec, tmp_path, monkeypatch):
    """The 3D workload with the tile schedule the autotuner picks (as the
    bench runs it), sampled nodes against the oracle."""
    monkeypatch.setenv("SDF_AUTOTUNE_CACHE", str(tmp_path / "autotune.tsv"))
    s = wl.config_c3()
    plan = pkg.Plan(3, s.dims, s.h, s.tau, precision=prec, outputs=("S", "dS", "sign"))
    pts = torch.from_numpy(s.points).cuda()
    w = torch.from_numpy(s.weights).cuda()
    tune = pkg.sdf_plan_autotune(plan.handle, s.K, pts, w, 2)
    out = plan.execute(pts, w)
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["stats"] = plan.stats()
    sel = _sample(s, n_uniform=600, n_near=1400, seed=11)
    ref = oracle_ref(s, sel=sel, want=("S", "dS", "mu", "R"))
    rep = check(s, res, ref, sel=sel, check_hess=False, label="c3-tuned-" + prec)
    print("c3 tuned", prec, tune, rep)
    assert rep["trusted"] > 300
    plan.close()

