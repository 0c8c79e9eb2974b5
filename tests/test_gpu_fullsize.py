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
