"""Padded sizes of 3 * 2^k (sdf_plan_set_padding), the radix-3 transform
stage behind them, and the autotuner's choice of padded size with its cache.

A padded size M >= 2N - 1 keeps the circular convolution equal to the linear
one on the N^D nodes, so the result is the paper's S whatever M is: every
case is checked against the FP64 oracle at the parity tolerances, and against
the same plan at its power-of-two padding."""
import os

import numpy as np
import pytest
import torch

import paper_1112_3010_gb300 as pkg
from paper_1112_3010_gb300 import workloads as wl

from parity_util import check, oracle_ref, sample_nodes

pytestmark = pytest.mark.gpu


def _run(s, prec, outs, padded=None):
    plan = pkg.Plan(s.D, s.dims, s.h, s.tau, precision=prec, outputs=outs)
    if padded is not None:
        plan.set_padding(padded)
    w = torch.from_numpy(s.weights).cuda() if s.weights is not None else None
    out = plan.execute(torch.from_numpy(s.points).cuda(), w)
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["stats"] = plan.stats()
    res["padded"] = tuple(plan.info.padded[: s.D])
    plan.close()
    return res


CASES = {
    # name: (workload, padded size per axis (3 * 2^k), outputs)
    "stars24_M48": (lambda: wl.stars(N=24, K=300, n_shapes=1, tau=0.06, seed=61, r_lo=0.2, r_hi=0.35,
                                     center=(0.5, 0.5)), 48, ("S", "dS", "d2S", "sign")),
    "stars96_M192": (lambda: wl.stars(N=96, K=1500, n_shapes=2, tau=0.02, seed=62), 192,
                     ("S", "dS", "d2S", "sign")),
    "stars384_M768": (lambda: wl.stars(N=384, K=6000, n_shapes=1, tau=2.0 / 384, seed=63, r_lo=0.15, r_hi=0.4,
                                       center=(0.5, 0.5)), 768, ("S", "dS", "d2S", "sign")),
    "sphere24_M48": (lambda: wl.sphere(N=24, K=1200, radius=0.3, tau=0.06, seed=64), 48, ("S", "dS", "sign")),
}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", list(CASES))
def test_radix3_padding_matches_oracle(name, prec):
    make, M, outs = CASES[name]
    s = make()
    res = _run(s, prec, outs, padded=(M,) * s.D)
    assert res["padded"] == (M,) * s.D
    sel = None if s.n_nodes <= 20000 else sample_nodes(s, n_uniform=1500, n_near=2500, seed=65)
    ref = oracle_ref(s, sel=sel, want=("S", "dS", "d2S", "mu", "R") if "d2S" in outs else ("S", "dS", "mu", "R"))
    rep = check(s, res, ref, sel=sel, check_hess="d2S" in outs, label="%s-%s" % (name, prec))
    print(name, prec, rep)
    assert rep["trusted"] > 50
    # the power-of-two padding of the same plan agrees to the tolerance where both trust the node
    pw = _run(s, prec, outs)
    assert max(pw["padded"]) > M
    ok = ((res["flags"] & pkg.SDF_FLAG_CAPPED) == 0) & ((pw["flags"] & pkg.SDF_FLAG_CAPPED) == 0)
    dS = np.abs(res["S"].astype(np.float64) - pw["S"].astype(np.float64))[ok].max()
    assert dS <= 2e-3 * s.tau


def test_radix3_1536_line_against_oracle():
    """A 768-node side padded to 1536 (3 * 2^9: radix 3, two radix-16 stages,
    a radix-2 stage), the size the batch's 768 shapes take."""
    s = wl.stars(N=768, K=12000, n_shapes=1, tau=2.0 / 768, seed=66, r_lo=0.15, r_hi=0.4, center=(0.5, 0.5))
    for prec in ("fp32", "fp64"):
        res = _run(s, prec, ("S", "dS", "sign"), padded=(1536, 1536))
        sel = sample_nodes(s, n_uniform=1500, n_near=2500, seed=67, reach=20.0)
        ref = oracle_ref(s, sel=sel, want=("S", "dS", "mu", "R"))
        rep = check(s, res, ref, sel=sel, check_hess=False, label="768-M1536-" + prec)
        print("768 at 1536", prec, rep)
        assert rep["trusted"] > 500


def test_mixed_padding_per_axis():
    """Axes padded differently (3 * 2^k along x, a power of two along y)."""
    s = wl.stars(N=96, K=1500, n_shapes=2, tau=0.02, seed=62)
    res = _run(s, "fp32", ("S", "dS", "sign"), padded=(192, 256))
    ref = oracle_ref(s, want=("S", "dS", "mu", "R"))
    check(s, res, ref, check_hess=False, label="mixed-padding")


def test_set_padding_rejects_bad_sizes():
    s = wl.stars(N=96, K=500, n_shapes=1, tau=0.02, seed=68)
    plan = pkg.Plan(2, s.dims, s.h, s.tau, precision="fp32", outputs=("S",))
    for bad in [(160, 192), (190, 192), (192, 96 * 2 - 2), (5 * 64, 192), (24576, 192)]:
        with pytest.raises(pkg.SDFError) as ei:
            plan.set_padding(bad)
        assert ei.value.code == 1
    assert tuple(plan.info.padded[:2]) == (256, 256)   # unchanged
    plan.close()
    p1 = pkg.Plan(1, (64,), 1 / 64, 0.05, precision="fp32", outputs=("S",))
    with pytest.raises(pkg.SDFError) as ei:
        p1.set_padding((192,))
    assert ei.value.code == 2
    p1.close()


def test_autotune_chooses_padding_and_caches_it(tmp_path, monkeypatch):
    cache = tmp_path / "autotune.tsv"
    monkeypatch.setenv("SDF_AUTOTUNE_CACHE", str(cache))
    s = wl.stars(N=384, K=6000, n_shapes=1, tau=2.0 / 384, seed=63, r_lo=0.15, r_hi=0.4, center=(0.5, 0.5))
    pts = torch.from_numpy(s.points).cuda()
    w = torch.from_numpy(s.weights).cuda()
    plan = pkg.Plan(2, s.dims, s.h, s.tau, precision="fp32", outputs=("S", "dS", "sign"))
    tune = pkg.sdf_plan_autotune(plan.handle, s.K, pts, w, 2)
    M = tuple(plan.info.padded[:2])
    assert all(m in (768, 1024) for m in M)
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and "|D2|384x384x1|fp32|" in lines[0]
    assert lines[0].split("\t")[1].split()[:2] == [str(m) for m in M]
    print("autotune 384:", M, tune)
    # the tuned plan is still the paper's S
    out = plan.execute(pts, w)
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["stats"] = plan.stats()
    sel = sample_nodes(s, n_uniform=800, n_near=1200, seed=69)
    check(s, res, oracle_ref(s, sel=sel, want=("S", "dS", "mu", "R")), sel=sel, check_hess=False,
          label="autotuned-384")
    plan.close()
    # a second plan of the same problem takes the cached choice, no new entry
    plan2 = pkg.Plan(2, s.dims, s.h, s.tau, precision="fp32", outputs=("S", "dS", "sign"))
    assert pkg.sdf_plan_autotune(plan2.handle, s.K, pts, w, 2) == tune
    assert tuple(plan2.info.padded[:2]) == M
    assert len(cache.read_text().splitlines()) == 1
    plan2.close()
