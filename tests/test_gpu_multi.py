"""sdf_execute_multi: several plans (a sweep of tau, or both kernel sets) on
one point set share the snapping and the tau-independent forward transforms.
Each plan's outputs must equal a separate sdf_execute bit for bit."""
import numpy as np
import pytest
import torch

import paper_1112_3010_gb300 as pkg
from paper_1112_3010_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    pkg.load_library()


def _separate_and_multi(s, taus, prec, outputs, kernels=None):
    kernels = kernels or ["exp"] * len(taus)
    mk = lambda: [pkg.Plan(s.D, s.dims, s.h, t, precision=prec, outputs=outputs, kernel=k)
                  for t, k in zip(taus, kernels)]
    x = torch.from_numpy(s.points).cuda()
    w = torch.from_numpy(s.weights).cuda() if ("sign" in outputs and s.weights is not None) else None
    sep_plans = mk()
    sep = [{k: v.clone() for k, v in p.execute(x, w).items()} for p in sep_plans]
    sep_stats = [p.stats() for p in sep_plans]
    plans = mk()
    outs = pkg.execute_multi(plans, x, w)
    torch.cuda.synchronize()
    for i, (a, b) in enumerate(zip(sep, outs)):
        assert set(a) == set(b)
        for k in a:
            assert torch.equal(a[k], b[k]), (i, k)
        st = plans[i].stats()
        for f in ("n_fixup_nodes", "n_capped", "n_fixup_terms", "n_unique"):
            assert getattr(st, f) == getattr(sep_stats[i], f), (i, f)
        assert st.theta64 == sep_stats[i].theta64
    return plans, outs


def test_2d_fp32_tau_sweep():
    s = wl.stars(N=256, K=3000, n_shapes=3, tau=0.004, seed=31)
    plans, _ = _separate_and_multi(s, [0.004, 0.002, 0.008], "fp32", ("S", "dS", "d2S", "sign"))
    assert plans[1].stats().n_fixup_nodes > 0


def test_2d_fp64_both_kernel_sets():
    s = wl.stars(N=200, K=2000, n_shapes=2, tau=0.006, seed=32)
    _separate_and_multi(s, [0.006, 0.006], "fp64", ("S", "dS", "sign"), kernels=["exp", "green"])


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_3d_two_taus(prec):
    s = wl.sphere(N=40, K=3000, radius=0.3, tau=0.03, seed=33)
    _separate_and_multi(s, [0.03, 0.02], prec, ("S", "dS", "sign"))


def test_single_plan_and_1d():
    s = wl.stars(N=128, K=1000, n_shapes=2, tau=0.01, seed=34)
    _separate_and_multi(s, [0.01], "fp32", ("S", "dS", "sign"))
    rng = np.random.default_rng(35)
    line = wl.Shape(1, (500,), 1 / 500, 2 / 500, rng.uniform(0.3, 0.7, (80, 1)), None)
    _separate_and_multi(line, [2 / 500, 1 / 500], "fp32", ("S", "dS", "d2S"))


def test_mismatched_plans_rejected():
    s = wl.stars(N=128, K=1000, n_shapes=2, tau=0.01, seed=36)
    x = torch.from_numpy(s.points).cuda()
    a = pkg.Plan(2, s.dims, s.h, 0.01, precision="fp32", outputs=("S",))
    b = pkg.Plan(2, (128, 120), s.h, 0.01, precision="fp32", outputs=("S",))
    c = pkg.Plan(2, s.dims, s.h, 0.01, precision="fp64", outputs=("S",))
    for plans in ([a, b], [a, c], [a, a]):
        with pytest.raises(pkg.SDFError) as ei:
            pkg.execute_multi(plans, x)
        assert ei.value.code == 1
    # the plans stay usable
    out = pkg.execute_multi([a], x)[0]
    assert torch.isfinite(out["S"]).all()


@pytest.mark.parametrize("pinned,outputs", [
    ("all", ("S", "dS", "d2S", "sign")),
    ("none", ("S", "dS", "d2S", "sign")),
    ("all", ("S", "sign")),
    ("all", ("S", "dS", "sign")),
    # the first plan's S pageable: its outputs are copied after its fix-up
    ("not_S0", ("S", "dS", "d2S", "sign")),
])
def test_multi_host_matches_device(pinned, outputs):
    """sdf_execute_multi_host: host points and outputs equal to the device
    results, twice in a row.  With the first plan's S, dS and d2S pinned, they
    are copied right after its epilogue and its fix-up writes the nodes it
    recomputes into them directly; otherwise each plan's outputs are copied
    after its fix-up."""
    s = wl.stars(N=256, K=3000, n_shapes=2, tau=0.004, seed=37)
    taus = [0.004, 0.002]
    plans = [pkg.Plan(2, s.dims, s.h, t, precision="fp32", outputs=outputs) for t in taus]
    dev = pkg.execute_multi(plans, torch.from_numpy(s.points).cuda(), torch.from_numpy(s.weights).cuda())
    assert plans[0].stats().n_fixup_nodes > 0
    shp = (s.dims[1], s.dims[0])

    def host(shape, dtype, i, k):
        t = torch.empty(shape, dtype=dtype)
        if pinned == "none" or (pinned == "not_S0" and i == 0 and k == "S"):
            return t
        return t.pin_memory()

    shapes = {"S": (shp, torch.float32), "dS": ((2,) + shp, torch.float32), "d2S": ((3,) + shp, torch.float32),
              "sign": (shp, torch.int8), "flags": (shp, torch.uint8)}
    want = [k for k in shapes if k in outputs or k == "flags"]
    outs = [{k: host(*shapes[k], i, k) for k in want} for i in range(len(taus))]
    col = lambda k: [o[k] for o in outs] if k in want else None
    for rep in range(2):
        for o in outs:
            for v in o.values():
                v.fill_(7)
        pkg.sdf_execute_multi_host([p.handle for p in plans], s.K, torch.from_numpy(s.points),
                                   torch.from_numpy(s.weights), col("S"), col("dS"), col("d2S"), col("sign"),
                                   col("flags"))
        for o, d in zip(outs, dev):
            for k in o:
                assert torch.equal(o[k], d[k].cpu()), (rep, k)


@pytest.mark.parametrize("case", ["2d_single", "3d_pair", "1d_pair", "2d_fp64_pair"])
def test_multi_host_other_shapes(case):
    """sdf_execute_multi_host with one plan (outputs copied after its fix-up),
    3D and FP64 plans, and 1D lines (each plan's outputs copied after its
    execute): the host outputs equal the device ones."""
    rng = np.random.default_rng(39)
    if case == "1d_pair":
        s = wl.Shape(1, (500,), 1 / 500, 2 / 500, rng.uniform(0.3, 0.7, (80, 1)), None)
        taus, outputs, prec = [2 / 500, 1 / 500], ("S", "dS", "d2S"), "fp32"
    elif case == "3d_pair":
        s = wl.sphere(N=40, K=3000, radius=0.3, tau=0.03, seed=33)
        taus, outputs, prec = [0.03, 0.02], ("S", "dS", "d2S", "sign"), "fp32"
    elif case == "2d_fp64_pair":
        s = wl.stars(N=200, K=2000, n_shapes=2, tau=0.006, seed=32)
        taus, outputs, prec = [0.006, 0.004], ("S", "dS", "sign"), "fp64"
    else:
        s = wl.stars(N=256, K=3000, n_shapes=2, tau=0.004, seed=37)
        taus, outputs, prec = [0.004], ("S", "dS", "d2S", "sign"), "fp32"
    plans = [pkg.Plan(s.D, s.dims, s.h, t, precision=prec, outputs=outputs) for t in taus]
    w = torch.from_numpy(s.weights).cuda() if "sign" in outputs else None
    dev = pkg.execute_multi(plans, torch.from_numpy(s.points).cuda(), w)
    torch.cuda.synchronize()
    dt = torch.float64 if prec == "fp64" else torch.float32
    nd, nh = (1, 1) if s.D == 1 else (s.D, s.D * (s.D + 1) // 2)
    shp = tuple(reversed(s.dims))
    shapes = {"S": (shp, dt), "dS": ((nd,) + shp if s.D > 1 else shp, dt),
              "d2S": ((nh,) + shp if s.D > 1 else shp, dt), "sign": (shp, torch.int8), "flags": (shp, torch.uint8)}
    want = [k for k in shapes if k in outputs or k == "flags"]
    outs = [{k: torch.empty(*shapes[k][:1], dtype=shapes[k][1]).pin_memory() for k in want} for _ in taus]
    col = lambda k: [o[k] for o in outs] if k in want else None
    pkg.sdf_execute_multi_host([p.handle for p in plans], s.K, torch.from_numpy(s.points),
                               torch.from_numpy(s.weights) if w is not None else None, col("S"), col("dS"),
                               col("d2S"), col("sign"), col("flags"))
    for o, d in zip(outs, dev):
        for k in o:
            assert torch.equal(o[k], d[k].cpu().reshape(o[k].shape)), k
    for p in plans:
        p.close()


def test_multi_after_pending_work_on_other_streams():
    """Plans on their own streams, with an execute still queued on the second
    plan's stream when the multi-execute starts: the first plan's stream
    waits for it before writing into the second plan's buffers."""
    s = wl.stars(N=256, K=3000, n_shapes=2, tau=0.004, seed=38)
    x = torch.from_numpy(s.points).cuda()
    w = torch.from_numpy(s.weights).cuda()
    outputs = ("S", "dS", "d2S", "sign")
    ref = [{k: v.clone() for k, v in pkg.Plan(2, s.dims, s.h, t, precision="fp32", outputs=outputs)
            .execute(x, w).items()} for t in (0.004, 0.002)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    plans = [pkg.Plan(2, s.dims, s.h, t, precision="fp32", outputs=outputs, stream=st)
             for t, st in zip((0.004, 0.002), streams)]
    for _ in range(3):
        o1 = plans[1].alloc_outputs(["S", "dS", "d2S", "sign", "flags"])
        # queued, not waited for
        pkg.sdf_execute(plans[1].handle, x.shape[0], x, w, o1["S"], o1["dS"], o1["d2S"], o1["sign"], o1["flags"])
        outs = pkg.execute_multi(plans, x, w, check=False)
        torch.cuda.synchronize()
        for a, b in zip(ref, outs):
            for k in a:
                assert torch.equal(a[k], b[k]), k
        for k in ref[1]:
            assert torch.equal(ref[1][k], o1[k]), k


def test_multi_reports_points_off_the_grid():
    s = wl.stars(N=128, K=1000, n_shapes=2, tau=0.01, seed=39)
    bad = torch.from_numpy(np.concatenate([s.points, [[1.5, 0.5]]])).cuda()
    plans = [pkg.Plan(2, s.dims, s.h, t, precision="fp32", outputs=("S", "dS")) for t in (0.01, 0.005)]
    with pytest.raises(pkg.SDFError) as ei:
        pkg.execute_multi(plans, bad)
    assert ei.value.code == 3
    # the plans stay usable
    outs = pkg.execute_multi(plans, torch.from_numpy(s.points).cuda())
    assert all(torch.isfinite(o["S"]).all() for o in outs)
