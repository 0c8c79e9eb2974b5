"""Benchmark: signed S + grad S grid points per second on one GB300.

Workload (the 2D mixed-precision configuration): a 2048^2 grid (h = 1/2048,
padded to 4096^2), K = 40000 points sampled along 8 seeded non-intersecting
star polygons with chord tangents, tau in {0.002, 0.0005}; outputs S (signed),
grad S, Hessian and sign.  One step = every output at both tau values, through
one sdf_execute_multi (the points and the tau-independent transforms once,
each tau's passes on its own stream).  Inputs are resident in HBM before the
timed region; L2 is flushed (256 MiB write) between timed steps, outside the
CUDA-event brackets.

Also reported: the same metric through sdf_execute_multi_host (host buffers,
copies inside the timed region), the plain FP64 GPU path with max|S - S_FP64|
over its trust region beside the library's own error report, the dominant
kernel's roofline from live CUDA events, the FP64 oracle's throughput on the
host cores (bounded sample), SM clocks sampled during the timed region, and
the other configurations under the same clock: the 3D mixed workload (c3), the
96-shape batch (c4), the 3D adjoint (c5), and the 2D workload in full-range
mode (every node from the paper's S, none capped).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "signed S+gradS grid pts/s, mixed-prec vs FP64 GPU path at fixed max|S-S_FP64|"
UNIT = "grid_pts/s"
N_GRID = 2048
K_PTS = 40000
TAUS = (0.002, 0.0005)
WORKLOAD = "2D mixed precision: 2048^2 grid padded to 4096^2, K=40000 on 8 star polygons, tau in {0.002, 0.0005}"


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest of a per-rank number over all ranks: the replicas start
    together (barrier) and the job ends when the slowest one does."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_step, steps, seconds):
    """Whole-job throughput of `world` replicas, each processing
    `units_per_step` units per step for `steps` steps, the job taking
    `seconds` (the max over ranks)."""
    return world * units_per_step * steps / seconds


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons (every 200 ms)."""

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self, dev_index=0):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or f[0] != str(dev_index):
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def workloads():
    from paper_1112_3010_gb300 import workloads as wl
    return [wl.config_c2(tau=t) for t in TAUS]


def cpu_baseline(shapes, n_nodes=12288, seed=0, keep=None):
    """The FP64 oracle (as it stands) on a seeded random sample of nodes of
    each tau's grid: S, grad S, Hessian and mu.  Returns grid pts/s.  With
    `keep` (a list), the sampled node indices and the oracle's values there
    are appended to it, one (sel, values) pair per shape: the full-range leg
    compares its outputs with them."""
    import oracle
    rng = np.random.default_rng(seed)
    total_t, total_n = 0.0, 0
    for s in shapes:
        idx, inside = oracle.snap(s.points, s.h, s.dims)
        Y = idx[inside].astype(np.float64) * s.h
        W = s.weights[inside]
        sel = rng.choice(s.n_nodes, n_nodes // len(shapes), replace=False)
        X = oracle.grid_nodes(s.dims, s.h, sel)
        t0 = time.perf_counter()
        ref = oracle.evaluate(Y, X, s.tau, weights=W, want=("S", "dS", "d2S", "mu", "R"))
        ref["wmax"] = float(np.linalg.norm(W, axis=1).max())
        total_t += time.perf_counter() - t0
        total_n += len(sel)
        if keep is not None:
            keep.append((sel, ref))
    rate = total_n / total_t
    # every node costs the oracle the same (a sum over all points), so a
    # uniform sample gives the full grid's time by proportion
    return {"value": rate, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "%d random nodes per tau of the 2048^2 grid (direct FP64 sum over all K=40000 points), "
                      "S, grad S, Hessian, mu; %.1f s" % (total_n // len(shapes), total_t),
            "extrapolated_full_step_s": sum(s.n_nodes for s in shapes) / rate}


def oracle_accuracy(pkg, shapes, outs, samples):
    """The bench's own outputs (the last timed step) against the oracle
    values of the cpu_baseline leg's sampled nodes: over the nodes the
    library does not cap, max |S - S_oracle| / tau, |grad S - oracle| and
    |Hessian - oracle| * tau; and sign mismatches away from the points
    (farther than 2 max|weight| + h sqrt(2) from every point) where the
    oracle's |mu| is not within 0.05 of 1/2."""
    acc = []
    for s, o, (sel, ref) in zip(shapes, outs, samples):
        fl = o["flags"].cpu().numpy().ravel()[sel]
        ok = (fl & pkg.SDF_FLAG_CAPPED) == 0
        sg = o["sign"].cpu().numpy().ravel()[sel]
        S = o["S"].double().cpu().numpy().ravel()[sel] * sg
        G = o["dS"].double().cpu().numpy().reshape(2, -1)[:, sel].T
        H = o["d2S"].double().cpu().numpy().reshape(3, -1)[:, sel].T
        band = 2 * ref["wmax"] + s.h * np.sqrt(2.0)
        off = (ref["R"] > band) & (np.abs(np.abs(ref["mu"]) - 0.5) >= 0.05)
        osign = np.where(np.abs(ref["mu"]) >= 0.5, 1, -1)
        acc.append({"tau": s.tau, "sampled_nodes": int(len(sel)), "uncapped": int(ok.sum()),
                    "max_abs_S_minus_oracle_over_tau": float(np.abs(S - ref["S"])[ok].max() / s.tau),
                    "max_abs_dS_minus_oracle": float(np.abs(G - ref["dS"])[ok].max()),
                    "max_abs_d2S_minus_oracle_times_tau": float(np.abs(H - ref["d2S"])[ok].max() * s.tau),
                    "sign_checked": int(off.sum()), "sign_mismatch": int((sg[off] != osign[off]).sum())})
    return acc


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores, bounded samples."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    shapes = workloads()
    per_step = max(512, int(os.environ.get("SDF_REF_NODES", "4096")))
    for _ in range(args.warmup):
        cpu_baseline(shapes, n_nodes=256, seed=1)
    t0 = time.perf_counter()
    vals = []
    for k in range(args.steps):
        vals.append(cpu_baseline(shapes, n_nodes=per_step, seed=100 + k))
    el = time.perf_counter() - t0
    v = float(np.mean([x["value"] for x in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_nodes_per_step": per_step,
                                             "l2": "n/a (host)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def algorithmic_bytes(plan_info, name, stats, n_field, n_group, n_kern):
    """Algorithmic DRAM bytes of one launch of each 2D pass (FP32 plan)."""
    N0, N1 = plan_info.dims[0], plan_info.dims[1]
    M0, M1 = plan_info.padded[0], plan_info.padded[1]
    c = 8  # complex float
    if name == "xpass":
        return n_field * M0 * N1 * c
    if name == "fused":
        return (n_field + n_group) * M0 * N1 * c + n_kern * (M0 // 2 + 1) * (M1 // 2 + 1) * 4
    if name == "epilogue":
        return n_group * M0 * N1 * c + N0 * N1 * (4 * (1 + 2 + 3) + 1 + 1)
    return None


# FP32 FMA-pipe operations per node-point term of the fix-up's summing loop
# (2D, S + grad S + Hessian in moment form): r^2, r, the exponent, E, E/r,
# the Hessian factor (3), five running sums (sE, sA, 2 gradient), two
# Hessian moments with their one product (the third comes from the trace
# at the end), and the per-point offsets (4) shared by the thread's two
# nodes.
FIXUP_FMA_OPS = 17


def fixup_peak_gterms(sms=None):
    """FP32-pipe bound on the fix-up's node-point terms per second: the
    device's multiprocessors x 128 FP32 lanes x the maximum SM clock (from
    MEASURED_PEAKS.json, else 2.07 GHz) / FMA-pipe operations per term."""
    lanes, ghz = 128, 2.07
    if sms is None:
        sms = 152
        try:
            import torch
            if torch.cuda.is_available():
                sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        except Exception:
            pass
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        ghz = float(json.load(open(p)).get("sm_max_mhz", 2070.0)) / 1000.0
    return sms * lanes * ghz / FIXUP_FMA_OPS


def measured_traffic(kernel, n_launch_terms=None):
    """DRAM bytes per launch from the committed ncu summary of `kernel`, when
    it was taken on the source that is built now (else None)."""
    import hashlib
    f = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(f):
        return None
    d = json.load(open(f)).get(kernel)
    if not d:
        return None
    src = os.path.join(ROOT, "paper_1112_3010_gb300", "csrc", d["source"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest() != d["sha256"]:
        return None
    return d["bytes_per_launch"]


def fork_join(torch, run, main, streams):
    """run() enqueues on `streams` after everything already on `main`;
    `main` then waits for all of them."""
    fork = torch.cuda.Event()
    fork.record(main)
    for st in streams:
        st.wait_event(fork)
    run()
    for st in streams:
        main.wait_stream(st)


class C2Problem:
    """The benchmarked configuration, set up and stepped exactly as the
    headline number is measured: one FP32 plan per tau, each on its own
    stream, outputs S, grad S, Hessian, sign and flags; the tile schedule
    chosen by sdf_plan_autotune on the workload itself; a step is one
    sdf_execute_multi over both plans (the one point set snapped and
    transformed once), forked from and joined back to `self.stream`."""

    def __init__(self, torch, pkg, tune=True, reps=2, full_range=False, tuning=None):
        self.torch, self.pkg = torch, pkg
        self.shapes = workloads()
        self.stream = torch.cuda.Stream()
        self.pstreams = [torch.cuda.Stream() for _ in self.shapes]
        torch.cuda.synchronize()
        with torch.cuda.stream(self.stream):
            self.plans = [pkg.Plan(2, s.dims, s.h, s.tau, precision="fp32", outputs=("S", "dS", "d2S", "sign"),
                                   stream=ps, full_range=full_range) for s, ps in zip(self.shapes, self.pstreams)]
            self.pts = [torch.from_numpy(s.points).cuda() for s in self.shapes]
            self.wts = [torch.from_numpy(s.weights).cuda() for s in self.shapes]
            self.outs = [p.alloc_outputs(["S", "dS", "d2S", "sign", "flags"]) for p in self.plans]
        torch.cuda.synchronize()
        self.tuning = []
        if tuning is not None:
            for p, t in zip(self.plans, tuning):
                pkg.sdf_plan_set_tuning(p.handle, *t)
            self.tuning = list(tuning)
        elif tune:
            # plan-time work, untimed
            for p, x, w in zip(self.plans, self.pts, self.wts):
                self.tuning.append(pkg.sdf_plan_autotune(p.handle, x.shape[0], x, w, reps))
        self.shared_pts = all(np.array_equal(s.points, self.shapes[0].points) and
                              np.array_equal(s.weights, self.shapes[0].weights) for s in self.shapes)

    def step(self, serial=False):
        pkg, torch = self.pkg, self.torch
        plans, pts, wts, outs = self.plans, self.pts, self.wts, self.outs

        def run():
            if self.shared_pts:
                col = lambda k: [o[k] for o in outs]
                pkg.sdf_execute_multi([p.handle for p in plans], pts[0].shape[0], pts[0], wts[0], col("S"),
                                      col("dS"), col("d2S"), col("sign"), col("flags"))
                return
            for p, x, w, o in zip(plans, pts, wts, outs):
                pkg.sdf_execute(p.handle, x.shape[0], x, w, o["S"], o["dS"], o["d2S"], o["sign"], o["flags"])
        if not serial:
            fork_join(torch, run, self.stream, self.pstreams)
            return
        # one problem at a time (the kernel-timing pass)
        for p, x, w, o, ps in zip(plans, pts, wts, outs, self.pstreams):
            fork_join(torch, lambda: pkg.sdf_execute(p.handle, x.shape[0], x, w, o["S"], o["dS"], o["d2S"],
                                                     o["sign"], o["flags"]), self.stream, [ps])

    def close(self):
        for p in self.plans:
            p.close()


def _timed(torch, stream, flush, steps, fn):
    """Device time of fn() per call (ms, mean over `steps`), CUDA events on
    `stream`, L2 flushed before each call outside the events."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            fn()
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in ev]))


def _dominant(prof_items):
    tot = sum(t for _, (n, t) in prof_items) or 1e-12
    name, (n, t) = max(prof_items, key=lambda kv: kv[1][1])
    return {"kernel": name, "share": t / tot, "avg_ms": t / max(1, n)}


def bench_c3(torch, pkg, flush, steps):
    """3D mixed precision: 256^3 grid padded to 512^3, K = 200000 on a torus
    plus a sphere, tau = 0.004, outputs S, grad S, sign; against the FP64 path."""
    from paper_1112_3010_gb300 import workloads as wl
    s = wl.config_c3()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        pts = torch.from_numpy(s.points).cuda()
        w = torch.from_numpy(s.weights).cuda()
    res = {"workload": "3D mixed: 256^3 grid padded to 512^3, K=200000 on a torus + sphere, tau=0.004, "
                       "outputs S, grad S, sign"}
    outs = {}
    for prec in ("fp32", "fp64"):
        with torch.cuda.stream(st):
            p = pkg.Plan(3, s.dims, s.h, s.tau, precision=prec, outputs=("S", "dS", "sign"), stream=st)
            o = p.alloc_outputs(["S", "dS", "sign", "flags"])
        # the tile schedule chosen by the autotuner for both paths (plan-time
        # work, untimed)
        tuning = pkg.sdf_plan_autotune(p.handle, s.K, pts, w, 2)
        run = lambda: pkg.sdf_execute(p.handle, s.K, pts, w, o["S"], o["dS"], None, o["sign"], o["flags"])
        with torch.cuda.stream(st):
            run()
        p.sync()
        ms = _timed(torch, st, flush, steps if prec == "fp32" else max(2, steps // 2), run)
        p.profile(True)
        p.profile_read()
        _timed(torch, st, flush, 1, run)
        prof = p.profile_read()
        p.profile(False)
        stt = p.stats()
        res[prec] = {"ms_per_execute": ms, "grid_pts_per_s": s.n_nodes / (ms * 1e-3),
                     "tile_schedule": {"lines_T": tuning[0], "lines_F": tuning[1], "fused_variant": tuning[2]},
                     "dominant_kernel": _dominant(list(prof.items())),
                     "err_bound_S_over_tau": stt.err_bound_S / s.tau, "err_bound_dS": stt.err_bound_dS,
                     "trusted_frac": stt.trusted_frac}
        if prec == "fp32":
            res[prec]["fixup_terms"] = stt.n_fixup_terms
            res[prec]["fixup_nodes"] = stt.n_fixup_nodes
        outs[prec] = (o, stt)
        p.close()
    (o32, b32), (o64, b64) = outs["fp32"], outs["fp64"]
    ok = ((o32["flags"] & pkg.SDF_FLAG_CAPPED) == 0) & ((o64["flags"] & pkg.SDF_FLAG_CAPPED) == 0)
    u32 = o32["S"].double() * o32["sign"].double()
    u64 = o64["S"].double() * o64["sign"].double()
    res["max_abs_S_minus_S64_over_tau"] = (u32 - u64)[ok].abs().max().item() / s.tau
    res["bound_S_32_plus_64_over_tau"] = (b32.err_bound_S + b64.err_bound_S) / s.tau
    res["sign_diff_in_trust_region"] = int(((o32["sign"] != o64["sign"]) & ok).sum().item())
    res["speedup_mixed_over_fp64"] = res["fp64"]["ms_per_execute"] / res["fp32"]["ms_per_execute"]
    return res


def bench_c4(torch, pkg, flush, steps):
    """The batch: 96 independent 2D shapes (sides 256-1024, K 500-20000,
    tau = 2h), outputs S and sign, FP32, one graph launch per step."""
    from paper_1112_3010_gb300 import workloads as wl
    shapes = wl.batch_stars(n=96, seed=4)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        b = pkg.Batch(2, [x.dims for x in shapes], [x.h for x in shapes], [x.tau for x in shapes],
                      precision="fp32", outputs=("S", "sign"), n_streams=16, stream=st)
        pts = [torch.from_numpy(x.points).cuda() for x in shapes]
        wts = [torch.from_numpy(x.weights).cuda() for x in shapes]
        outs = b.alloc_outputs()
    torch.cuda.synchronize()

    def timed_batch():
        with torch.cuda.stream(st):
            b.execute(pts, wts, outs)   # plain run + graph capture
            b.execute(pts, wts, outs)
        b.sync()
        ms = _timed(torch, st, flush, steps, lambda: b.execute(pts, wts, outs))
        b.sync()
        padded = [int(pkg.sdf_plan_get_info(pkg.sdf_batch_plan(b.handle, i)).padded[0]) for i in range(len(shapes))]
        return ms, padded

    ms0, padded0 = timed_batch()   # powers of two, built-in tile schedule
    b.autotune(pts, wts, reps=2)   # padded sizes and tile schedules (plan-time work, untimed)
    ms, padded = timed_batch()
    n_pts = sum(x.n_nodes for x in shapes)
    b.close()
    sides = sorted(set(x.dims[0] for x in shapes))
    by_side = lambda pad: {str(sd): sorted(set(m for x, m in zip(shapes, pad) if x.dims[0] == sd)) for sd in sides}
    return {"workload": "96 2D shapes (seed 4): sides uniform over {256,384,512,768,1024}, K 500-20000, "
                        "tau=2h, outputs S, sign; one CUDA-graph launch",
            "ms_per_batch": ms, "grid_pts": n_pts, "grid_pts_per_s": n_pts / (ms * 1e-3),
            "padded_by_side": by_side(padded),
            "untuned": {"ms_per_batch": ms0, "grid_pts_per_s": n_pts / (ms0 * 1e-3),
                        "padded_by_side": by_side(padded0)}}


def bench_c5(torch, pkg, flush, steps):
    """Differentiation: 128^3 grid, K = 20000 jittered sphere points (the
    library snaps them), tau = 0.01, FP32; forward (S, grad S) and the
    adjoint of L = sum w S, with w ~ N(0, 1) on a band of half-width tau
    around the sphere (0 elsewhere)."""
    from paper_1112_3010_gb300 import workloads as wl
    s = wl.config_c5()
    Y = np.ascontiguousarray(s.points)
    n = s.dims[0]
    g = np.arange(n) * s.h - 0.5
    zz, yy, xx = np.meshgrid(g, g, g, indexing="ij")   # x fastest, as the grid arrays
    d = np.abs(np.sqrt(xx * xx + yy * yy + zz * zz).ravel() - 0.3)
    wv = wl.loss_weights(s.n_nodes, seed=50)
    wv[d > s.tau] = 0.0
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        p = pkg.Plan(3, s.dims, s.h, s.tau, precision="fp32", outputs=("S", "dS"), stream=st)
        pts = torch.from_numpy(Y).cuda()
        o = p.alloc_outputs(["S", "dS", "flags"])
        wt = torch.from_numpy(wv).float().cuda().reshape(o["S"].shape)
        dY = torch.empty_like(pts)
        dtau = torch.zeros(1, dtype=torch.float64, device="cuda")
    # the autotuner's tile schedule (plan-time work, untimed)
    tuning = pkg.sdf_plan_autotune(p.handle, pts.shape[0], pts, None, 2)
    fwd = lambda: pkg.sdf_execute(p.handle, pts.shape[0], pts, None, o["S"], o["dS"], None, None, o["flags"])
    bwd = lambda: pkg.sdf_backward(p.handle, pts.shape[0], pts, wt, o["S"], o["flags"], dY, dtau)
    with torch.cuda.stream(st):
        fwd()
        bwd()
    p.sync()
    ms_f = _timed(torch, st, flush, steps, fwd)
    ms_b = _timed(torch, st, flush, steps, bwd)
    p.sync()
    p.close()
    return {"workload": "3D adjoint: 128^3 grid padded to 256^3, K=20000 jittered sphere points (snapped), "
                        "tau=0.01, FP32; dL/dY and dL/dtau of L = sum w S",
            "tile_schedule": {"lines_T": tuning[0], "lines_F": tuning[1], "fused_variant": tuning[2]},
            "forward_ms": ms_f, "backward_ms": ms_b, "grid_pts_per_s_forward_plus_backward":
                s.n_nodes / ((ms_f + ms_b) * 1e-3)}


def bench_full_range(torch, pkg, flush, steps, tuning, samples=None):
    """The 2D workload in full-range mode: every node from the paper's S
    (the fix-up sums whatever the float transform does not trust, nothing is
    capped).  Accuracy against the oracle values the cpu_baseline leg
    computed on its sampled nodes (`samples`, when that leg ran)."""
    prob = C2Problem(torch, pkg, tune=False, full_range=True, tuning=tuning or None)
    with torch.cuda.stream(prob.stream):
        prob.step()
    torch.cuda.synchronize()
    ms = _timed(torch, prob.stream, flush, steps, prob.step)
    stats = [p.stats() for p in prob.plans]
    acc = []
    for i, (s, o, st) in enumerate(zip(prob.shapes, prob.outs, stats)):
        a = {"tau": s.tau, "capped": st.n_capped, "fixup_nodes": st.n_fixup_nodes,
             "fixup_terms": st.n_fixup_terms, "err_bound_S_over_tau": st.err_bound_S / s.tau,
             "err_bound_dS": st.err_bound_dS}
        if samples is not None and i < len(samples):
            sel, ref = samples[i]
            S = (o["S"].double() * o["sign"].double()).cpu().numpy().ravel()[sel]
            G = o["dS"].double().cpu().numpy().reshape(2, -1)[:, sel].T
            a["sampled_nodes"] = int(len(sel))
            a["max_abs_S_minus_oracle_over_tau"] = float(np.abs(S - ref["S"]).max() / s.tau)
            a["max_abs_dS_minus_oracle"] = float(np.abs(G - ref["dS"]).max())
        acc.append(a)
    n_pts = sum(s.n_nodes for s in prob.shapes)
    prob.close()
    return {"ms_per_step": ms, "grid_pts_per_s": n_pts / (ms * 1e-3),
            "sample": "the cpu_baseline leg's random nodes, against its FP64 oracle values", "accuracy": acc}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the c3/c4/c5/full-range legs")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_1112_3010_gb300 as pkg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    pkg.load_library()
    prob = C2Problem(torch, pkg, tune=not args.no_tune)
    stream, pstreams, shapes, plans = prob.stream, prob.pstreams, prob.shapes, prob.plans
    pts, wts, outs, tuning, shared_pts = prob.pts, prob.wts, prob.outs, prob.tuning, prob.shared_pts
    step = prob.step
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    for p in plans:
        p.sync()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    launches = 0
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    for p in plans:
        launches += p.stats().n_launches * args.steps
    if dist:
        dist.barrier()
    time.sleep(0.2)
    clk = clocks.stop(local)
    ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(sum(ms))
    total_ms = max_over_ranks(total_ms, dist, device="cuda")
    pts_per_step = sum(s.n_nodes for s in shapes)
    value = job_throughput(world, pts_per_step, args.steps, total_ms * 1e-3)
    # kernel times: the same steps again, the two problems one after the
    # other so that each kernel's CUDA-event duration is its own (events on
    # the stream each kernel runs on)
    for p in plans:
        p.profile(True)
        p.profile_read()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)
            step(serial=True)
    torch.cuda.synchronize()
    prof = {}
    per_plan = []
    for p in plans:
        pp = p.profile_read()
        per_plan.append(pp)
        for name, (n, t) in pp.items():
            a = prof.setdefault(name, [0, 0.0])
            a[0] += n
            a[1] += t
        p.profile(False)
    stats = [p.stats() for p in plans]

    # roofline of the dominant kernel, and of each FFT pass against HBM
    hbm_peak, peak_kind = load_peaks()
    info = plans[0].info
    n_field, n_group, n_kern = 2, 4, info.n_kernels
    passes = {}
    for name in ("xpass", "fused", "epilogue"):
        if name in prof:
            n, t = prof[name]
            b = algorithmic_bytes(info, name, None, n_field, n_group, n_kern)
            gbs = b / (t / n * 1e-3) / 1e9
            passes[name] = {"bytes_per_launch": b, "avg_ms": t / n, "achieved_GBs": gbs,
                            "frac_of_" + peak_kind + "_hbm": gbs / hbm_peak}
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0] if prof else None
    roof = None
    if dom == "fixup":
        # node-point terms per second against the FP32 pipe: every term costs
        # FIXUP_FMA_OPS issue slots of the 128-lane FMA pipe (and 2 MUFU ops,
        # 16 lanes per SM, which bind later)
        n, t = prof["fixup"]
        terms = sum(st.n_fixup_terms for st in stats)  # all plans, one execute each
        ach = terms / (t / n * len(plans) * 1e-3) / 1e9
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        peak = fixup_peak_gterms(sms)
        roof = {"kernel": "fixup", "bound": "alu", "achieved": ach, "peak": peak, "unit": "Gterm/s",
                "frac": ach / peak, "traffic": measured_traffic("fixup", n_launch_terms=terms / len(plans)),
                "peak_source": "derived: %d SMs x 128 FP32 lanes x max SM clock / %d FMA-pipe ops per term"
                               % (sms, FIXUP_FMA_OPS),
                "avg_launch_ms": t / n}
    elif dom in passes:
        pz = passes[dom]
        roof = {"kernel": dom, "bound": "hbm", "achieved": pz["achieved_GBs"], "peak": hbm_peak, "unit": "GB/s",
                "frac": pz["achieved_GBs"] / hbm_peak, "traffic": measured_traffic(dom),
                "peak_source": peak_kind, "avg_launch_ms": pz["avg_ms"]}
    per_kernel = {k: {"launches": v[0], "avg_ms": v[1] / max(1, v[0]),
                      "share": v[1] / max(1e-9, sum(x[1] for x in prof.values()))} for k, v in prof.items()}

    # end to end through sdf_execute_host (host buffers, copies inside)
    e2e = None
    if not args.no_e2e:
        shp = (N_GRID, N_GRID)
        host_out = [{"S": torch.empty(shp, dtype=torch.float32).pin_memory(),
                     "dS": torch.empty((2,) + shp, dtype=torch.float32).pin_memory(),
                     "d2S": torch.empty((3,) + shp, dtype=torch.float32).pin_memory(),
                     "sign": torch.empty(shp, dtype=torch.int8).pin_memory()} for _ in shapes]
        hp = [torch.from_numpy(s.points).pin_memory() for s in shapes]
        hw = [torch.from_numpy(s.weights).pin_memory() for s in shapes]

        import concurrent.futures as cf
        pool = cf.ThreadPoolExecutor(len(plans))

        def host_step():
            if shared_pts:
                # one call for both tau: the points cross once, outputs come back per tau
                col = lambda k: [o[k] for o in host_out]
                pkg.sdf_execute_multi_host([p.handle for p in plans], hp[0].shape[0], hp[0], hw[0], col("S"),
                                           col("dS"), col("d2S"), col("sign"), None)
                return
            # the public call is synchronous: one host thread per problem
            # (ctypes releases the GIL) so the two run concurrently
            futs = [pool.submit(pkg.sdf_execute_host, p.handle, x.shape[0], x, w, o["S"], o["dS"], o["d2S"],
                                o["sign"], None) for p, x, w, o in zip(plans, hp, hw, host_out)]
            for f in futs:
                f.result()

        for _ in range(2):
            host_step()
        n_e2e = max(3, args.steps // 2)
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            host_step()
        el = max_over_ranks(time.perf_counter() - t0, dist, device="cuda")
        h2d = (2 * shapes[0].K * 2 * 8) if shared_pts else sum(2 * s.K * 2 * 8 for s in shapes)
        d2h = sum(s.n_nodes * (4 * 6 + 1) for s in shapes)
        e2e = {"value": job_throughput(world, pts_per_step, n_e2e, el), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * el / n_e2e}

    # the plain FP64 GPU path on the same workload, and max|S - S_FP64|
    fp64 = None
    if args.fp64_steps > 0:
        with torch.cuda.stream(stream):
            p64 = [pkg.Plan(2, s.dims, s.h, s.tau, precision="fp64", outputs=("S", "dS", "d2S", "sign"),
                            stream=ps) for s, ps in zip(shapes, pstreams)]
            o64 = [p.alloc_outputs(["S", "dS", "d2S", "sign", "flags"]) for p in p64]
        torch.cuda.synchronize()

        def step64():
            def run():
                if shared_pts:  # the same sharing as the mixed path
                    col = lambda k: [o[k] for o in o64]
                    pkg.sdf_execute_multi([p.handle for p in p64], pts[0].shape[0], pts[0], wts[0], col("S"),
                                          col("dS"), col("d2S"), col("sign"), col("flags"))
                    return
                for p, x, w, o in zip(p64, pts, wts, o64):
                    pkg.sdf_execute(p.handle, x.shape[0], x, w, o["S"], o["dS"], o["d2S"], o["sign"], o["flags"])
            fork_join(torch, run, stream, pstreams)

        with torch.cuda.stream(stream):
            step64()
        torch.cuda.synchronize()
        e64 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.fp64_steps)]
        for k in range(args.fp64_steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
                e64[k][0].record(stream)
                step64()
                e64[k][1].record(stream)
        torch.cuda.synchronize()
        ms64 = float(np.mean([a.elapsed_time(b) for a, b in e64]))
        # accuracy of the mixed path against the FP64 path over the FP64 trust region
        acc = []
        for s, o32, o_64, p in zip(shapes, outs, o64, p64):
            st64 = p.stats()
            ok = (o_64["flags"] & pkg.SDF_FLAG_CAPPED) == 0
            S64 = o_64["S"].double()
            S32 = o32["S"].double()
            # exclude nodes within 0.1% of the threshold (either path may decide)
            near = (S64.abs() - st64.s_cap).abs() < s.tau * 1e-3
            m = ok & ~near
            dS = (S32 - S64).abs()[m].max().item() if m.any() else 0.0
            dG = (o32["dS"].double() - o_64["dS"].double()).abs()[:, m].max().item() if m.any() else 0.0
            dH = (o32["d2S"].double() - o_64["d2S"].double()).abs()[:, m].max().item() if m.any() else 0.0
            sgn_mis = int(((o32["sign"] != o_64["sign"]) & m).sum().item())
            st32 = next(st for st, s2 in zip(stats, shapes) if s2 is s)
            acc.append({"tau": s.tau, "max_abs_S_minus_S64_over_tau": dS / s.tau, "max_abs_dS": dG,
                        "max_abs_d2S_times_tau": dH * s.tau, "trusted_frac": m.float().mean().item(),
                        "sign_diff_in_trust_region": sgn_mis,
                        # the library's own error report: |S_32 - S_64| <= bound_32 + bound_64
                        "reported_bound_S_over_tau": (st32.err_bound_S + st64.err_bound_S) / s.tau,
                        "reported_bound_dS": st32.err_bound_dS + st64.err_bound_dS,
                        "reported_bound_d2S_times_tau": (st32.err_bound_d2S + st64.err_bound_d2S) * s.tau})
        fp64 = {"ms_per_step": ms64, "value": pts_per_step / (ms64 * 1e-3), "unit": UNIT,
                "speedup_mixed_over_fp64": (value / world) / (pts_per_step / (ms64 * 1e-3)),
                "accuracy": acc}
        for p in p64:
            p.close()

    cpu = None
    samples = []
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(shapes, keep=samples)
        cpu["accuracy_of_this_run"] = oracle_accuracy(pkg, shapes, outs, samples)

    # the other configurations under the same clock (one GPU, rank 0 alone)
    extra = {}
    if world == 1 and not args.no_extra:
        for p in plans:
            p.sync()
        ext_steps = max(3, min(args.steps, 10))
        extra["full_range"] = bench_full_range(torch, pkg, flush, max(2, ext_steps // 2), tuning, samples or None)
        extra["c3"] = bench_c3(torch, pkg, flush, ext_steps)
        extra["c4"] = bench_c4(torch, pkg, flush, ext_steps)
        extra["c5"] = bench_c5(torch, pkg, flush, ext_steps)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [N_GRID, N_GRID], "padded": [info.padded[0], info.padded[1]],
                       "K": K_PTS, "taus": list(TAUS), "outputs": "S,dS,d2S,sign,flags",
                       "precision": "mixed (fp32 FFT + shifted direct-sum fix-up)",
                       "l2": "flushed between steps (256 MiB write)", "parallelism": "replicas" if world > 1 else "1 GPU",
                       "concurrency": ("one point set at both tau: one sdf_execute_multi per step snaps the "
                                       "points and runs the x-pass once, then each tau's fused pass, epilogue "
                                       "and fix-up on its own stream of one GPU; " if shared_pts else
                                       "the two problems (one per tau) run on two streams of one GPU; ") +
                                      "kernel times and rooflines from a second pass of the same steps "
                                      "run one problem at a time (separate executes)",
                       "tile_schedule": [{"lines_T": a, "lines_F": b, "fused_variant": c} for a, b, c in tuning]},
            "roofline": roof, "cpu_baseline": cpu, "clocks": clk, "e2e": e2e, "gpu_launches": launches,
            "kernels": per_kernel, "fft_passes": passes, "fp64_path": fp64,
            "error_report": [{"tau": s.tau, "err_bound_S_over_tau": st.err_bound_S / s.tau,
                              "err_bound_dS": st.err_bound_dS, "err_bound_d2S_times_tau": st.err_bound_d2S * s.tau,
                              "trusted_frac": st.trusted_frac} for s, st in zip(shapes, stats)],
            "fixup": [{"tau": s.tau, "tiles": st.n_fixup_tiles, "nodes": st.n_fixup_nodes,
                       "capped": st.n_capped, "terms": st.n_fixup_terms, "theta32": st.theta32,
                       "theta64": st.theta64,
                       "ms": pp.get("fixup", (1, 0.0))[1] / max(1, pp.get("fixup", (1, 0.0))[0]),
                       "terms_per_s": st.n_fixup_terms / max(1e-12, 1e-3 * pp.get("fixup", (1, 0.0))[1]
                                                             / max(1, pp.get("fixup", (1, 0.0))[0]))}
                      for s, st, pp in zip(shapes, stats, per_plan)]}
    line.update(extra)
    if rank == 0:
        print(json.dumps(line))
    for p in plans:
        p.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
