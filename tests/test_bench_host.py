"""Host-side pieces of bench.py that need no GPU: the algorithmic byte counts
of the 2D passes, the clock-record parsing, and the rule that a DRAM traffic
figure is reported only for the kernel source it was captured on."""
import hashlib
import json
import os
from types import SimpleNamespace

import pytest

import bench


def test_algorithmic_bytes_of_the_2048_grid():
    # 2048^2 nodes padded to 4096^2, complex64 lines
    info = SimpleNamespace(dims=(2048, 2048), padded=(4096, 4096))
    field = 4096 * 2048 * 8  # one transformed field after the x-pass: M0 x N1 complex64
    # x-pass: writes the two input fields (counts, packed tangents)
    assert bench.algorithmic_bytes(info, "xpass", None, 2, 4, 8) == 2 * field == 134217728
    # fused: reads the two fields and eight stored real spectra of
    # (M0/2 + 1) x (M1/2 + 1) floats, writes four packed groups
    spectra = 8 * 2049 * 2049 * 4
    assert bench.algorithmic_bytes(info, "fused", None, 2, 4, 8) == 6 * field + spectra == 537002016
    # epilogue: reads the four groups, writes S, grad S (2), Hessian (3) as
    # float and sign, flags as bytes
    assert bench.algorithmic_bytes(info, "epilogue", None, 2, 4, 8) == 4 * field + 2048 * 2048 * 26 == 377487360
    assert bench.algorithmic_bytes(info, "fixup", None, 2, 4, 8) is None


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _clock_record(tmp_path, rows):
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")
    c = bench.Clocks()
    c.proc, c.path = _Proc(), str(path)
    return c


def test_clock_record_median_and_reasons(tmp_path):
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2040, 2070, 1100.5, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "1, 1000, 2070, 100.0, 0x8, Active, Not Active, Not Active, Not Active",  # another GPU
        "garbage line",
    ]
    r = _clock_record(tmp_path, rows).stop(0)
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 3
    assert r["reasons"] == ["sw_power_cap"]


def test_clock_record_flags_thermal_slowdown(tmp_path):
    rows = ["0, 1500, 2070, 1400.0, 0x40, Not Active, Active, Not Active, Not Active"]
    r = _clock_record(tmp_path, rows).stop(0)
    assert r["reasons"] == ["hw_thermal_slowdown"] and r["sm_mhz"] == 1500.0


def test_clock_record_without_nvidia_smi():
    r = bench.Clocks().stop(0)
    assert r["sm_mhz"] is None and r["reasons"] == ["nvidia-smi unavailable"]


@pytest.fixture
def fake_root(tmp_path, monkeypatch):
    src_dir = tmp_path / "paper_1112_3010_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = src_dir / "kern.cu"
    src.write_text("__global__ void k() {}\n")
    rec = {"kern": {"source": "kern.cu", "sha256": hashlib.sha256(src.read_bytes()).hexdigest(),
                    "bytes_per_launch": 1234.0}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return src


def test_traffic_reported_for_the_captured_source(fake_root):
    assert bench.measured_traffic("kern") == 1234.0
    assert bench.measured_traffic("other") is None


def test_traffic_dropped_once_the_source_changes(fake_root):
    fake_root.write_text("__global__ void k() { /* changed */ }\n")
    assert bench.measured_traffic("kern") is None
    os.unlink(fake_root)
    assert bench.measured_traffic("kern") is None


def test_fixup_alu_peak():
    # 152 SMs x 128 FP32 lanes at the clock, over the FMA-pipe operations per term
    ghz = 2.07
    peaks = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks):
        ghz = float(json.load(open(peaks)).get("sm_max_mhz", 2070.0)) / 1000.0
    assert bench.fixup_peak_gterms() == pytest.approx(152 * 128 * ghz / bench.FIXUP_FMA_OPS)


def test_oracle_accuracy_reports_planted_errors():
    """The bench's check of its own outputs against the oracle's sampled
    values: outputs built from the oracle itself, then an S error of 1e-3 tau
    at one uncapped node, a wild value at a capped node (ignored) and a sign
    flip at a node off the boundary band."""
    import numpy as np
    import torch

    import paper_1112_3010_gb300 as pkg
    from paper_1112_3010_gb300 import workloads as wl

    s = wl.stars(N=64, K=400, n_shapes=1, tau=0.02, seed=5)
    samples = []
    bench.cpu_baseline([s], n_nodes=300, seed=3, keep=samples)
    sel, ref = samples[0]
    n = s.n_nodes
    sgn = np.where(np.abs(ref["mu"]) >= 0.5, 1, -1)
    S = np.zeros(n)
    dS = np.zeros((2, n))
    d2S = np.zeros((3, n))
    sign = np.ones(n, np.int8)
    flags = np.zeros(n, np.uint8)
    S[sel] = ref["S"] * sgn
    dS[:, sel] = ref["dS"].T
    d2S[:, sel] = ref["d2S"].T
    sign[sel] = sgn
    band = 2 * ref["wmax"] + s.h * np.sqrt(2.0)
    off = np.nonzero((ref["R"] > band) & (np.abs(np.abs(ref["mu"]) - 0.5) >= 0.05))[0]
    assert len(off) >= 3
    a, b, c = off[0], off[1], off[2]
    S[sel[a]] += 1e-3 * s.tau * sgn[a]          # an S error at an uncapped node
    flags[sel[b]] = pkg.SDF_FLAG_CAPPED          # a capped node with a wild value: not counted
    S[sel[b]] = 1e6
    sign[sel[c]] = -sgn[c]                       # a sign flip off the band
    S[sel[c]] = ref["S"][c] * -sgn[c]            # (S carries the sign)
    outs = [{"S": torch.from_numpy(S.astype(np.float32)), "dS": torch.from_numpy(dS.astype(np.float32)),
             "d2S": torch.from_numpy(d2S.astype(np.float32)), "sign": torch.from_numpy(sign),
             "flags": torch.from_numpy(flags)}]
    rep = bench.oracle_accuracy(pkg, [s], outs, samples)[0]
    assert rep["sampled_nodes"] == len(sel) and rep["uncapped"] == len(sel) - 1
    assert rep["max_abs_S_minus_oracle_over_tau"] == pytest.approx(1e-3, rel=1e-3)
    assert rep["sign_mismatch"] == 1 and rep["sign_checked"] == len(off)
    assert rep["max_abs_dS_minus_oracle"] < 1e-6
