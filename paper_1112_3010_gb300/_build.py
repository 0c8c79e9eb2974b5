"""Build the CUDA library in-tree: one nvcc call per translation unit, run in
parallel, then one link into ``_lib/libsdf_gb300.so`` (sm_103a only)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libsdf_gb300.so")
SOURCES = ["passes_fused_f2.cu", "passes_fused_f3.cu", "passes_inv.cu", "passes_fwd.cu", "passes_fused_d.cu",
           "passes_fused.cu", "api.cu", "points.cu", "spectra.cu", "fixup.cu", "adjoint.cu", "noalloc.cu", "batch.cu",
           "curvature.cu", "mesh.cu", "line1d.cu", "debugcheck.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags(verbose=False):
    f = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", os.path.join(HERE, "..", "include")] + ARCH
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _stale(objs, srcs):
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "sdf.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    os.makedirs(OUT, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    objs = [os.path.join(OUT, os.path.splitext(s)[0] + ".o") for s in SOURCES]
    if not force and not _stale(objs, srcs):
        return LIB
    cc = nvcc()

    def one(i):
        cmd = [cc, "-c", srcs[i], "-o", objs[i]] + _flags(verbose)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (srcs[i], r.stdout, r.stderr))
        return r.stdout + r.stderr

    logs = []
    with cf.ThreadPoolExecutor(max_workers=jobs or len(srcs)) as ex:
        for out in ex.map(one, range(len(srcs))):
            logs.append(out)
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = [cc, "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fPIC", "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    if verbose:
        print("\n".join(logs))
    return LIB


if __name__ == "__main__":
    import sys
    build(force=True, verbose="-v" in sys.argv)
    print(LIB)
