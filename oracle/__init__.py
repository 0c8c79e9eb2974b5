"""FP64 CPU oracle for the convolution-based signed distance method.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The
product path (``paper_1112_3010_gb300``) never imports this package.

The arithmetic lives in ``sdf_oracle.c`` (plain C, OpenMP over evaluation
points); this module only compiles it with gcc and marshals numpy arrays.
Every quantity is the paper's definition summed directly over the points:

* :func:`snap` -- nearest-node rounding (Sec. 6, Examples 3-4).
* :func:`evaluate` -- S (eq. STilde), grad S (eq. SxSy), Hessian (eqs. Sxx,
  Syy, Sxy; the same differentiation in 3D), winding number (eq.
  kappdiscreteZ) or topological degree (eq. normflux), and R (eq. Rdef).
* :func:`adjoint` -- dL/dY_k and dL/dtau of L = sum_X w(X) S(X), the chain
  rule applied to eq. STilde.
* :func:`curvature` -- Gaussian, mean and principal curvatures from grad S
  and the Hessian (Sec. 5): of the graph z = S(x, y) in 2D, of the level
  surfaces of S in 3D.
* :func:`mesh_sources` -- triangle incentres and area-weighted normals as the
  3D degree's sources (Sec. 4.2, Example 5); :func:`solid_angle_degree` --
  the exact degree of a closed triangle mesh (a textbook check).
* :func:`sign_from_mu` -- inside/outside from mu: inside iff |mu| >= 1/2
  (the nonzero-winding rule of Sec. 4.1), positive inside (Sec. 1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sdf_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libsdf_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (-O2, OpenMP, strict FP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d = ctypes.POINTER(ctypes.c_double)
            i64 = ctypes.c_int64
            lib.oracle_snap.argtypes = [ctypes.c_int, i64, d, ctypes.c_double,
                                        ctypes.POINTER(i64), ctypes.POINTER(i64)]
            lib.oracle_snap.restype = i64
            lib.oracle_eval.argtypes = [ctypes.c_int, i64, d, d, i64, d,
                                        ctypes.c_double, d, d, d, d, d, d]
            lib.oracle_eval.restype = None
            lib.oracle_adjoint.argtypes = [ctypes.c_int, i64, d, i64, d, d,
                                           ctypes.c_double, d, d]
            lib.oracle_adjoint.restype = None
            lib.oracle_curvature.argtypes = [ctypes.c_int, i64, d, d, d]
            lib.oracle_curvature.restype = None
            lib.oracle_mesh_sources.argtypes = [i64, d, ctypes.POINTER(i64), d, d, d]
            lib.oracle_mesh_sources.restype = None
            lib.oracle_solid_angle_degree.argtypes = [i64, d, ctypes.POINTER(i64), i64, d, d]
            lib.oracle_solid_angle_degree.restype = None
            lib.oracle_num_threads.argtypes = []
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def _dp(a):
    if a is None:
        return ctypes.POINTER(ctypes.c_double)()
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def snap(points, h, dims):
    """Nearest-node indices floor(y/h + 0.5) per axis, and an in-grid mask."""
    pts = _c64(points)
    K, D = pts.shape
    dims = np.ascontiguousarray(dims, dtype=np.int64)
    idx = np.empty((K, D), dtype=np.int64)
    _load().oracle_snap(D, K, _dp(pts), float(h),
                        dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                        idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    inside = np.all((idx >= 0) & (idx < dims[None, :]), axis=1)
    return idx, inside


def evaluate(points, X, tau, weights=None, want=("S", "dS", "d2S", "mu", "R")):
    """Direct FP64 sums at real evaluation points X (nX x D).

    Returns a dict with the requested keys among S, dS (nX x D), d2S
    (nX x D(D+1)/2, order xx,yy[,zz],xy[,xz,yz]), mu, R, logphi.
    """
    Y = _c64(points)
    K, D = Y.shape
    Xa = _c64(X).reshape(-1, D)
    nX = Xa.shape[0]
    W = None if weights is None else _c64(weights, (K, D))
    nH = D * (D + 1) // 2
    out = {}
    S = np.empty(nX) if "S" in want else None
    dS = np.empty((nX, D)) if "dS" in want else None
    d2S = np.empty((nX, nH)) if "d2S" in want else None
    mu = np.empty(nX) if ("mu" in want and W is not None) else None
    R = np.empty(nX) if "R" in want else None
    lp = np.empty(nX) if "logphi" in want else None
    _load().oracle_eval(D, K, _dp(Y), _dp(W), nX, _dp(Xa), float(tau),
                        _dp(S), _dp(dS), _dp(d2S), _dp(mu), _dp(R), _dp(lp))
    for k, v in (("S", S), ("dS", dS), ("d2S", d2S), ("mu", mu), ("R", R),
                 ("logphi", lp)):
        if v is not None:
            out[k] = v
    return out


def adjoint(points, X, wX, tau):
    """dL/dY (K x D) and dL/dtau for L = sum_X wX * S(X) at continuous Y."""
    Y = _c64(points)
    K, D = Y.shape
    Xa = _c64(X).reshape(-1, D)
    w = _c64(wX).reshape(-1)
    assert w.shape[0] == Xa.shape[0]
    dY = np.empty((K, D))
    dt = np.zeros(1)
    _load().oracle_adjoint(D, K, _dp(Y), Xa.shape[0], _dp(Xa), _dp(w),
                           float(tau), _dp(dY), _dp(dt))
    return dY, float(dt[0])


def curvature(dS, d2S):
    """Curvatures (n x 4: K, H, k1, k2) from grad S (n x D) and the Hessian
    (n x D(D+1)/2): the graph z = S(x, y) in 2D, level surfaces in 3D."""
    g = _c64(dS)
    D = g.shape[1]
    h = _c64(d2S, (g.shape[0], D * (D + 1) // 2))
    out = np.empty((g.shape[0], 4))
    _load().oracle_curvature(D, g.shape[0], _dp(g), _dp(h), _dp(out))
    return out


def _i64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def mesh_sources(V, F, center=None):
    """Incentres Y (nf x 3) and area-weighted normals P (nf x 3) of a triangle
    mesh; ``center`` (3,) applies the Example 5 orientation rule."""
    Va = _c64(V).reshape(-1, 3)
    Fa = np.ascontiguousarray(F, dtype=np.int64).reshape(-1, 3)
    Y = np.empty((Fa.shape[0], 3))
    P = np.empty((Fa.shape[0], 3))
    c = None if center is None else _c64(center).reshape(3)
    _load().oracle_mesh_sources(Fa.shape[0], _dp(Va), _i64p(Fa), _dp(c), _dp(Y), _dp(P))
    return Y, P


def solid_angle_degree(V, F, X):
    """Exact degree (solid angle / 4 pi) of a closed triangle mesh at X (n x 3)."""
    Va = _c64(V).reshape(-1, 3)
    Fa = np.ascontiguousarray(F, dtype=np.int64).reshape(-1, 3)
    Xa = _c64(X).reshape(-1, 3)
    out = np.empty(Xa.shape[0])
    _load().oracle_solid_angle_degree(Fa.shape[0], _dp(Va), _i64p(Fa), Xa.shape[0], _dp(Xa), _dp(out))
    return out


def sign_from_mu(mu):
    """+1 inside (|mu| >= 1/2), -1 outside (Sec. 4.1 nonzero winding rule)."""
    return np.where(np.abs(np.asarray(mu)) >= 0.5, 1, -1).astype(np.int8)


def grid_nodes(dims, h, sel=None):
    """World coordinates of grid nodes i*h (x fastest).  ``sel`` is an optional
    array of flat node indices; returns (len(sel) or prod(dims)) x D."""
    dims = [int(n) for n in dims]
    D = len(dims)
    total = int(np.prod(dims))
    flat = np.arange(total, dtype=np.int64) if sel is None else np.asarray(sel, np.int64)
    coords = np.empty((flat.shape[0], D))
    rem = flat.copy()
    for a in range(D):
        coords[:, a] = (rem % dims[a]) * h
        rem //= dims[a]
    return coords


def snapped_points(points, h, dims):
    """Snapped world coordinates j*h of the in-grid points (with multiplicity)."""
    idx, inside = snap(points, h, dims)
    return idx[inside].astype(np.float64) * h, inside
