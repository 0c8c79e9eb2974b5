"""GB300 (sm_103a) implementation of the convolution-based signed distance
method of Gurumoorthy & Rangarajan.

This module is a thin ctypes binding of the C ABI in ``include/sdf.h``: the
functions ``sdf_plan_create``, ``sdf_execute``, ``sdf_execute_host``,
``sdf_backward``, ``sdf_sync``, ``sdf_plan_get_info``, ``sdf_get_stats`` and
``sdf_plan_destroy`` marshal arguments and nothing else; every step of the
method runs in the CUDA library.  :class:`Plan` wraps them with torch device
buffers and the current CUDA stream.  There is no CPU fallback: if the
library cannot be loaded, :func:`load_library` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libsdf_gb300.so")

SDF_FP64, SDF_FP32 = 0, 1
SDF_OUT_S, SDF_OUT_DS, SDF_OUT_D2S, SDF_OUT_SIGN = 1, 2, 4, 8
SDF_FLAG_CAPPED, SDF_FLAG_FIXUP, SDF_FLAG_SOURCE = 1, 2, 4
SDF_KERNEL_EXP, SDF_KERNEL_GREEN = 0, 1
STATUS = {0: "SDF_OK", 1: "SDF_ERR_INVALID_ARG", 2: "SDF_ERR_UNSUPPORTED",
          3: "SDF_ERR_POINT_OUT_OF_GRID", 4: "SDF_ERR_OOM", 5: "SDF_ERR_CUDA",
          6: "SDF_ERR_TIMEOUT", 7: "SDF_ERR_CAPACITY", 8: "SDF_ERR_INTERNAL"}

EXPORTED = ["sdf_plan_create", "sdf_execute", "sdf_execute_host", "sdf_backward", "sdf_sync",
            "sdf_plan_get_info", "sdf_get_stats", "sdf_plan_destroy", "sdf_status_string",
            "sdf_last_error", "sdf_profile_enable", "sdf_profile_read",
            "sdf_plan_set_noise_constants", "sdf_execute_noalloc", "sdf_batch_create",
            "sdf_batch_execute", "sdf_batch_sync", "sdf_batch_plan", "sdf_batch_destroy",
            "sdf_plan_set_tuning", "sdf_plan_autotune", "sdf_curvature", "sdf_plan_set_full_range",
            "sdf_mesh_sources", "sdf_plan_set_kernel", "sdf_green_profile", "sdf_execute_multi",
            "sdf_execute_multi_host", "sdf_plan_set_padding", "sdf_batch_autotune",
            "sdf_plan_set_epilogue_loads", "sdf_debug_hook", "sdf_set_debug_checks",
            "sdf_get_debug_checks"]
SDF_HOOK_FAIL_ALLOC, SDF_HOOK_TMA_WAIT_POLLS, SDF_HOOK_CORRUPT_BINS = 1, 2, 3


class SDFError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        msg = "%s: %s" % (where, STATUS.get(code, str(code)))
        try:
            extra = _lib().sdf_last_error().decode()
            if extra and code in (4, 5, 8):
                msg += " (%s)" % extra
        except Exception:
            pass
        super().__init__(msg)


class PlanInfo(ctypes.Structure):
    _fields_ = [("D", ctypes.c_int), ("precision", ctypes.c_int), ("outputs", ctypes.c_uint),
                ("dims", ctypes.c_int64 * 3), ("padded", ctypes.c_int64 * 3),
                ("h", ctypes.c_double), ("tau", ctypes.c_double),
                ("kernel_l1", ctypes.c_double * 16), ("n_kernels", ctypes.c_int),
                ("noise_const_fp32", ctypes.c_double), ("noise_const_fp64", ctypes.c_double),
                ("plan_ms", ctypes.c_double), ("workspace_bytes", ctypes.c_size_t)]


class ExecStats(ctypes.Structure):
    _fields_ = [("theta64", ctypes.c_double), ("theta32", ctypes.c_double), ("s_cap", ctypes.c_double),
                ("g_norm2", ctypes.c_double), ("n_unique", ctypes.c_int64),
                ("n_fixup_tiles", ctypes.c_int64), ("n_fixup_nodes", ctypes.c_int64),
                ("n_capped", ctypes.c_int64), ("n_launches", ctypes.c_int64),
                ("n_fixup_terms", ctypes.c_int64), ("err_bound_S", ctypes.c_double),
                ("err_bound_dS", ctypes.c_double), ("err_bound_d2S", ctypes.c_double),
                ("trusted_frac", ctypes.c_double)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


_LIBH = None
_LOCK = threading.Lock()


def load_library(path: str | None = None):
    """Load the CUDA library (building nothing).  Raises if it is missing."""
    global _LIBH
    with _LOCK:
        if _LIBH is not None:
            return _LIBH
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError("CUDA library %s is missing: run __graft_entry__.build()" % p)
        L = ctypes.CDLL(p)
        vp, i64, d, u = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_uint
        L.sdf_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(i64), d, d,
                                      ctypes.c_int, u, vp]
        L.sdf_execute.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp]
        L.sdf_execute_host.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp]
        L.sdf_backward.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp]
        L.sdf_curvature.argtypes = [vp, vp, vp, vp, vp]
        L.sdf_plan_set_full_range.argtypes = [vp, ctypes.c_int]
        L.sdf_plan_set_kernel.argtypes = [vp, ctypes.c_int]
        L.sdf_execute_multi.argtypes = [ctypes.c_int, ctypes.POINTER(vp), i64, vp, vp, ctypes.POINTER(vp),
                                        ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp)]
        L.sdf_execute_multi_host.argtypes = L.sdf_execute_multi.argtypes
        L.sdf_green_profile.argtypes = [ctypes.c_int, i64, vp, vp, vp, vp]
        L.sdf_mesh_sources.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp]
        L.sdf_sync.argtypes = [vp]
        L.sdf_plan_get_info.argtypes = [vp, ctypes.POINTER(PlanInfo)]
        L.sdf_get_stats.argtypes = [vp, ctypes.POINTER(ExecStats)]
        L.sdf_plan_destroy.argtypes = [vp]
        L.sdf_plan_destroy.restype = None
        L.sdf_status_string.argtypes = [ctypes.c_int]
        L.sdf_status_string.restype = ctypes.c_char_p
        L.sdf_last_error.argtypes = []
        L.sdf_last_error.restype = ctypes.c_char_p
        L.sdf_execute_noalloc.argtypes = [ctypes.c_int, ctypes.POINTER(i64), d, d, ctypes.c_int, u, i64,
                                          vp, vp, vp, vp, vp, vp, vp, vp]
        L.sdf_execute_noalloc.restype = ctypes.c_int
        pp = ctypes.POINTER(vp)
        L.sdf_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.POINTER(i64),
                                       ctypes.POINTER(d), ctypes.POINTER(d), ctypes.c_int, u, ctypes.c_int, vp]
        L.sdf_batch_create.restype = ctypes.c_int
        L.sdf_batch_execute.argtypes = [vp, ctypes.POINTER(i64), pp, pp, pp, pp, pp, pp, pp]
        L.sdf_batch_execute.restype = ctypes.c_int
        L.sdf_batch_sync.argtypes = [vp]
        L.sdf_batch_sync.restype = ctypes.c_int
        L.sdf_batch_plan.argtypes = [vp, ctypes.c_int]
        L.sdf_batch_plan.restype = vp
        L.sdf_batch_destroy.argtypes = [vp]
        L.sdf_batch_destroy.restype = None
        L.sdf_plan_set_tuning.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.sdf_plan_set_tuning.restype = ctypes.c_int
        ip = ctypes.POINTER(ctypes.c_int)
        L.sdf_plan_autotune.argtypes = [vp, i64, vp, vp, ctypes.c_int, ip, ip, ip]
        L.sdf_plan_autotune.restype = ctypes.c_int
        L.sdf_debug_hook.argtypes = [ctypes.c_int, i64]
        L.sdf_debug_hook.restype = ctypes.c_int
        L.sdf_set_debug_checks.argtypes = [ctypes.c_int]
        L.sdf_set_debug_checks.restype = ctypes.c_int
        L.sdf_get_debug_checks.argtypes = []
        L.sdf_get_debug_checks.restype = ctypes.c_int
        L.sdf_plan_set_epilogue_loads.argtypes = [vp, ctypes.c_int]
        L.sdf_plan_set_epilogue_loads.restype = ctypes.c_int
        L.sdf_plan_set_padding.argtypes = [vp, ctypes.POINTER(i64)]
        L.sdf_plan_set_padding.restype = ctypes.c_int
        L.sdf_batch_autotune.argtypes = [vp, ctypes.POINTER(i64), pp, pp, ctypes.c_int]
        L.sdf_batch_autotune.restype = ctypes.c_int
        L.sdf_plan_set_noise_constants.argtypes = [vp, d, d]
        L.sdf_plan_set_noise_constants.restype = ctypes.c_int
        L.sdf_profile_enable.argtypes = [vp, ctypes.c_int]
        L.sdf_profile_enable.restype = ctypes.c_int
        L.sdf_profile_read.argtypes = [vp, ctypes.POINTER(KernelTime), ctypes.c_int]
        L.sdf_profile_read.restype = ctypes.c_int
        for n in ("sdf_plan_create", "sdf_execute", "sdf_execute_host", "sdf_backward", "sdf_sync",
                  "sdf_plan_get_info", "sdf_get_stats", "sdf_curvature", "sdf_plan_set_full_range", "sdf_mesh_sources",
                  "sdf_plan_set_kernel", "sdf_green_profile", "sdf_execute_multi",
                  "sdf_execute_multi_host"):
            getattr(L, n).restype = ctypes.c_int
        _LIBH = L
        return L


def _lib():
    return load_library()


def _ck(code, where):
    if code != 0:
        raise SDFError(code, where)


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------- C-ABI names
def sdf_plan_create(D, dims, h, tau, precision, outputs, stream):
    """Create a plan; returns the opaque handle (ctypes.c_void_p)."""
    handle = ctypes.c_void_p()
    dims_arr = (ctypes.c_int64 * len(dims))(*[int(x) for x in dims])
    _ck(_lib().sdf_plan_create(ctypes.byref(handle), int(D), dims_arr, float(h), float(tau),
                               int(precision), int(outputs), ctypes.c_void_p(stream or 0)),
        "sdf_plan_create")
    return handle


def sdf_execute(handle, K, points, weights, S, dS, d2S, sign, flags):
    _ck(_lib().sdf_execute(handle, int(K), _ptr(points), _ptr(weights), _ptr(S), _ptr(dS),
                           _ptr(d2S), _ptr(sign), _ptr(flags)), "sdf_execute")


def sdf_execute_multi(handles, K, points, weights, S, dS, d2S, sign, flags):
    """handles: list of plan handles; S ... flags: lists (one tensor or None
    per plan) or None."""
    n = len(handles)
    hv = (ctypes.c_void_p * n)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])

    def arr(lst):
        if lst is None:
            return None
        return (ctypes.c_void_p * n)(*[(t.data_ptr() if t is not None else None) for t in lst])
    _ck(_lib().sdf_execute_multi(n, hv, int(K), _ptr(points), _ptr(weights), arr(S), arr(dS), arr(d2S),
                                 arr(sign), arr(flags)), "sdf_execute_multi")


def sdf_execute_multi_host(handles, K, points, weights, S, dS, d2S, sign, flags):
    """As sdf_execute_multi with host tensors: outputs come back by the copy
    engine, the first plan's S/dS/d2S (when pinned) while the other plans
    still compute."""
    n = len(handles)
    hv = (ctypes.c_void_p * n)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])

    def arr(lst):
        if lst is None:
            return None
        return (ctypes.c_void_p * n)(*[(t.data_ptr() if t is not None else None) for t in lst])
    _ck(_lib().sdf_execute_multi_host(n, hv, int(K), _ptr(points), _ptr(weights), arr(S), arr(dS), arr(d2S),
                                      arr(sign), arr(flags)), "sdf_execute_multi_host")


def sdf_execute_host(handle, K, points, weights, S, dS, d2S, sign, flags):
    _ck(_lib().sdf_execute_host(handle, int(K), _ptr(points), _ptr(weights), _ptr(S), _ptr(dS),
                                _ptr(d2S), _ptr(sign), _ptr(flags)), "sdf_execute_host")


def sdf_backward(handle, K, points, w, S_saved, flags, dL_dY, dL_dtau):
    _ck(_lib().sdf_backward(handle, int(K), _ptr(points), _ptr(w), _ptr(S_saved), _ptr(flags),
                            _ptr(dL_dY), _ptr(dL_dtau)), "sdf_backward")


def sdf_plan_set_full_range(handle, enable):
    _ck(_lib().sdf_plan_set_full_range(handle, 1 if enable else 0), "sdf_plan_set_full_range")


def sdf_plan_set_kernel(handle, kernel_set):
    _ck(_lib().sdf_plan_set_kernel(handle, int(kernel_set)), "sdf_plan_set_kernel")


def sdf_green_profile(D, z):
    """Gamma_D(z), Gamma_D'(z), Gamma_D''(z) of the Green's function set (host
    arrays; see include/sdf.h)."""
    z = np.ascontiguousarray(z, dtype=np.float64).ravel()
    g, g1, g2 = (np.empty_like(z) for _ in range(3))
    vp = ctypes.c_void_p
    _ck(_lib().sdf_green_profile(int(D), z.size, vp(z.ctypes.data), vp(g.ctypes.data), vp(g1.ctypes.data),
                                 vp(g2.ctypes.data)), "sdf_green_profile")
    return g, g1, g2


def sdf_mesh_sources(handle, nf, nv, V, F, center, points, weights):
    c = None
    if center is not None:
        c = (ctypes.c_double * 3)(*[float(x) for x in center])
    _ck(_lib().sdf_mesh_sources(handle, int(nf), int(nv), _ptr(V), _ptr(F),
                                ctypes.cast(c, ctypes.c_void_p) if c is not None else None,
                                _ptr(points), _ptr(weights)), "sdf_mesh_sources")


def sdf_curvature(handle, dS, d2S, flags, curv):
    _ck(_lib().sdf_curvature(handle, _ptr(dS), _ptr(d2S), _ptr(flags), _ptr(curv)), "sdf_curvature")


def sdf_sync(handle):
    return int(_lib().sdf_sync(handle))


def sdf_plan_get_info(handle) -> PlanInfo:
    info = PlanInfo()
    _ck(_lib().sdf_plan_get_info(handle, ctypes.byref(info)), "sdf_plan_get_info")
    return info


def sdf_get_stats(handle) -> ExecStats:
    st = ExecStats()
    _ck(_lib().sdf_get_stats(handle, ctypes.byref(st)), "sdf_get_stats")
    return st


def sdf_plan_set_noise_constants(handle, c_fp32, c_fp64):
    _ck(_lib().sdf_plan_set_noise_constants(handle, float(c_fp32), float(c_fp64)),
        "sdf_plan_set_noise_constants")


def sdf_execute_noalloc(D, dims, h, tau, precision, outputs, K, points, weights, S, dS, d2S, sign,
                        flags, stream):
    """The whole path for a small problem with no device allocation (scratch in
    a static array inside the library).  Synchronous; returns nothing."""
    dims_arr = (ctypes.c_int64 * len(dims))(*[int(x) for x in dims])
    _ck(_lib().sdf_execute_noalloc(int(D), dims_arr, float(h), float(tau), int(precision), int(outputs),
                                   int(K), _ptr(points), _ptr(weights), _ptr(S), _ptr(dS), _ptr(d2S),
                                   _ptr(sign), _ptr(flags), ctypes.c_void_p(stream or 0)),
        "sdf_execute_noalloc")


def sdf_plan_set_tuning(handle, lines_T, lines_F, fused_variant):
    _ck(_lib().sdf_plan_set_tuning(handle, int(lines_T), int(lines_F), int(fused_variant)),
        "sdf_plan_set_tuning")


def sdf_plan_autotune(handle, K, points, weights, reps):
    """Returns (lines_T, lines_F, fused_variant) chosen by the library."""
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _ck(_lib().sdf_plan_autotune(handle, int(K), _ptr(points), _ptr(weights), int(reps), ctypes.byref(a),
                                 ctypes.byref(b), ctypes.byref(c)), "sdf_plan_autotune")
    return a.value, b.value, c.value


def _ptr_array(ts):
    if ts is None:
        return None
    arr = (ctypes.c_void_p * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = None if t is None else t.data_ptr()
    return arr


def sdf_batch_create(D, dims_list, h_list, tau_list, precision, outputs, n_streams, stream):
    n = len(dims_list)
    dims = (ctypes.c_int64 * (n * D))(*[int(x) for dd in dims_list for x in dd])
    hs = (ctypes.c_double * n)(*[float(x) for x in h_list])
    ts = (ctypes.c_double * n)(*[float(x) for x in tau_list])
    handle = ctypes.c_void_p()
    _ck(_lib().sdf_batch_create(ctypes.byref(handle), n, int(D), dims, hs, ts, int(precision), int(outputs),
                                int(n_streams), ctypes.c_void_p(stream or 0)), "sdf_batch_create")
    return handle


def sdf_batch_execute(handle, K, points, weights, S, dS, d2S, sign, flags):
    Ks = (ctypes.c_int64 * len(K))(*[int(k) for k in K])
    _ck(_lib().sdf_batch_execute(handle, Ks, _ptr_array(points), _ptr_array(weights), _ptr_array(S),
                                 _ptr_array(dS), _ptr_array(d2S), _ptr_array(sign), _ptr_array(flags)),
        "sdf_batch_execute")


def sdf_debug_hook(hook, value):
    """Test hooks of the failure paths (SDF_HOOK_*)."""
    _ck(_lib().sdf_debug_hook(int(hook), int(value)), "sdf_debug_hook")


def sdf_set_debug_checks(on):
    """Device-side consistency checks for every later execute (process-wide):
    a failed check raises SDFError with code 8 (SDF_ERR_INTERNAL) at sync."""
    _ck(_lib().sdf_set_debug_checks(1 if on else 0), "sdf_set_debug_checks")


def sdf_get_debug_checks():
    return bool(_lib().sdf_get_debug_checks())


def sdf_plan_set_epilogue_loads(handle, mode):
    """0: TMA staging where it applies (default); 1: per-thread loads."""
    _ck(_lib().sdf_plan_set_epilogue_loads(handle, int(mode)), "sdf_plan_set_epilogue_loads")


def sdf_plan_set_padding(handle, padded):
    """Padded transform size per axis (2^k or 3*2^k, >= 2N-1)."""
    arr = (ctypes.c_int64 * len(padded))(*[int(x) for x in padded])
    _ck(_lib().sdf_plan_set_padding(handle, arr), "sdf_plan_set_padding")


def sdf_batch_autotune(handle, K, points, weights, reps):
    n = len(K)
    kv = (ctypes.c_int64 * n)(*[int(k) for k in K])
    _ck(_lib().sdf_batch_autotune(handle, kv, _ptr_array(points), _ptr_array(weights), int(reps)),
        "sdf_batch_autotune")


def sdf_batch_sync(handle):
    return int(_lib().sdf_batch_sync(handle))


def sdf_batch_plan(handle, i):
    return ctypes.c_void_p(_lib().sdf_batch_plan(handle, int(i)))


def sdf_batch_destroy(handle):
    _lib().sdf_batch_destroy(handle)


def sdf_profile_enable(handle, enable):
    _ck(_lib().sdf_profile_enable(handle, int(bool(enable))), "sdf_profile_enable")


def sdf_profile_read(handle, max_entries=64):
    """{kernel name: (launches, total_ms)} since the last read."""
    arr = (KernelTime * max_entries)()
    n = _lib().sdf_profile_read(handle, arr, max_entries)
    if n < 0:
        raise SDFError(5, "sdf_profile_read")
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(n)}


def sdf_plan_destroy(handle):
    _lib().sdf_plan_destroy(handle)


# ---------------------------------------------------------------- convenience
_OUTS = {"S": SDF_OUT_S, "dS": SDF_OUT_DS, "d2S": SDF_OUT_D2S, "sign": SDF_OUT_SIGN}
_KERNELS = {"exp": SDF_KERNEL_EXP, "green": SDF_KERNEL_GREEN}


def execute_multi(plans, points, weights=None, outs=None, check=True):
    """sdf_execute_multi over Plan objects: one snapping and forward transform
    for all of them (same D, dims, h, precision, outputs).  Returns one output
    dict per plan."""
    t = plans[0].torch
    pts = points.to(device="cuda", dtype=t.float64).contiguous()
    w = None if weights is None else weights.to(device="cuda", dtype=t.float64).contiguous()
    if outs is None:
        outs = []
        for p in plans:
            want = [k for k, v in _OUTS.items() if p.outputs & v] + ["flags"]
            outs.append(p.alloc_outputs(want, signed=w is not None))
    col = lambda k: [o.get(k) for o in outs] if any(k in o for o in outs) else None
    sdf_execute_multi([p.handle for p in plans], pts.shape[0], pts, w, col("S"), col("dS"), col("d2S"),
                      col("sign"), col("flags"))
    if check:
        for p in plans:
            p.sync()
    return outs


class Plan:
    """A plan for one grid (D, dims, h) and tau, on the current torch stream."""

    def __init__(self, D, dims, h, tau, precision="fp32", outputs=("S", "dS", "sign"), stream=None,
                 full_range=False, kernel="exp"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.torch = torch
        self.D = int(D)
        self.dims = tuple(int(x) for x in dims)
        self.h, self.tau = float(h), float(tau)
        self.precision = SDF_FP64 if precision in ("fp64", SDF_FP64) else SDF_FP32
        mask = 0
        for o in outputs:
            mask |= _OUTS[o]
        self.outputs = mask | SDF_OUT_S
        if self.outputs & SDF_OUT_D2S:
            self.outputs |= SDF_OUT_DS
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = sdf_plan_create(self.D, self.dims, self.h, self.tau, self.precision,
                                      self.outputs, self.stream.cuda_stream)
        self.dtype = torch.float64 if self.precision == SDF_FP64 else torch.float32
        self.n_nodes = int(np.prod(self.dims))
        if full_range:
            sdf_plan_set_full_range(self.handle, True)
        if kernel != "exp":
            self.set_kernel(kernel)

    def set_padding(self, padded):
        """Padded transform size per axis (sdf_plan_set_padding)."""
        sdf_plan_set_padding(self.handle, padded)

    def set_kernel(self, kernel):
        """'exp' (the paper's G~, default) or 'green' (the exact Green's
        function, SDF_FP64 plans)."""
        sdf_plan_set_kernel(self.handle, _KERNELS[kernel])

    def close(self):
        if getattr(self, "handle", None) is not None:
            sdf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def info(self) -> PlanInfo:
        return sdf_plan_get_info(self.handle)

    def stats(self) -> ExecStats:
        return sdf_get_stats(self.handle)

    def profile(self, enable=True):
        sdf_profile_enable(self.handle, enable)

    def profile_read(self):
        return sdf_profile_read(self.handle)

    def sync(self):
        _ck(sdf_sync(self.handle), "sdf_sync")

    def alloc_outputs(self, want=None, signed=True):
        t = self.torch
        dev = t.device("cuda")
        want = want or [k for k, v in _OUTS.items() if self.outputs & v]
        shp = tuple(reversed(self.dims))
        nh = self.D * (self.D + 1) // 2
        out = {}
        if "S" in want:
            out["S"] = t.empty(shp, dtype=self.dtype, device=dev)
        if "dS" in want and self.outputs & SDF_OUT_DS:
            out["dS"] = t.empty((self.D,) + shp, dtype=self.dtype, device=dev)
        if "d2S" in want and self.outputs & SDF_OUT_D2S:
            out["d2S"] = t.empty((nh,) + shp, dtype=self.dtype, device=dev)
        if "sign" in want and self.outputs & SDF_OUT_SIGN and signed:
            out["sign"] = t.empty(shp, dtype=t.int8, device=dev)
        if "flags" in want:
            out["flags"] = t.empty(shp, dtype=t.uint8, device=dev)
        return out

    def execute(self, points, weights=None, out=None, flags=True, check=True):
        """Run the whole path on device tensors; returns the output dict.
        Grid arrays are shaped (N_z, N_y, N_x) / (N_y, N_x) (x fastest)."""
        t = self.torch
        pts = points.to(device="cuda", dtype=t.float64).contiguous()
        w = None if weights is None else weights.to(device="cuda", dtype=t.float64).contiguous()
        if out is None:
            want = [k for k, v in _OUTS.items() if self.outputs & v] + (["flags"] if flags else [])
            out = self.alloc_outputs(want, signed=w is not None)
        sdf_execute(self.handle, pts.shape[0], pts, w, out.get("S"), out.get("dS"), out.get("d2S"),
                    out.get("sign"), out.get("flags"))
        if check:
            self.sync()
        return out

    def execute_host(self, points, weights=None, out=None):
        """sdf_execute_host on host tensors (pinned S/dS/d2S are written by the kernels directly)."""
        t = self.torch
        pts = points.to(dtype=t.float64).contiguous()
        w = None if weights is None else weights.to(dtype=t.float64).contiguous()
        if out is None:
            shp = tuple(reversed(self.dims))
            out = {"S": t.empty(shp, dtype=self.dtype, pin_memory=True)}
        sdf_execute_host(self.handle, pts.shape[0], pts, w, out.get("S"), out.get("dS"),
                         out.get("d2S"), out.get("sign"), out.get("flags"))
        return out

    def mesh_sources(self, V, F, center=None):
        """Incentres and area-weighted normals (device, nf x 3 each) of a
        triangle mesh (V: nv x 3, F: nf x 3 int64) for execute()."""
        t = self.torch
        Vd = V.to(device="cuda", dtype=t.float64).contiguous()
        Fd = F.to(device="cuda", dtype=t.int64).contiguous()
        pts = t.empty((Fd.shape[0], 3), dtype=t.float64, device="cuda")
        w = t.empty_like(pts)
        sdf_mesh_sources(self.handle, Fd.shape[0], Vd.shape[0], Vd, Fd, center, pts, w)
        self.sync()
        return pts, w

    def curvature(self, out):
        """Gaussian, mean and principal curvatures (4, *grid) from an execute's
        output dict (needs dS and d2S; flags used when present)."""
        t = self.torch
        curv = t.empty((4,) + tuple(out["S"].shape), dtype=self.dtype, device="cuda")
        sdf_curvature(self.handle, out["dS"], out["d2S"], out.get("flags"), curv)
        self.sync()
        return curv

    def backward(self, points, w, S_saved, flags=None):
        """dL/dY (K x D, float64, device) and dL/dtau (float64 scalar)."""
        t = self.torch
        pts = points.to(device="cuda", dtype=t.float64).contiguous()
        dY = t.empty_like(pts)
        dtau = t.zeros(1, dtype=t.float64, device="cuda")
        sdf_backward(self.handle, pts.shape[0], pts, w.contiguous(), S_saved.contiguous(),
                     None if flags is None else flags.contiguous(), dY, dtau)
        self.sync()
        return dY, dtau


class Batch:
    """Independent problems of one dimension D executed as one graph launch."""

    def __init__(self, D, dims_list, h_list, tau_list, precision="fp32", outputs=("S", "sign"),
                 n_streams=8, stream=None):
        import torch
        self.torch = torch
        self.D = int(D)
        self.dims = [tuple(int(x) for x in d) for d in dims_list]
        self.precision = SDF_FP64 if precision in ("fp64", SDF_FP64) else SDF_FP32
        mask = 0
        for o in outputs:
            mask |= _OUTS[o]
        self.outputs = mask | SDF_OUT_S
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = sdf_batch_create(self.D, self.dims, h_list, tau_list, self.precision, self.outputs,
                                       n_streams, self.stream.cuda_stream)
        self.dtype = torch.float64 if self.precision == SDF_FP64 else torch.float32

    def alloc_outputs(self, signed=True, flags=True):
        t = self.torch
        outs = []
        for d in self.dims:
            shp = tuple(reversed(d))
            o = {"S": t.empty(shp, dtype=self.dtype, device="cuda")}
            if self.outputs & SDF_OUT_SIGN and signed:
                o["sign"] = t.empty(shp, dtype=t.int8, device="cuda")
            if flags:
                o["flags"] = t.empty(shp, dtype=t.uint8, device="cuda")
            outs.append(o)
        return outs

    def execute(self, points, weights, outs):
        """points/weights: lists of device float64 tensors; outs from alloc_outputs."""
        K = [int(p.shape[0]) for p in points]
        col = lambda k: [o.get(k) for o in outs] if any(k in o for o in outs) else None
        sdf_batch_execute(self.handle, K, points, weights, col("S"), col("dS"), col("d2S"), col("sign"),
                          col("flags"))

    def autotune(self, points, weights, reps=2):
        """sdf_batch_autotune on device tensors (padded sizes and tile schedules)."""
        sdf_batch_autotune(self.handle, [int(p.shape[0]) for p in points], points, weights, reps)

    def sync(self):
        _ck(sdf_batch_sync(self.handle), "sdf_batch_sync")

    def close(self):
        if getattr(self, "handle", None) is not None:
            sdf_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
