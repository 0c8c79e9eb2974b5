"""CPU-side checks of the C ABI: the library builds, loads and exports every
entry point include/sdf.h declares (no compute calls without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sdf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sdf_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1112_3010_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_path(lib):
    names = _declared()
    for n in ("sdf_plan_create", "sdf_execute", "sdf_backward", "sdf_plan_destroy", "sdf_sync"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    import paper_1112_3010_gb300 as pkg
    for n in _declared():
        assert n in pkg.EXPORTED, n


def test_status_strings(lib):
    lib.sdf_status_string.restype = ctypes.c_char_p
    for code in range(8):
        assert lib.sdf_status_string(code)
    assert lib.sdf_status_string(0) == b"ok"


def test_invalid_arguments_rejected_on_host(lib):
    """Argument checks run before any CUDA call, so they work without a GPU."""
    lib.sdf_plan_create.restype = ctypes.c_int
    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 3)(64, 64, 64)
    # D = 4 -> SDF_ERR_UNSUPPORTED
    assert lib.sdf_plan_create(ctypes.byref(h), 4, dims, ctypes.c_double(0.1),
                               ctypes.c_double(0.01), 1, 1, None) == 2
    # tau <= 0 -> SDF_ERR_INVALID_ARG
    assert lib.sdf_plan_create(ctypes.byref(h), 2, dims, ctypes.c_double(0.1),
                               ctypes.c_double(-1.0), 1, 1, None) == 1
    # grid too large -> SDF_ERR_UNSUPPORTED
    big = (ctypes.c_int64 * 3)(8192, 8192, 1)
    assert lib.sdf_plan_create(ctypes.byref(h), 2, big, ctypes.c_double(0.1),
                               ctypes.c_double(0.01), 1, 1, None) == 2
    # execute on a NULL plan -> SDF_ERR_INVALID_ARG
    lib.sdf_execute.restype = ctypes.c_int
    assert lib.sdf_execute(None, ctypes.c_int64(10), None, None, None, None, None, None, None) == 1


def test_oracle_is_not_linked_by_the_product():
    """The product path never imports the oracle."""
    pkg_dir = os.path.join(ROOT, "paper_1112_3010_gb300")
    for dp, _, fs in os.walk(pkg_dir):
        for f in fs:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert "import oracle" not in txt and "sdf_oracle" not in txt, f


def test_green_profile_host_utility():
    """sdf_green_profile (host only) against scipy's K_0 / K_1 and the closed
    forms of the 1D and 3D profiles; z = 0 gives the unit-box integral."""
    import numpy as np
    import scipy.integrate as si
    import scipy.special as sp

    import paper_1112_3010_gb300 as pkg
    pkg.load_library()
    z = np.concatenate([np.logspace(-8, 0, 40), np.linspace(1.0, 60.0, 200), [19.999, 20.0, 20.001, 700.0]])
    g, g1, g2 = pkg.sdf_green_profile(2, z)
    k0, k1 = sp.k0(z), sp.k1(z)
    np.testing.assert_allclose(g, k0, rtol=1e-13)
    np.testing.assert_allclose(-g1, k1, rtol=1e-13)
    np.testing.assert_allclose(g2, k0 + k1 / z, rtol=1e-13)
    g, g1, g2 = pkg.sdf_green_profile(3, z)
    np.testing.assert_allclose(g, np.exp(-z) / z, rtol=1e-14)
    np.testing.assert_allclose(g1, -np.exp(-z) * (1 / z + 1 / z ** 2), rtol=1e-14)
    g, g1, g2 = pkg.sdf_green_profile(1, z)
    np.testing.assert_allclose(g, np.exp(-z), rtol=1e-15)
    # the unit-box integrals by direct adaptive quadrature of the singular integrands
    a2 = 4 * si.dblquad(lambda y, x: sp.k0(np.hypot(x, y)), 0, 0.5, 0, 0.5, epsabs=1e-14, epsrel=1e-13)[0]
    assert abs(pkg.sdf_green_profile(2, [0.0])[0][0] - a2) < 1e-12
    a3 = 8 * si.tplquad(lambda c, b, a: np.exp(-np.sqrt(a * a + b * b + c * c)) / np.sqrt(a * a + b * b + c * c),
                        0, 0.5, 0, 0.5, 0, 0.5, epsabs=1e-12, epsrel=1e-12)[0]
    assert abs(pkg.sdf_green_profile(3, [0.0])[0][0] - a3) < 1e-10
    with pytest.raises(pkg.SDFError):
        pkg.sdf_green_profile(2, [-1.0])
    with pytest.raises(pkg.SDFError):
        pkg.sdf_green_profile(4, [1.0])


def test_multi_execute_rejects_bad_arguments_on_host(lib):
    """sdf_execute_multi / _host check their arguments before any CUDA call."""
    for fn in (lib.sdf_execute_multi, lib.sdf_execute_multi_host):
        fn.restype = ctypes.c_int
        vp = ctypes.c_void_p
        pts = (ctypes.c_double * 4)()
        plans = (vp * 2)(None, None)
        assert fn(0, plans, ctypes.c_int64(2), pts, None, None, None, None, None, None) == 1  # n < 1
        assert fn(2, None, ctypes.c_int64(2), pts, None, None, None, None, None, None) == 1   # no plans
        assert fn(2, plans, ctypes.c_int64(2), pts, None, None, None, None, None, None) == 1  # NULL plan


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """No CPU fallback: without the built library the binding raises, and a
    Plan cannot be made on a machine without a GPU."""
    import paper_1112_3010_gb300 as pkg
    monkeypatch.setattr(pkg, "_LIBH", None)
    with pytest.raises(ImportError):
        pkg.load_library(str(tmp_path / "absent.so"))
    import torch
    if not torch.cuda.is_available():
        with pytest.raises(RuntimeError):
            pkg.Plan(2, (16, 16), 1 / 16, 0.1)
