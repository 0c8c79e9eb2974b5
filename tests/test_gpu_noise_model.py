"""Calibration pin of the transform error model behind the trust threshold.

With the trust threshold switched off (noise constants ~0), the FFT's phi is
recovered from S at every node and compared with the oracle's phi.  The
largest absolute error must stay below C_p u_p sqrt(log2 n) ||k||_1 ||g||_2 /
sqrt(n) with the library's built-in C_p, for phi and for the gradient
numerators.  The measured ratios are printed (they are the calibration)."""
import numpy as np
import pytest
import torch

import paper_1112_3010_gb300 as pkg
from paper_1112_3010_gb300 import workloads as wl

from parity_util import oracle_ref, sample_nodes

pytestmark = pytest.mark.gpu


def _cases():
    return {
        "circle128": lambda: wl.config_c1(),
        "stars256": lambda: wl.stars(N=256, K=3000, n_shapes=3, tau=0.006, seed=5),
        "stars256_small_tau": lambda: wl.stars(N=256, K=3000, n_shapes=3, tau=0.002, seed=6),
        "sphere40": lambda: wl.sphere(N=40, K=3000, radius=0.3, tau=0.03, seed=8),
    }


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", list(_cases()))
def test_noise_model(name, prec):
    s = _cases()[name]()
    plan = pkg.Plan(s.D, s.dims, s.h, s.tau, precision=prec, outputs=("S", "dS"))
    info = plan.info
    c_builtin = info.noise_const_fp64 if prec == "fp64" else info.noise_const_fp32
    pkg.sdf_plan_set_noise_constants(plan.handle, 1e-30, 1e-30)
    out = plan.execute(torch.from_numpy(s.points).cuda())
    st = plan.stats()
    flags = out["flags"].cpu().numpy().ravel()
    S = out["S"].cpu().numpy().ravel().astype(np.float64)
    G = out["dS"].cpu().numpy().reshape(s.D, -1).T.astype(np.float64)
    ref = oracle_ref(s, with_weights=False, want=("S", "dS"))
    phi_t = np.exp(-ref["S"] / s.tau)
    use = (flags & (pkg.SDF_FLAG_CAPPED | pkg.SDF_FLAG_FIXUP)) == 0
    # S -> phi = exp(-S/tau) amplifies S's own rounding by |S|/tau; keep nodes
    # where that is far below the transform noise
    use &= phi_t < 1e-3 * phi_t.max()
    phi_g = np.exp(-S / s.tau)
    n = float(np.prod(info.padded[: s.D]))
    u = 2.0 ** -53 if prec == "fp64" else 2.0 ** -24
    l1 = list(info.kernel_l1[: info.n_kernels])   # PHI, GX, GY[, GZ]
    base = u * np.sqrt(np.log2(n)) * st.g_norm2 / np.sqrt(n)
    # a channel's noise follows the larger l1 norm of its packed pair:
    # (PHI, GX), then GY alone (2D) or (GY, GZ) (3D)
    pair = [max(l1[0], l1[1]), l1[2] if s.D == 2 else max(l1[2], l1[3])]
    n_ch = [pair[0], pair[0], pair[1]] + ([pair[1]] if s.D == 3 else [])
    err_phi = np.abs(phi_g[use] - phi_t[use]).max()
    c_phi = err_phi / (base * n_ch[0])
    num_g = G * phi_g[:, None]
    num_t = ref["dS"] * phi_t[:, None]
    c_g = max(np.abs(num_g[use, a] - num_t[use, a]).max() / (base * n_ch[1 + a]) for a in range(s.D))
    print("noise-model %s %s: C_phi=%.3g C_grad=%.3g (built-in %.3g), nodes=%d"
          % (name, prec, c_phi, c_g, c_builtin, use.sum()))
    assert use.sum() > 100
    assert c_phi <= c_builtin
    assert c_g <= c_builtin


def _full_cases():
    return {
        "stars2048_tau0.002": lambda: wl.config_c2(tau=0.002),
        "stars2048_tau0.0005": lambda: wl.config_c2(tau=0.0005),
        "torus_sphere256": lambda: wl.config_c3(),
    }


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", list(_full_cases()))
def test_noise_model_full_size(name, prec):
    """The same calibration at the bench and 3D workload sizes (4096^2- and
    512^3-point transforms), on sampled nodes the oracle computes one by one:
    uniform nodes (mostly the far field, where the noise shows) plus nodes
    near the points.  The measured ratios are printed."""
    s = _full_cases()[name]()
    outs = ("S", "dS")
    plan = pkg.Plan(s.D, s.dims, s.h, s.tau, precision=prec, outputs=outs)
    info = plan.info
    c_builtin = info.noise_const_fp64 if prec == "fp64" else info.noise_const_fp32
    pkg.sdf_plan_set_noise_constants(plan.handle, 1e-30, 1e-30)
    out = plan.execute(torch.from_numpy(s.points).cuda())
    st = plan.stats()
    plan.close()
    sel = sample_nodes(s, n_uniform=6000, n_near=3000, seed=55)
    flags = out["flags"].cpu().numpy().ravel()[sel]
    S = out["S"].cpu().numpy().ravel()[sel].astype(np.float64)
    G = out["dS"].cpu().numpy().reshape(s.D, -1)[:, sel].T.astype(np.float64)
    ref = oracle_ref(s, sel=sel, with_weights=False, want=("S", "dS"))
    phi_t = np.exp(-ref["S"] / s.tau)
    use = (flags & (pkg.SDF_FLAG_CAPPED | pkg.SDF_FLAG_FIXUP)) == 0
    use &= phi_t < 1e-3 * phi_t.max()
    phi_g = np.exp(-S / s.tau)
    n = float(np.prod(info.padded[: s.D]))
    u = 2.0 ** -53 if prec == "fp64" else 2.0 ** -24
    l1 = list(info.kernel_l1[: info.n_kernels])
    base = u * np.sqrt(np.log2(n)) * st.g_norm2 / np.sqrt(n)
    pair = [max(l1[0], l1[1]), l1[2] if s.D == 2 else max(l1[2], l1[3])]
    n_ch = [pair[0], pair[0], pair[1]] + ([pair[1]] if s.D == 3 else [])
    c_phi = np.abs(phi_g[use] - phi_t[use]).max() / (base * n_ch[0])
    num_g = G * phi_g[:, None]
    num_t = ref["dS"] * phi_t[:, None]
    c_g = max(np.abs(num_g[use, a] - num_t[use, a]).max() / (base * n_ch[1 + a]) for a in range(s.D))
    print("noise-model %s %s: C_phi=%.3g C_grad=%.3g (built-in %.3g), nodes=%d"
          % (name, prec, c_phi, c_g, c_builtin, use.sum()))
    assert use.sum() > 1000
    assert c_phi <= c_builtin
    assert c_g <= c_builtin
