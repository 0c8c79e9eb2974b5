"""Triangle-mesh input for the 3D sign (sdf_mesh_sources, Sec. 4.2 and
Example 5): sources against the oracle, then the degree's sign on a grid
against the oracle (exactly, off the boundary band) and against the exact
solid-angle degree of the mesh far from the surface."""
import numpy as np
import pytest
import torch

import oracle
import paper_1112_3010_gb300 as pkg
from paper_1112_3010_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

MESHES = {"sphere": lambda: wl.mesh_sphere(r=0.3),
          "cube": lambda: wl.mesh_cube(half=0.25),
          "cylinder": lambda: wl.mesh_cylinder(r=0.22, half_height=0.3)}


@pytest.mark.parametrize("kind", list(MESHES))
@pytest.mark.parametrize("center", [None, (0.5, 0.5, 0.5)])
def test_mesh_sources_match_oracle(kind, center):
    V, F = MESHES[kind]()
    plan = pkg.Plan(3, (16, 16, 16), 1 / 16, 0.1, precision="fp64", outputs=("S", "sign"))
    Y, P = plan.mesh_sources(torch.from_numpy(V), torch.from_numpy(F), center=center)
    Yo, Po = oracle.mesh_sources(V, F, center=center)
    assert np.allclose(Y.cpu().numpy(), Yo, rtol=1e-12, atol=1e-15)
    assert np.allclose(P.cpu().numpy(), Po, rtol=1e-12, atol=1e-15)
    plan.close()


@pytest.mark.parametrize("kind", list(MESHES))
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mesh_sign_matches_oracle_and_exact_degree(kind, precision):
    V, F = MESHES[kind]()
    N = 48
    h = 1.0 / N
    tau = 1.5 * h
    plan = pkg.Plan(3, (N, N, N), h, tau, precision=precision, outputs=("S", "sign"))
    Y, P = plan.mesh_sources(torch.from_numpy(V), torch.from_numpy(F))
    out = plan.execute(Y, P)
    sign = out["sign"].reshape(-1).cpu().numpy()
    n = N ** 3
    rng = np.random.default_rng(11)
    sel = rng.choice(n, 6000, replace=False)
    X = oracle.grid_nodes((N, N, N), h, sel)
    # the oracle on the same snapped sources
    idx, inside = oracle.snap(Y.cpu().numpy(), h, (N, N, N))
    Ys = idx[inside].astype(np.float64) * h
    Ps = P.cpu().numpy()[inside]
    mu = oracle.evaluate(Ys, X, tau, weights=Ps, want=("mu",))["mu"]
    d_src = np.min(np.linalg.norm(X[:, None, :] - Ys[None, :, :], axis=2), axis=1)
    band = 2 * np.linalg.norm(Ps, axis=1).max() + h * np.sqrt(3)
    off = (d_src > band) & (np.abs(np.abs(mu) - 0.5) >= 0.05)
    assert off.sum() > 3000
    assert np.array_equal(sign[sel][off], oracle.sign_from_mu(mu[off]))
    # far from the surface the method's sign is the exact degree's
    deg = oracle.solid_angle_degree(V, F, X)
    far = d_src > 4 * h
    assert np.array_equal(sign[sel][far], np.where(deg[far] > 0.5, 1, -1).astype(np.int8))
    plan.close()


def test_mesh_bad_face_index_reported():
    V, F = MESHES["cube"]()
    F = F.copy()
    F[5, 1] = V.shape[0] + 3
    plan = pkg.Plan(3, (16, 16, 16), 1 / 16, 0.1, precision="fp32", outputs=("S", "sign"))
    with pytest.raises(pkg.SDFError):
        plan.mesh_sources(torch.from_numpy(V), torch.from_numpy(F))
    # the plan stays usable
    Vs, Fs = MESHES["sphere"]()
    Y, P = plan.mesh_sources(torch.from_numpy(Vs), torch.from_numpy(Fs))
    out = plan.execute(Y, P)
    assert out["sign"].numel() == 16 ** 3
    plan.close()
