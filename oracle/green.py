"""FP64 oracle for the exact Green's function kernel set.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` (and nothing in the product
path).  Plain numpy; K_0 and K_1 come from ``scipy.special`` and the box
integral at the origin from ``scipy.integrate`` (library primitives).

What it computes, step by step as the paper states it:

* Sec. 2.1, eqs. GreensFunction1D/2D/3D: the Green's function of
  -tau^2 lap phi + phi = psi is G(X) = tau^-D c_D Gamma_D(||X||/tau) with
  Gamma_1 = exp(-z), Gamma_2 = K_0(z), Gamma_3 = exp(-z)/z and
  c_1 = 1/2, c_2 = 1/(2 pi), c_3 = 1/(4 pi).
* Sec. 2.2: psi_k = tau^-D/2 on the box of side tau around Y_k (square
  integrable to one), so phi(X) = tau^-D/2 sum_k int_{B_k(X)} G; eq.
  phiapproxSol takes each integral at its mid-point value tau^D G(X - Y_k),
  i.e. gamma = D/2:  phi(X) = tau^-D/2 c_D sum_k Gamma_D(||X - Y_k||/tau).
* Where the mid-point value is infinite (X = Y_k, D >= 2) the integral is
  kept: tau^-D/2 int_{box} G = tau^-D/2 c_D A_D, A_D the integral of Gamma_D
  over the unit box [-1/2, 1/2]^D (computed here by adaptive quadrature of
  the singular integrand).
* eq. SfromPhi: S = -tau log phi; grad S = -tau grad phi / phi and
  d_ab S = -tau d_ab phi / phi + S_a S_b / tau (the differentiation of eq.
  SfromPhi), with the derivative terms of a point on the node itself taken
  as zero (the value at the origin of an odd kernel, and the convention of
  Sec. 4.1 for the derivative kernels).

The sums are evaluated with the log-sum-exp shift of Sec. 2.4 (eq. Bound1):
phi = P exp(-z_min) sum_k Gs(z_k) exp(-(z_k - z_min)) with Gs = exp(z) Gamma.
"""
from __future__ import annotations

import functools

import numpy as np
import scipy.integrate as si
import scipy.special as sp

C_D = {1: 0.5, 2: 1.0 / (2.0 * np.pi), 3: 1.0 / (4.0 * np.pi)}


@functools.lru_cache(maxsize=None)
def origin_integral(D: int) -> float:
    """A_D = int_{[-1/2,1/2]^D} Gamma_D(|u|) du (D = 2, 3); Gamma_1(0) = 1."""
    if D == 1:
        return 1.0
    if D == 2:
        v, _ = si.dblquad(lambda y, x: sp.k0(np.hypot(x, y)), 0.0, 0.5, 0.0, 0.5,
                          epsabs=1e-14, epsrel=1e-13)
        return 4.0 * v

    def f(z, y, x):
        r = np.sqrt(x * x + y * y + z * z)
        return np.exp(-r) / r
    v, _ = si.tplquad(f, 0.0, 0.5, 0.0, 0.5, 0.0, 0.5, epsabs=1e-13, epsrel=1e-12)
    return 8.0 * v


def profile_scaled(D: int, z: np.ndarray):
    """exp(z) Gamma_D(z), exp(z) Gamma_D'(z), exp(z) Gamma_D''(z) for z > 0."""
    z = np.asarray(z, dtype=np.float64)
    if D == 1:
        one = np.ones_like(z)
        return one, -one, one
    if D == 2:
        k0, k1 = sp.k0e(z), sp.k1e(z)
        return k0, -k1, k0 + k1 / z   # K_0' = -K_1, K_0'' = K_0 + K_1 / z
    iz = 1.0 / z
    return iz, -iz * (1.0 + iz), iz * (1.0 + 2.0 * iz + 2.0 * iz * iz)


def profile(D: int, z):
    """Gamma_D(z), Gamma_D'(z), Gamma_D''(z) (z > 0)."""
    z = np.asarray(z, dtype=np.float64)
    e = np.exp(-z)
    a, b, c = profile_scaled(D, z)
    return a * e, b * e, c * e


def prefactor(D: int, tau: float) -> float:
    """P = tau^-D/2 c_D (eq. phiapproxSol with gamma = D/2)."""
    return tau ** (-0.5 * D) * C_D[D]


def phi(Y: np.ndarray, X: np.ndarray, tau: float) -> np.ndarray:
    """phi(X) = P sum_k Gamma_D(||X - Y_k|| / tau), unshifted (small cases)."""
    Y = np.atleast_2d(np.asarray(Y, dtype=np.float64))
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    D = X.shape[1]
    r = np.linalg.norm(X[:, None, :] - Y[None, :, :], axis=2)
    z = r / tau
    G = np.where(z > 0, profile(D, np.where(z > 0, z, 1.0))[0], origin_integral(D))
    return prefactor(D, tau) * G.sum(axis=1)


def evaluate(Y: np.ndarray, X: np.ndarray, tau: float, want=("S", "dS", "d2S"), chunk: int = 512):
    """S, grad S and the Hessian (xx, yy[, zz], xy[, xz, yz]) of the exact
    Green's function set at the nodes X (n x D) from the points Y (K x D; a
    point repeated m times counts m times)."""
    Y = np.asarray(Y, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    n, D = X.shape
    P = prefactor(D, tau)
    A = origin_integral(D)
    pairs = [(a, b) for a in range(D) for b in range(a + 1, D)]  # xy[, xz, yz]
    out = {"S": np.empty(n)}
    if "dS" in want or "d2S" in want:
        out["dS"] = np.empty((n, D))
    if "d2S" in want:
        out["d2S"] = np.empty((n, D + len(pairs)))
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        d = X[a:b, None, :] - Y[None, :, :]
        r = np.linalg.norm(d, axis=2)
        z = r / tau
        src = z == 0.0
        zs = np.where(src, 1.0, z)
        g0, g1, g2 = profile_scaled(D, zs)
        g0 = np.where(src, A, g0)
        g1 = np.where(src, 0.0, g1)
        g2 = np.where(src, 0.0, g2)
        zmin = z.min(axis=1, keepdims=True)
        w = np.exp(-(z - zmin))
        ps = (g0 * w).sum(axis=1)
        out["S"][a:b] = tau * zmin[:, 0] - tau * np.log(P) - tau * np.log(ps)
        if "dS" in out:
            nrm = d / np.where(src, 1.0, r)[:, :, None]
            nrm[src] = 0.0
            t1 = (g1 * w)[:, :, None] * nrm
            G = -t1.sum(axis=1) / ps[:, None]
            out["dS"][a:b] = G
        if "d2S" in out:
            rr = np.where(src, 1.0, r)
            cols = [(i, i) for i in range(D)] + pairs
            for c, (i, j) in enumerate(cols):
                nn = nrm[:, :, i] * nrm[:, :, j]
                dlt = 1.0 if i == j else 0.0
                term = (g2 * nn / tau + g1 * (dlt - nn) / rr) * w
                term[src] = 0.0
                out["d2S"][a:b, c] = -term.sum(axis=1) / ps + G[:, i] * G[:, j] / tau
    return out
