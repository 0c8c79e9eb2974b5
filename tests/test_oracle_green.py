"""Pins for the oracle of the exact Green's function kernel set (oracle/green.py).

Each test checks the oracle against a fact fixed independently of its code:
the unit mass of the Green's function, the screened Poisson equation it
solves, the divergence theorem on the unit box, finite differences, repeated
points, and the tau -> 0 limit the paper proves (App. A).
"""
import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp

from oracle import green

SPHERE_AREA = {1: 2.0, 2: 2.0 * np.pi, 3: 4.0 * np.pi}


@pytest.mark.parametrize("D", [1, 2, 3])
def test_unit_mass(D):
    """The Green's function of -tau^2 lap + 1 integrates to 1 over R^D (its
    Fourier transform at k = 0): c_D |S^{D-1}| int_0^inf Gamma_D(z) z^{D-1} dz = 1."""
    f = lambda z: green.profile(D, z)[0] * z ** (D - 1)
    v = si.quad(f, 0.0, 1.0, limit=200)[0] + si.quad(f, 1.0, np.inf, limit=200)[0]
    assert abs(green.C_D[D] * SPHERE_AREA[D] * v - 1.0) < 1e-10


@pytest.mark.parametrize("D", [2, 3])
def test_screened_poisson_equation(D):
    """phi of a few points solves -tau^2 lap phi + phi = 0 away from them (Sec. 2,
    eq. phiEquationwithtau with psi = 0 there); finite-difference Laplacian.
    The exp(-r/tau) kernel would leave a residual of order tau/r."""
    rng = np.random.default_rng(3)
    tau = 0.05
    Y = rng.uniform(0.3, 0.7, (4, D))
    X = rng.uniform(0.0, 1.0, (20, D))
    X = X[np.min(np.linalg.norm(X[:, None] - Y[None], axis=2), axis=1) > 2 * tau]
    dlt = 1e-3 * tau
    for x in X:
        p0 = green.phi(Y, x[None], tau)[0]
        lap = 0.0
        for a in range(D):
            e = np.zeros(D)
            e[a] = dlt
            lap += (green.phi(Y, (x + e)[None], tau)[0] - 2 * p0 + green.phi(Y, (x - e)[None], tau)[0]) / dlt ** 2
        assert abs(-tau ** 2 * lap + p0) <= 1e-5 * p0
        # the same residual for exp(-r/tau) is far from zero
        r = np.linalg.norm(x - Y, axis=1)
        E = np.exp(-r / tau)
        lapE = np.sum(E * (1 / tau ** 2 - (D - 1) / (tau * r)))
        assert abs(-tau ** 2 * lapE + E.sum()) > 1e-3 * E.sum()


@pytest.mark.parametrize("D", [2, 3])
def test_origin_integral_divergence_theorem(D):
    """int_B Gamma = 1/c_D + int_{dB} dGamma/dn over the unit box B (Gauss on
    -lap Gamma + Gamma = delta/c_D); on a face dGamma/dn = Gamma'(r)/(2r)."""
    if D == 2:
        flux = si.quad(lambda y: -sp.k1(np.hypot(0.5, y)) / (2 * np.hypot(0.5, y)), -0.5, 0.5,
                       epsabs=1e-15)[0]
    else:
        def f(z, y):
            r = np.sqrt(0.25 + y * y + z * z)
            return -np.exp(-r) * (1 + r) / r ** 2 / (2 * r)
        flux = si.dblquad(f, -0.5, 0.5, -0.5, 0.5, epsabs=1e-14)[0]
    ref = 1.0 / green.C_D[D] + 2 * D * flux
    assert abs(green.origin_integral(D) - ref) < 1e-10 * ref


@pytest.mark.parametrize("D", [2, 3])
def test_derivatives_match_finite_differences(D):
    rng = np.random.default_rng(7)
    tau = 0.03
    Y = rng.uniform(0.2, 0.8, (60, D))
    X = rng.uniform(0.0, 1.0, (15, D))
    o = green.evaluate(Y, X, tau)
    dlt = 1e-5
    pairs = [(a, a) for a in range(D)] + [(a, b) for a in range(D) for b in range(a + 1, D)]
    for a in range(D):
        e = np.zeros(D)
        e[a] = dlt
        p, m = green.evaluate(Y, X + e, tau), green.evaluate(Y, X - e, tau)
        np.testing.assert_allclose(o["dS"][:, a], (p["S"] - m["S"]) / (2 * dlt), atol=1e-6)
        for c, (i, j) in enumerate(pairs):
            if i == a:
                np.testing.assert_allclose(o["d2S"][:, c], (p["dS"][:, j] - m["dS"][:, j]) / (2 * dlt),
                                           atol=1e-5 / tau, rtol=1e-5)
            if j == a:
                np.testing.assert_allclose(o["d2S"][:, c], (p["dS"][:, i] - m["dS"][:, i]) / (2 * dlt),
                                           atol=1e-5 / tau, rtol=1e-5)


@pytest.mark.parametrize("D", [2, 3])
def test_single_point_and_multiplicity(D):
    """K = 1: S = -tau log(tau^-D/2 c_D Gamma_D(r/tau)) with Gamma from the
    unscaled Bessel / exponential routines; m coincident points lower S by
    exactly tau log m; on the point itself phi = tau^-D/2 c_D A_D."""
    rng = np.random.default_rng(11)
    tau = 0.02
    Y = rng.uniform(0.3, 0.7, (1, D))
    X = rng.uniform(0.0, 1.0, (30, D))
    r = np.linalg.norm(X - Y, axis=1)
    gam = sp.k0(r / tau) if D == 2 else np.exp(-r / tau) / (r / tau)
    ref = -tau * np.log(tau ** (-D / 2) * green.C_D[D] * gam)
    o1 = green.evaluate(Y, X, tau, want=("S",))
    np.testing.assert_allclose(o1["S"], ref, rtol=1e-12, atol=1e-14)
    o5 = green.evaluate(np.repeat(Y, 5, axis=0), X, tau, want=("S", "dS"))
    np.testing.assert_allclose(o5["S"], ref - tau * np.log(5), rtol=1e-12, atol=1e-14)
    on = green.evaluate(Y, Y, tau)
    assert abs(on["S"][0] + tau * np.log(tau ** (-D / 2) * green.C_D[D] * green.origin_integral(D))) < 1e-14
    assert np.all(on["dS"] == 0)


@pytest.mark.parametrize("D", [2, 3])
def test_tends_to_distance(D):
    """App. A: S -> R as tau -> 0 (here max |S - R| over nodes off the points
    shrinks with tau and ends below a few tau log(1/tau))."""
    rng = np.random.default_rng(5)
    Y = rng.uniform(0.3, 0.7, (40, D))
    X = rng.uniform(0.0, 1.0, (200, D))
    R = np.min(np.linalg.norm(X[:, None] - Y[None], axis=2), axis=1)
    errs = []
    for tau in (0.02, 0.005, 0.00125, 0.0003):
        errs.append(np.max(np.abs(green.evaluate(Y, X, tau, want=("S",))["S"] - R)))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 4 * 0.0003 * np.log(1 / 0.0003)


def test_1d_green_is_exp_up_to_a_constant():
    """In 1D the Green's function is (1/2tau) exp(-|x|/tau) (eq.
    GreensFunction1D): with the tau^1/2 of eq. phiapproxSol the set differs
    from exp(-r/tau) only by S_G = S - tau log(tau^-1/2 / 2), derivatives equal."""
    import oracle
    rng = np.random.default_rng(2)
    Y = rng.uniform(0.2, 0.8, (30, 1))
    X = rng.uniform(0.0, 1.0, (80, 1))
    tau = 0.01
    e = oracle.evaluate(Y, X, tau, want=("S", "dS", "d2S"))
    g = green.evaluate(Y, X, tau)
    np.testing.assert_allclose(g["S"], e["S"] - tau * np.log(tau ** -0.5 / 2), atol=1e-14)
    np.testing.assert_allclose(g["dS"], e["dS"], atol=1e-13)
    np.testing.assert_allclose(g["d2S"], e["d2S"], atol=1e-9 / tau)
