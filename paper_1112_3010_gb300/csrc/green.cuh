// green.cuh -- the exact Green's functions of -tau^2 lap phi + phi = psi
// (Sec. 2.1, eqs. GreensFunction1D/2D/3D) as an alternative kernel set.
//
// In the unit z = r/tau every one of them is P * Gamma_D(z):
//   G(X) = tau^-D c_D Gamma_D(||X||/tau),  c_1 = 1/2, c_2 = 1/(2 pi), c_3 = 1/(4 pi)
//   Gamma_1 = exp(-z),  Gamma_2 = K_0(z),  Gamma_3 = exp(-z)/z.
// The point-source field of Sec. 2.2, phi(X) = tau^-D/2 sum_k int_{B_k(X)} G,
// B_k the box of side tau around X - Y_k (psi_k = tau^-D/2 on it), is taken
// at its mid-point value tau^D G(X - Y_k) (eq. phiapproxSol with gamma = D/2):
//   g(o) = tau^-D/2 c_D Gamma_D(||o||/tau),  o != 0.
// At o = 0 the mid-point value is infinite for D >= 2; there g keeps the
// box integral itself, tau^-D/2 c_D A_D with A_D the integral of Gamma_D over
// the unit box [-1/2, 1/2]^D.  A_D follows from the divergence theorem applied
// to -lap Gamma + Gamma = delta / c_D over the unit box:
//   c_D A_D = 1 + c_D (flux of grad Gamma_D through the box's faces),
// an integral of a smooth function over the faces (Gauss-Legendre).
//
// K_0 and K_1 (2D): for z < 20 the trapezoidal rule on the integral
// representation K_nu(z) = int_0^inf exp(-z cosh t) cosh(nu t) dt (DLMF
// 10.32.9), scaled by exp(z), which converges geometrically in the step; for
// z >= 20 the large-argument expansion (DLMF 10.40.2) summed to its smallest
// term.
#pragma once
#include <math.h>

namespace sdf {

// exp(z) K_0(z) and exp(z) K_1(z), z > 0.
__host__ __device__ inline void bessel_k01_scaled(double z, double *k0e, double *k1e) {
    if (z >= 20.0) {
        // a_k(nu) = prod_{j=1..k} (4 nu^2 - (2j - 1)^2) / (k! 8^k)
        const double pre = sqrt(1.5707963267948966 / z);
        double t0 = 1.0, t1 = 1.0, s0 = 1.0, s1 = 1.0;
        for (int k = 1; k < 60; ++k) {
            const double o = (double)(2 * k - 1);
            const double n0 = (0.0 - o * o) / (k * 8.0 * z), n1 = (4.0 - o * o) / (k * 8.0 * z);
            if (fabs(n0) >= 1.0) break;  // past the smallest term
            t0 *= n0;
            t1 *= n1;
            s0 += t0;
            s1 += t1;
            if (fabs(t0) < 1e-18 && fabs(t1) < 1e-18) break;
        }
        *k0e = pre * s0;
        *k1e = pre * s1;
        return;
    }
    // trapezoid on t in [0, t_max], integrand exp(-z (cosh t - 1)) [cosh t]
    const double dt = 0.1;
    double a0 = 0.5, a1 = 0.5;  // t = 0 end point (weight 1/2)
    for (int j = 1; j < 400; ++j) {
        const double t = j * dt;
        const double c = cosh(t);
        const double x = z * (c - 1.0);
        if (x > 45.0) break;
        const double e = exp(-x);
        a0 += e;
        a1 += e * c;
    }
    *k0e = a0 * dt;
    *k1e = a1 * dt;
}

// Gamma_D(z), Gamma_D'(z), Gamma_D''(z) for z > 0.
__host__ __device__ inline void green_profile(int D, double z, double *g, double *g1, double *g2) {
    const double ez = exp(-z);
    if (D == 1) {
        *g = ez;
        *g1 = -ez;
        *g2 = ez;
    } else if (D == 2) {
        double k0e, k1e;
        bessel_k01_scaled(z, &k0e, &k1e);
        const double k0 = k0e * ez, k1 = k1e * ez;
        *g = k0;
        *g1 = -k1;                // K_0' = -K_1
        *g2 = k0 + k1 / z;        // from z^2 K'' + z K' - z^2 K = 0
    } else {
        const double G = ez / z;
        *g = G;
        *g1 = -G * (1.0 + 1.0 / z);
        *g2 = G * (1.0 + 2.0 / z + 2.0 / (z * z));
    }
}

// c_D of G = tau^-D c_D Gamma_D.
__host__ __device__ inline double green_cD(int D) {
    return D == 1 ? 0.5 : (D == 2 ? 0.15915494309189535 : 0.07957747154594767);
}

}  // namespace sdf
