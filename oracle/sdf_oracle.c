/*
 * sdf_oracle.c -- plain FP64 CPU oracle for the convolution-based signed
 * distance method of Gurumoorthy & Rangarajan ("Fast convolution based method
 * for computing the signed distance function and its derivatives").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file: it is built and used by tests/, by __graft_entry__.smoke() and by
 * the cpu_baseline leg of bench.py, to check the CUDA path against the
 * definitions the paper gives.  It shares no code with the CUDA library.
 *
 * Everything here is a direct sum over the source points, written the way the
 * paper states each quantity, in double precision, with no blocking, fusion or
 * FFT.  The only numerical device is the log-sum-exp shift of Sec. 2.4
 * (eq. Bound1): S = R - tau*log(sum_k exp(-(r_k - R)/tau)), which is the same
 * number as eq. STilde but does not underflow far from the points.
 *
 * Functions:
 *   oracle_snap     -- rounding of points to the nearest grid node (Sec. 6,
 *                      Examples 3 and 4: "rounded the point cloud to the
 *                      nearest grid points").
 *   oracle_eval     -- S (eq. STilde), grad S (eq. SxSy), Hessian (eqs. Sxx,
 *                      Syy, Sxy in 2D; the same differentiation in 3D), the
 *                      winding number (eq. kappdiscreteZ, 2D) or topological
 *                      degree (eq. normflux, 3D), and R = min_k ||X - Y_k||
 *                      (eq. Rdef), at arbitrary real evaluation points X.
 *   oracle_adjoint  -- dL/dY_k and dL/dtau for L = sum_X w(X) S(X), obtained
 *                      by differentiating eq. STilde with respect to Y_k and
 *                      tau (the paper does not state these; the derivation is
 *                      the chain rule applied to eq. STilde).
 *
 * Conventions (readings of the paper):
 *   - Kernels that are singular at the origin (f_c, f_s, f_r and their
 *     products, Sec. 4.1, and the normal-flux kernel X/||X||^3) are set to 0
 *     there, as Sec. 4.1 states for f_c, f_s, f_r.  The same convention is
 *     used for the gradient and Hessian terms of a point with r_k = 0, which
 *     is what the convolution kernels f_c*f and the Hessian kernels of Sec. 5
 *     give at the origin.  The S kernel f(0) = exp(0) = 1.
 *   - Hessian component order: 2D (xx, yy, xy); 3D (xx, yy, zz, xy, xz, yz).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Nearest-node rounding of each coordinate: j = floor(y/h + 0.5) (ties go up).
 * Y is K x D (row-major), dims[a] = N_a.  idx receives K x D node indices.
 * Returns the number of points whose node falls outside [0, N_a) on some axis
 * (their indices are still written).
 */
int64_t oracle_snap(int D, int64_t K, const double *Y, double h,
                    const int64_t *dims, int64_t *idx) {
    int64_t bad = 0;
    for (int64_t k = 0; k < K; ++k) {
        int out = 0;
        for (int a = 0; a < D; ++a) {
            double q = floor(Y[k * D + a] / h + 0.5);
            int64_t j = (int64_t)q;
            idx[k * D + a] = j;
            if (j < 0 || j >= dims[a]) out = 1;
        }
        bad += out;
    }
    return bad;
}

/*
 * Direct evaluation at nX points X (nX x D, row-major).  Y: K x D source
 * points.  W: K x D tangents Z_k (2D, eq. tangentVec) or normals P_k (3D,
 * eq. normflux), may be NULL.  tau > 0.
 * Outputs (each may be NULL):
 *   S[nX]          eq. STilde (via the log-sum-exp form of eq. Bound1)
 *   dS[nX*D]       eq. SxSy:  S_i = sum_k n_ki E_k / sum_k E_k,
 *                  n_k = (X - Y_k)/r_k
 *   d2S[nX*D(D+1)/2]
 *                  H_ij = sum_k w_k [(delta_ij - n_ki n_kj)/r_k - n_ki n_kj/tau]
 *                         + S_i S_j / tau,  w_k = E_k / sum_l E_l
 *                  (2D: eqs. Sxx, Syy, Sxy written per point)
 *   mu[nX]         2D eq. kappdiscreteZ, 3D eq. normflux
 *   R[nX]          eq. Rdef
 *   logphi[nX]     log(sum_k exp(-r_k/tau)) = -S/tau
 */
void oracle_eval(int D, int64_t K, const double *Y, const double *W,
                 int64_t nX, const double *X, double tau,
                 double *S, double *dS, double *d2S, double *mu, double *R,
                 double *logphi) {
    const int nH = D * (D + 1) / 2;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nX; ++i) {
        const double *x = X + i * D;
        /* R(X) = min_k ||X - Y_k||  (eq. Rdef) */
        double Rmin = INFINITY;
        for (int64_t k = 0; k < K; ++k) {
            double s = 0.0;
            for (int a = 0; a < D; ++a) {
                double d = x[a] - Y[k * D + a];
                s += d * d;
            }
            double r = sqrt(s);
            if (r < Rmin) Rmin = r;
        }
        /* phi(X) exp(R/tau) = sum_k exp(-(r_k - R)/tau), and the weighted sums
           that give the derivatives (Sec. 5). */
        double sumE = 0.0;
        double g[3] = {0.0, 0.0, 0.0};
        double hk[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        double mus = 0.0;
        for (int64_t k = 0; k < K; ++k) {
            double d[3] = {0.0, 0.0, 0.0};
            double s = 0.0;
            for (int a = 0; a < D; ++a) {
                d[a] = x[a] - Y[k * D + a];
                s += d[a] * d[a];
            }
            double r = sqrt(s);
            double E = exp(-(r - Rmin) / tau);
            sumE += E;
            if (r > 0.0) {
                double n[3] = {d[0] / r, d[1] / r, D == 3 ? d[2] / r : 0.0};
                for (int a = 0; a < D; ++a) g[a] += n[a] * E;
                if (d2S) {
                    /* [(delta_ij - n_i n_j)/r - n_i n_j / tau] E_k */
                    int c = 0;
                    for (int a = 0; a < D; ++a, ++c)
                        hk[c] += ((1.0 - n[a] * n[a]) / r - n[a] * n[a] / tau) * E;
                    for (int a = 0; a < D; ++a)
                        for (int b = a + 1; b < D; ++b, ++c)
                            hk[c] += (-n[a] * n[b] / r - n[a] * n[b] / tau) * E;
                }
                if (W && mu) {
                    /* the vector Y_k - X enters both sign formulas */
                    double yx[3] = {-d[0], -d[1], D == 3 ? -d[2] : 0.0};
                    const double *w = W + k * D;
                    if (D == 2) {
                        /* eq. kappdiscreteZ */
                        mus += (yx[0] * w[1] - yx[1] * w[0]) / s;
                    } else {
                        /* eq. normflux */
                        mus += (yx[0] * w[0] + yx[1] * w[1] + yx[2] * w[2]) / (s * r);
                    }
                }
            }
        }
        double Si = Rmin - tau * log(sumE);
        double grad[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < D; ++a) grad[a] = g[a] / sumE;
        if (S) S[i] = Si;
        if (logphi) logphi[i] = -Si / tau;
        if (R) R[i] = Rmin;
        if (dS)
            for (int a = 0; a < D; ++a) dS[i * D + a] = grad[a];
        if (d2S) {
            int c = 0;
            for (int a = 0; a < D; ++a, ++c)
                d2S[i * nH + c] = hk[c] / sumE + grad[a] * grad[a] / tau;
            for (int a = 0; a < D; ++a)
                for (int b = a + 1; b < D; ++b, ++c)
                    d2S[i * nH + c] = hk[c] / sumE + grad[a] * grad[b] / tau;
        }
        if (mu && W)
            mu[i] = (D == 2) ? mus / (2.0 * ORACLE_PI) : mus / (4.0 * ORACLE_PI);
    }
}

/*
 * Gradient of L = sum_X w(X) S(X) with respect to the source points and tau,
 * for S of eq. STilde at continuous Y:
 *   dS(X)/dY_k  = -w_k(X) n_k(X),   w_k = E_k/sum E,  n_k = (X - Y_k)/r_k
 *   dS(X)/dtau  = S(X)/tau - (1/tau) sum_k w_k(X) r_k(X)
 * so dL/dY_k = -sum_X w(X) w_k(X) n_k(X) and
 *    dL/dtau = sum_X w(X) [S(X) - sum_k w_k r_k] / tau.
 * A term with r_k = 0 contributes no direction (n_k := 0, as in Sec. 4.1).
 * X: nX x D evaluation points; wX: nX loss weights.  dLdY: K x D output.
 */
void oracle_adjoint(int D, int64_t K, const double *Y, int64_t nX,
                    const double *X, const double *wX, double tau,
                    double *dLdY, double *dLdtau) {
    double *Rm = (double *)malloc(sizeof(double) * (size_t)nX);
    double *Sx = (double *)malloc(sizeof(double) * (size_t)nX);
    double *wr = (double *)malloc(sizeof(double) * (size_t)nX);
    /* pass 1: R(X), S(X) and the weighted mean distance at every X */
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nX; ++i) {
        const double *x = X + i * D;
        double Rmin = INFINITY;
        for (int64_t k = 0; k < K; ++k) {
            double s = 0.0;
            for (int a = 0; a < D; ++a) {
                double d = x[a] - Y[k * D + a];
                s += d * d;
            }
            double r = sqrt(s);
            if (r < Rmin) Rmin = r;
        }
        double sumE = 0.0, sumEr = 0.0;
        for (int64_t k = 0; k < K; ++k) {
            double s = 0.0;
            for (int a = 0; a < D; ++a) {
                double d = x[a] - Y[k * D + a];
                s += d * d;
            }
            double r = sqrt(s);
            double E = exp(-(r - Rmin) / tau);
            sumE += E;
            sumEr += E * r;
        }
        Rm[i] = Rmin;
        Sx[i] = Rmin - tau * log(sumE);
        wr[i] = sumEr / sumE;
    }
    /* pass 2: one source at a time, sum over X */
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < K; ++k) {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int64_t i = 0; i < nX; ++i) {
            if (wX[i] == 0.0) continue;
            const double *x = X + i * D;
            double d[3] = {0.0, 0.0, 0.0};
            double s = 0.0;
            for (int a = 0; a < D; ++a) {
                d[a] = x[a] - Y[k * D + a];
                s += d[a] * d[a];
            }
            double r = sqrt(s);
            if (r == 0.0) continue;
            /* w_k(X) = E_k/sum E = exp(-(r_k - S(X))/tau) */
            double wk = exp(-(r - Sx[i]) / tau);
            for (int a = 0; a < D; ++a) acc[a] -= wX[i] * wk * d[a] / r;
        }
        for (int a = 0; a < D; ++a) dLdY[k * D + a] = acc[a];
    }
    double t = 0.0;
    for (int64_t i = 0; i < nX; ++i) t += wX[i] * (Sx[i] - wr[i]);
    *dLdtau = t / tau;
    (void)Rm;
    free(Rm);
    free(Sx);
    free(wr);
}

/*
 * oracle_curvature -- curvature fields from grad S and the Hessian at nX
 * points (Sec. 5: from the derivatives one obtains "derived quantities such as
 * curvature (Gaussian, mean and principal curvatures)" of the surface S(X)).
 *   2D: the surface is the graph z = S(x, y) (a Monge patch, upward normal),
 *       W = 1 + S_x^2 + S_y^2:
 *         K = (S_xx S_yy - S_xy^2) / W^2
 *         H = ((1 + S_y^2) S_xx - 2 S_x S_y S_xy + (1 + S_x^2) S_yy) / (2 W^{3/2})
 *   3D: the paper is silent; read as the level surfaces of S, normal
 *       n = grad S/|grad S|, g = |grad S|:
 *         H = (g^2 tr(Hess) - grad S^T Hess grad S) / (2 g^3)
 *         K = grad S^T adj(Hess) grad S / g^4   (adj: the adjugate matrix)
 *       and 0 where g = 0.
 *   Principal curvatures k1 >= k2: H +- sqrt(max(H^2 - K, 0)).
 * dS: nX x D, d2S: nX x D(D+1)/2 (xx, yy[, zz], xy[, xz, yz]);
 * out: nX x 4 (K, H, k1, k2).
 */
void oracle_curvature(int D, int64_t nX, const double *dS, const double *d2S, double *out) {
    const int nH = D * (D + 1) / 2;
    for (int64_t i = 0; i < nX; ++i) {
        const double *g = dS + i * D, *h = d2S + i * nH;
        double K = 0.0, H = 0.0;
        if (D == 2) {
            const double sx = g[0], sy = g[1], sxx = h[0], syy = h[1], sxy = h[2];
            const double W = 1.0 + sx * sx + sy * sy;
            K = (sxx * syy - sxy * sxy) / (W * W);
            H = ((1.0 + sy * sy) * sxx - 2.0 * sx * sy * sxy + (1.0 + sx * sx) * syy) / (2.0 * pow(W, 1.5));
        } else {
            const double sx = g[0], sy = g[1], sz = g[2];
            const double a = h[0], b = h[1], c = h[2], d = h[3], e = h[4], f = h[5];
            const double g2 = sx * sx + sy * sy + sz * sz;
            if (g2 > 0.0) {
                const double gn = sqrt(g2);
                /* grad S^T Hess grad S */
                const double gHg = sx * (a * sx + d * sy + e * sz) + sy * (d * sx + b * sy + f * sz) +
                                   sz * (e * sx + f * sy + c * sz);
                H = (g2 * (a + b + c) - gHg) / (2.0 * g2 * gn);
                /* grad S^T adj(Hess) grad S, adj of [[a,d,e],[d,b,f],[e,f,c]] */
                const double gAg = sx * sx * (b * c - f * f) + sy * sy * (a * c - e * e) + sz * sz * (a * b - d * d) +
                                   2.0 * sx * sy * (e * f - c * d) + 2.0 * sx * sz * (d * f - b * e) +
                                   2.0 * sy * sz * (d * e - a * f);
                K = gAg / (g2 * g2);
            }
        }
        const double disc = H * H - K;
        const double sq = disc > 0.0 ? sqrt(disc) : 0.0;
        out[i * 4 + 0] = K;
        out[i * 4 + 1] = H;
        out[i * 4 + 2] = H + sq;
        out[i * 4 + 3] = H - sq;
    }
}

/*
 * oracle_mesh_sources -- point sources of a triangle mesh for the 3D degree
 * (Sec. 4.2 and Example 5): Y_k = the incentre of triangle k (vertices A, B,
 * C weighted by the opposite side lengths), P_k = (B - A) x (C - A) / 2, the
 * edge cross product scaled to the triangle's area (area-weighted normal).
 * If center != NULL, P_k is negated where <Y_k - center, P_k> < 0 (the
 * orientation rule of Example 5, with the object's centre as origin);
 * otherwise the faces' vertex order orients P_k.
 * V: nv x 3, F: nf x 3 vertex indices; Y, P: nf x 3.
 */
void oracle_mesh_sources(int64_t nf, const double *V, const int64_t *F, const double *center, double *Y, double *P) {
    for (int64_t k = 0; k < nf; ++k) {
        const double *A = V + 3 * F[3 * k], *B = V + 3 * F[3 * k + 1], *C = V + 3 * F[3 * k + 2];
        double ab[3], ac[3], bc[3];
        for (int a = 0; a < 3; ++a) {
            ab[a] = B[a] - A[a];
            ac[a] = C[a] - A[a];
            bc[a] = C[a] - B[a];
        }
        const double la = sqrt(bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]); /* opposite A */
        const double lb = sqrt(ac[0] * ac[0] + ac[1] * ac[1] + ac[2] * ac[2]); /* opposite B */
        const double lc = sqrt(ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2]); /* opposite C */
        const double sum = la + lb + lc;
        for (int a = 0; a < 3; ++a) Y[3 * k + a] = (la * A[a] + lb * B[a] + lc * C[a]) / sum;
        double n[3] = {0.5 * (ab[1] * ac[2] - ab[2] * ac[1]), 0.5 * (ab[2] * ac[0] - ab[0] * ac[2]),
                       0.5 * (ab[0] * ac[1] - ab[1] * ac[0])};
        if (center) {
            double dot = 0.0;
            for (int a = 0; a < 3; ++a) dot += (Y[3 * k + a] - center[a]) * n[a];
            if (dot < 0.0)
                for (int a = 0; a < 3; ++a) n[a] = -n[a];
        }
        for (int a = 0; a < 3; ++a) P[3 * k + a] = n[a];
    }
}

/*
 * oracle_solid_angle_degree -- the exact degree of a closed oriented triangle
 * mesh about each evaluation point: (1/4 pi) sum_k Omega_k(X), Omega_k the
 * signed solid angle of triangle k seen from X (Van Oosterom and Strackee's
 * formula: tan(Omega/2) = a.(b x c) / (|a||b||c| + (a.b)|c| + (a.c)|b| +
 * (b.c)|a|), a, b, c the vertices relative to X).  1 inside a closed
 * outward-oriented surface, 0 outside (a textbook check for the normalized
 * flux of Sec. 4.2).
 */
void oracle_solid_angle_degree(int64_t nf, const double *V, const int64_t *F, int64_t nX, const double *X,
                               double *deg) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nX; ++i) {
        const double *x = X + 3 * i;
        double tot = 0.0;
        for (int64_t k = 0; k < nf; ++k) {
            double p[3][3], l[3];
            for (int v = 0; v < 3; ++v) {
                const double *q = V + 3 * F[3 * k + v];
                for (int a = 0; a < 3; ++a) p[v][a] = q[a] - x[a];
                l[v] = sqrt(p[v][0] * p[v][0] + p[v][1] * p[v][1] + p[v][2] * p[v][2]);
            }
            const double triple = p[0][0] * (p[1][1] * p[2][2] - p[1][2] * p[2][1]) -
                                  p[0][1] * (p[1][0] * p[2][2] - p[1][2] * p[2][0]) +
                                  p[0][2] * (p[1][0] * p[2][1] - p[1][1] * p[2][0]);
            const double d01 = p[0][0] * p[1][0] + p[0][1] * p[1][1] + p[0][2] * p[1][2];
            const double d02 = p[0][0] * p[2][0] + p[0][1] * p[2][1] + p[0][2] * p[2][2];
            const double d12 = p[1][0] * p[2][0] + p[1][1] * p[2][1] + p[1][2] * p[2][2];
            const double den = l[0] * l[1] * l[2] + d01 * l[2] + d02 * l[1] + d12 * l[0];
            tot += 2.0 * atan2(triple, den);
        }
        deg[i] = tot / (4.0 * ORACLE_PI);
    }
}
