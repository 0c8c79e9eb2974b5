// spectra.cu -- step A0 (plan time): sample every kernel on the padded grid
// and transform it (Table 1 steps 1 and 3 for f; the same for the kernels of
// Secs. 4 and 5), in FP64, then keep 1/2^D of the spectrum in the plan's
// precision.
//
// Sampling.  Node offset j_a along axis a is taken in [-(N_a-1), N_a-1]
// (wrap-around index j_a or j_a - M_a); every other index holds 0, since it
// never reaches an output node.  Offsets in world units o = j*h, r = ||o||,
// n = o/r, E = exp(-r/tau):
//   PHI  E                                         eq. function_f (f(0) = 1)
//   G_a  n_a E                                     eq. SxSyconv (f_c f, f_s f)
//   H_ab [(delta_ab - n_a n_b)/r - n_a n_b/tau] E  eqs. Sxx, Syy, Sxy
//   W    2D: o_2/r^2, o_1/r^2 (f_sr, f_cr of eq. fcfsfr); 3D: o_a/r^3 (eq. mudef)
//   RF   r E                                       (d/dtau of E, adjoint)
// All but PHI are 0 at the origin (Sec. 4.1 sets f_c(0) = f_s(0) = f_r(0) = 0).
//
// Exact Green's function kernel set (green.cuh): E above becomes
// g = P Gamma(z), z = r/tau, P = tau^-D/2 c_D, with the derivative kernels
// -tau d_a g and -tau d_ab g, so that the epilogue's grad S = G/phi and
// Hessian = H/phi - ... hold unchanged:
//   PHI  P Gamma(z)                   (P A_D at the origin)
//   G_a  -P Gamma'(z) n_a
//   H_ab -P [Gamma''(z) n_a n_b / tau + Gamma'(z) (delta_ab - n_a n_b) / r]
// The winding kernels do not depend on the kernel set.
//
// Symmetry.  A kernel odd along the axes in `parity` has a spectrum
// (-i)^popcount(parity) * c(k) with c real, even/odd per axis like the kernel.
// c is stored on fold(k_a) = min(k_a, M_a - k_a) in [0, M_a/2] with the 1/prod(M)
// of the inverse transform folded in, laid out for the fused pass:
// 2D [f0][f1] (f1 fastest), 3D [f1][f0][f2] (f2 fastest).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <cmath>
#include <vector>

#include "green.cuh"
#include "sdf_internal.cuh"

namespace sdf {

template <typename T>
cudaError_t fwd_T_launch(const typename cplx_t<T>::type *in, typename cplx_t<T>::type *out, int logL, int n_in,
                         int64_t n_lines, int nfield, int64_t in_fs, int64_t out_fs,
                         const typename cplx_t<T>::type *tw, cudaStream_t st, sdf_plan_impl *p);

struct SampleCfg {
    int D;
    int64_t M[3], N[3];
    double h, tau;
    int id;
    int kset;           // SDF_KERNEL_EXP or SDF_KERNEL_GREEN
    double gP, gA;      // Green set: P = tau^-D/2 c_D and A_D (Gamma at the origin)
};

__device__ double green_kernel_value(const SampleCfg &c, const double o[3], double r, double r2) {
    const int D = c.D;
    const double tau = c.tau;
    if (r == 0.0) return c.id == KER_PHI ? c.gP * c.gA : 0.0;
    const double n[3] = {o[0] / r, o[1] / r, D == 3 ? o[2] / r : 0.0};
    double g, g1, g2;
    green_profile(D, r / tau, &g, &g1, &g2);
    const double P = c.gP;
    auto hess = [&](int a, int b) {
        const double nn = n[a] * n[b];
        return -P * (g2 * nn / tau + g1 * ((a == b ? 1.0 : 0.0) - nn) / r);
    };
    switch (c.id) {
        case KER_PHI: return P * g;
        case KER_GX: return -P * g1 * n[0];
        case KER_GY: return -P * g1 * n[1];
        case KER_GZ: return -P * g1 * n[2];
        case KER_HXX: return hess(0, 0);
        case KER_HYY: return hess(1, 1);
        case KER_HZZ: return hess(2, 2);
        case KER_HXY: return hess(0, 1);
        case KER_HXZ: return hess(0, 2);
        case KER_HYZ: return hess(1, 2);
        case KER_W1: return D == 2 ? o[1] / r2 : o[0] / (r2 * r);
        case KER_W2: return D == 2 ? o[0] / r2 : o[1] / (r2 * r);
        case KER_W3: return o[2] / (r2 * r);
        default: return 0.0;  // no tau-derivative kernel for this set
    }
}

__device__ double kernel_value(const SampleCfg &c, const double o[3]) {
    const int D = c.D;
    double r2 = 0.0;
    for (int a = 0; a < D; ++a) r2 += o[a] * o[a];
    const double r = sqrt(r2);
    const double tau = c.tau;
    if (c.kset == SDF_KERNEL_GREEN) return green_kernel_value(c, o, r, r2);
    if (c.id == KER_PHI) return exp(-r / tau);
    if (r == 0.0) return 0.0;
    const double E = exp(-r / tau);
    double n[3] = {o[0] / r, o[1] / r, D == 3 ? o[2] / r : 0.0};
    switch (c.id) {
        case KER_GX: return n[0] * E;
        case KER_GY: return n[1] * E;
        case KER_GZ: return n[2] * E;
        case KER_HXX: return ((1.0 - n[0] * n[0]) / r - n[0] * n[0] / tau) * E;
        case KER_HYY: return ((1.0 - n[1] * n[1]) / r - n[1] * n[1] / tau) * E;
        case KER_HZZ: return ((1.0 - n[2] * n[2]) / r - n[2] * n[2] / tau) * E;
        case KER_HXY: return (-n[0] * n[1] / r - n[0] * n[1] / tau) * E;
        case KER_HXZ: return (-n[0] * n[2] / r - n[0] * n[2] / tau) * E;
        case KER_HYZ: return (-n[1] * n[2] / r - n[1] * n[2] / tau) * E;
        case KER_W1: return D == 2 ? o[1] / r2 : o[0] / (r2 * r);
        case KER_W2: return D == 2 ? o[0] / r2 : o[1] / (r2 * r);
        case KER_W3: return o[2] / (r2 * r);
        case KER_RF: return r * E;
        default: return 0.0;
    }
}

// Sample into a natural-layout M^D complex grid; per-block partial l1 sums.
__global__ void k_sample(SampleCfg c, double2 *out, double *part, int64_t total) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t rem = i;
        bool inside = true;
        double o[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < c.D; ++a) {
            const int64_t j = rem % c.M[a];
            rem /= c.M[a];
            int64_t off;
            if (j <= c.N[a] - 1) off = j;
            else if (j >= c.M[a] - (c.N[a] - 1)) off = j - c.M[a];
            else { inside = false; off = 0; }
            o[a] = (double)off * c.h;
        }
        const double v = inside ? kernel_value(c, o) : 0.0;
        out[i] = make_double2(v, 0.0);
        acc += fabs(v);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Compress: c(fold) = Re(Khat(fold) * conj(zeta)) * scale, zeta = (-i)^nodd.
template <typename T>
__global__ void k_compress(const double2 *__restrict__ K, T *c, int D, int64_t M0, int64_t M1, int64_t M2, int nodd,
                           double scale, double *resid, int64_t Hp) {
    const int64_t H0 = M0 / 2 + 1, H1 = M1 / 2 + 1, H2 = (D == 3) ? M2 / 2 + 1 : 1;
    const int64_t total = H0 * H1 * H2;
    double worst = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t f0, f1 = 0, f2 = 0, dst;
        if (D == 1) {
            f0 = i;
            dst = i;
        } else if (D == 2) {
            f1 = i % H1;
            f0 = i / H1;
            dst = f0 * Hp + f1;
        } else {
            f2 = i % H2;
            f0 = (i / H2) % H0;
            f1 = i / (H2 * H0);
            dst = (f1 * H0 + f0) * Hp + f2;
        }
        const double2 k = K[f0 + M0 * (f1 + M1 * f2)];
        // conj(zeta) for zeta = (-i)^nodd: (+i)^nodd
        double re, im;
        switch (nodd & 3) {
            case 0: re = k.x; im = k.y; break;
            case 1: re = -k.y; im = k.x; break;   // k * i
            case 2: re = -k.x; im = -k.y; break;  // k * -1
            default: re = k.y; im = -k.x; break;  // k * -i
        }
        c[dst] = (T)(re * scale);
        worst = fmax(worst, fabs(im * scale));
    }
    if (resid) {
        // record the largest discarded imaginary part (a consistency check)
        unsigned long long *r = reinterpret_cast<unsigned long long *>(resid);
        atomicMax(r, (unsigned long long)__double_as_longlong(worst));
    }
}

static int parity_of(int id, int D) {
    switch (id) {
        case KER_GX: return 1;
        case KER_GY: return 2;
        case KER_GZ: return 4;
        case KER_HXY: return 3;
        case KER_HXZ: return 5;
        case KER_HYZ: return 6;
        case KER_W1: return D == 2 ? 2 : 1;
        case KER_W2: return D == 2 ? 1 : 2;
        case KER_W3: return 4;
        default: return 0;
    }
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_n from the
// Chebyshev guesses).
static void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double t = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
            const double dt = p1 / dp;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        x[i] = t;
        w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

// A_D = integral of Gamma_D over [-1/2, 1/2]^D (green.cuh): c_D A_D = 1 minus
// the outward flux of -c_D grad Gamma_D through the 2D faces; on the face
// u_0 = 1/2, d Gamma/dn = Gamma'(r) / (2 r).  D = 1: Gamma_1(0) = 1.
double green_origin_integral(int D) {
    static double cache[4] = {0, 0, 0, 0};
    if (D < 2 || D > 3) return 1.0;
    if (cache[D] != 0.0) return cache[D];
    std::vector<double> x, w;
    gauss_legendre(48, x, w);
    double flux = 0.0;  // integral over one face of Gamma'(r) / (2 r)
    if (D == 2) {
        for (size_t i = 0; i < x.size(); ++i) {
            const double y = 0.5 * x[i], r = sqrt(0.25 + y * y);
            double g, g1, g2;
            green_profile(2, r, &g, &g1, &g2);
            flux += 0.5 * w[i] * g1 / (2.0 * r);
        }
    } else {
        for (size_t i = 0; i < x.size(); ++i)
            for (size_t j = 0; j < x.size(); ++j) {
                const double y = 0.5 * x[i], z = 0.5 * x[j], r = sqrt(0.25 + y * y + z * z);
                double g, g1, g2;
                green_profile(3, r, &g, &g1, &g2);
                flux += 0.25 * w[i] * w[j] * g1 / (2.0 * r);
            }
    }
    const double cA = 1.0 + green_cD(D) * 2.0 * D * flux;
    cache[D] = cA / green_cD(D);
    return cache[D];
}

cudaError_t build_spectra(sdf_plan_impl *p) {
    cudaError_t e;
    const int D = p->D;
    cudaStream_t st = p->stream;
    int64_t total = 1;
    for (int a = 0; a < D; ++a) total *= p->M[a];
    // FP64 twiddle tables for the plan-time transforms
    std::vector<double2 *> tw64(D, nullptr);
    double2 *bufX = nullptr, *bufY = nullptr;
    double *part = nullptr, *resid = nullptr;
    auto release = [&]() {
        cudaFree(bufX);
        cudaFree(bufY);
        cudaFree(part);
        for (auto t : tw64) cudaFree(t);
    };
    for (int a = 0; a < D; ++a) {
        const int64_t L = p->M[a];
        std::vector<double2> h(L);
        fill_twiddle_table(line_code(L), h.data());
        if ((e = dev_alloc((void **)&tw64[a], sizeof(double2) * L)) != cudaSuccess ||
            (e = cudaMemcpy(tw64[a], h.data(), sizeof(double2) * L, cudaMemcpyHostToDevice)) != cudaSuccess) {
            release();
            return e;
        }
    }
    const int nblk = 1024;
    if ((e = dev_alloc((void **)&bufX, sizeof(double2) * total)) != cudaSuccess ||
        (e = dev_alloc((void **)&bufY, sizeof(double2) * total)) != cudaSuccess ||
        (e = dev_alloc((void **)&part, sizeof(double) * (nblk + 1))) != cudaSuccess) {
        release();
        return e;
    }
    resid = part + nblk;
    std::vector<double> hpart(nblk);
    double inv_n = 1.0 / (double)total;
    const int64_t H0 = p->M[0] / 2 + 1, H1 = p->M[1] / 2 + 1, H2 = (D == 3) ? p->M[2] / 2 + 1 : 1;
    const int64_t ctotal = spec_rows(p) * spec_row_len(p);
    (void)H0;
    (void)H1;
    (void)H2;
    const size_t esz = (p->prec == SDF_FP64) ? sizeof(double) : sizeof(float);
    for (auto &ks : p->kernels) {
        SampleCfg c;
        c.D = D;
        for (int a = 0; a < 3; ++a) {
            c.M[a] = p->M[a];
            c.N[a] = p->N[a];
        }
        c.h = p->h;
        c.tau = p->tau;
        c.id = ks.id;
        c.kset = p->kernel_set;
        c.gP = pow(p->tau, -0.5 * D) * green_cD(D);
        c.gA = green_origin_integral(D);
        k_sample<<<nblk, 256, 0, st>>>(c, bufX, part, total);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        // D forward passes, each along the fastest axis with a rotating layout
        double2 *src = bufX, *dst = bufY;
        for (int a = 0; a < D; ++a) {
            const int64_t L = p->M[a];
            const int64_t n_lines = total / L;
            if ((e = fwd_T_launch<double>(src, dst, p->logM[a], (int)L, n_lines, 1, 0, 0, tw64[a], st, nullptr)) !=
                cudaSuccess)
                break;
            std::swap(src, dst);
        }
        if (e != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(hpart.data(), part, sizeof(double) * nblk, cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess)
            break;
        if ((e = cudaMemsetAsync(resid, 0, sizeof(double), st)) != cudaSuccess) break;
        const int nodd = __builtin_popcount((unsigned)ks.parity);
        double scale = inv_n * ks.scale;
        if ((e = dev_alloc(&ks.c, esz * ctotal)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(ks.c, 0, esz * ctotal, st)) != cudaSuccess) break;
        if (p->prec == SDF_FP64)
            k_compress<double><<<1024, 256, 0, st>>>(src, reinterpret_cast<double *>(ks.c), D, p->M[0], p->M[1],
                                                     p->M[2], nodd, scale, resid, spec_row_len(p));
        else
            k_compress<float><<<1024, 256, 0, st>>>(src, reinterpret_cast<float *>(ks.c), D, p->M[0], p->M[1],
                                                    p->M[2], nodd, scale, resid, spec_row_len(p));
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
        double l1 = 0.0;
        for (int i = 0; i < nblk; ++i) l1 += hpart[i];
        ks.l1 = l1;
        p->workspace_bytes += esz * ctotal;
    }
    release();
    return e;
}

int kernel_parity(int id, int D) { return parity_of(id, D); }

// The same sampling, FP64 transform and compression as build_spectra, into
// memory the caller provides: bufX and bufY (prod(M) double2 each), part
// (kSpectraParts doubles), tw64[a] (M_a double2, already filled) and each
// p->kernels[i].c (compressed spectrum).  host_part receives kSpectraParts
// doubles.  Allocates nothing; synchronises the stream once per kernel.
cudaError_t build_spectra_into(sdf_plan_impl *p, double2 *bufX, double2 *bufY, double *part, double *host_part,
                               double2 *const *tw64) {
    cudaError_t e = cudaSuccess;
    const int D = p->D;
    cudaStream_t st = p->stream;
    int64_t total = 1;
    for (int a = 0; a < D; ++a) total *= p->M[a];
    const int nblk = kSpectraParts;
    const double inv_n = 1.0 / (double)total;
    for (auto &ks : p->kernels) {
        SampleCfg c;
        c.D = D;
        for (int a = 0; a < 3; ++a) {
            c.M[a] = p->M[a];
            c.N[a] = p->N[a];
        }
        c.h = p->h;
        c.tau = p->tau;
        c.id = ks.id;
        c.kset = p->kernel_set;
        c.gP = pow(p->tau, -0.5 * D) * green_cD(D);
        c.gA = green_origin_integral(D);
        k_sample<<<nblk, 256, 0, st>>>(c, bufX, part, total);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        double2 *src = bufX, *dst = bufY;
        for (int a = 0; a < D; ++a) {
            const int64_t L = p->M[a];
            if ((e = fwd_T_launch<double>(src, dst, p->logM[a], (int)L, total / L, 1, 0, 0, tw64[a], st,
                                          nullptr)) != cudaSuccess)
                return e;
            std::swap(src, dst);
        }
        if ((e = cudaMemcpyAsync(host_part, part, sizeof(double) * nblk, cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess)
            return e;
        const int nodd = __builtin_popcount((unsigned)ks.parity);
        const double scale = inv_n * ks.scale;
        if (p->prec == SDF_FP64)
            k_compress<double><<<1024, 256, 0, st>>>(src, reinterpret_cast<double *>(ks.c), D, p->M[0], p->M[1],
                                                     p->M[2], nodd, scale, nullptr, spec_row_len(p));
        else
            k_compress<float><<<1024, 256, 0, st>>>(src, reinterpret_cast<float *>(ks.c), D, p->M[0], p->M[1],
                                                    p->M[2], nodd, scale, nullptr, spec_row_len(p));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
        double l1 = 0.0;
        for (int i = 0; i < nblk; ++i) l1 += host_part[i];
        ks.l1 = l1;
    }
    return e;
}

}  // namespace sdf
