// adjoint.cu -- step A7: gradient of L = sum_X w(X) S(X) (unsigned S) with
// respect to the points and tau.  The paper gives no adjoint; it is the chain
// rule applied to eq. STilde:
//   dS(X)/dY_k = -(E_k/phi) n_k,  n_k = (X - Y_k)/r_k,  E_k = exp(-r_k/tau)
//   dS(X)/dtau = S/tau - (1/tau) sum_k (E_k/phi) r_k
// With a = w/phi these become convolutions evaluated at the points:
//   dL/dY_k = (a * k_grad)(Y_k),   k_grad(X) = f(X) X/||X||  (eq. SxSyconv's kernels)
//   dL/dtau = ( sum_X w S - sum_k (a * (||X|| f))(Y_k) ) / tau
// so one forward transform of a, two packed inverse transforms and a gather
// give both.  phi comes from the forward's S (phi = exp(-S/tau)); nothing of the
// forward transforms is kept.  Nodes flagged CAPPED have a = 0 (their S does
// not depend on the points).  Points snap as in the forward; the gradient is
// that of the continuous definition at the snapped positions.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <vector>

#include "sdf_internal.cuh"

namespace sdf {

cudaError_t launch_adjoint_transforms(sdf_plan_impl *p, const void *w, const void *S_saved, const uint8_t *flags);
cudaError_t build_kernel_list(sdf_plan_impl *p, const std::vector<int> &ids);


template <typename T>
__global__ void __launch_bounds__(256) k_wsum(const T *__restrict__ w, const T *__restrict__ S,
                                              const uint8_t *__restrict__ flags, int64_t n, double *part) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (flags && (flags[i] & SDF_FLAG_CAPPED)) continue;
        acc += (double)w[i] * (double)S[i];
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Per point: dL/dY_k from the D gradient planes at its node; the |X| f plane
// value summed per block (with multiplicity: every point counts).
template <typename T>
__global__ void __launch_bounds__(256) k_adj_gather(int D, int64_t K, const int *__restrict__ pt_bin,
                                                    const int *__restrict__ pt_lc, int N0, int N1, int nb0, int nb1,
                                                    const T *__restrict__ planes, int64_t nnodes, double *dLdY,
                                                    double *part) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < K; k += (int64_t)gridDim.x * blockDim.x) {
        const int lc = pt_lc[k];
        if (lc < 0) {
            for (int a = 0; a < D; ++a) dLdY[k * D + a] = 0.0;
            continue;
        }
        const int b = pt_bin[k];
        const int bx = b % nb0, by = (b / nb0) % nb1, bz = b / (nb0 * nb1);
        const int x = bx * 8 + (lc & 7), y = by * 8 + ((lc >> 3) & 7), z = bz * 8 + (lc >> 6);
        const int64_t node = x + (int64_t)N0 * (y + (int64_t)N1 * z);
        for (int a = 0; a < D; ++a) dLdY[k * D + a] = (double)planes[a * nnodes + node];
        acc += (double)planes[D * nnodes + node];
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// dL/dtau = (sum_X w S - sum_k rf(Y_k)) / tau, partials summed in fixed order.
__global__ void k_adj_final(const double *__restrict__ part, double inv_tau, double *out) {
    __shared__ double ra[256], rb[256];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < kAdjParts; i += blockDim.x) {
        a += part[i];
        b += part[kAdjParts + i];
    }
    ra[threadIdx.x] = a;
    rb[threadIdx.x] = b;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            ra[threadIdx.x] += ra[threadIdx.x + s];
            rb[threadIdx.x] += rb[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = (ra[0] - rb[0]) * inv_tau;
}

static double zr(int nodd) { const int q = nodd & 3; return q == 0 ? 1.0 : (q == 2 ? -1.0 : 0.0); }
static double zi(int nodd) { const int q = nodd & 3; return q == 1 ? -1.0 : (q == 3 ? 1.0 : 0.0); }

// Kernels, packed groups and buffers of the adjoint (first call only).
static cudaError_t adjoint_setup(sdf_plan_impl *p) {
    if (p->adj_ngroup > 0) return cudaSuccess;
    const int D = p->D;
    std::vector<int> ids = {KER_GX, KER_GY};
    if (D == 3) ids.push_back(KER_GZ);
    ids.push_back(KER_RF);
    cudaError_t e = build_kernel_list(p, ids);
    if (e != cudaSuccess) return e;
    auto term = [&](int id, double alpha_r, double alpha_i) {
        // beta = alpha * zeta(kernel)
        const int s = p->kslot[id];
        const int n = __builtin_popcount((unsigned)p->kernels[s].parity);
        const double r = zr(n), i = zi(n);
        return Term{s, 0, alpha_r * r - alpha_i * i, alpha_r * i + alpha_i * r};
    };
    Group &g0 = p->adj_group[0];
    g0.nterm = 2;
    g0.term[0] = term(KER_GX, 1, 0);
    g0.term[1] = term(KER_GY, 0, 1);
    p->adj_gch[0][0] = CH_AGX;
    p->adj_gch[0][1] = CH_AGY;
    Group &g1 = p->adj_group[1];
    if (D == 3) {
        g1.nterm = 2;
        g1.term[0] = term(KER_GZ, 1, 0);
        g1.term[1] = term(KER_RF, 0, 1);
        p->adj_gch[1][0] = CH_AGZ;
        p->adj_gch[1][1] = CH_ARF;
    } else {
        g1.nterm = 1;
        g1.term[0] = term(KER_RF, 1, 0);
        p->adj_gch[1][0] = CH_ARF;
        p->adj_gch[1][1] = CH_NONE;
    }
    const size_t esz = (p->prec == SDF_FP64) ? sizeof(double) : sizeof(float);
    if ((e = dev_alloc(&p->adj_planes, esz * (D + 1) * p->nnodes)) != cudaSuccess) return e;
    if ((e = dev_alloc((void **)&p->adj_part, sizeof(double) * 2 * kAdjParts)) != cudaSuccess) return e;
    p->workspace_bytes += esz * (D + 1) * p->nnodes + sizeof(double) * 2 * kAdjParts;
    p->adj_ngroup = 2;
    return cudaSuccess;
}

cudaError_t launch_adjoint(sdf_plan_impl *p, int64_t K, const double *points, const void *w, const void *S_saved,
                           const uint8_t *flags, double *dL_dY, double *dL_dtau) {
    cudaError_t e = adjoint_setup(p);
    if (e != cudaSuccess) return e;
    cudaStream_t st = p->stream;
    if ((e = launch_points(p, K, points, nullptr)) != cudaSuccess) return e;
    if ((e = launch_adjoint_transforms(p, w, S_saved, flags)) != cudaSuccess) return e;
    prof_begin(p, "adj_reduce", st);
    if (p->prec == SDF_FP64) {
        k_wsum<double><<<kAdjParts, 256, 0, st>>>(reinterpret_cast<const double *>(w),
                                                 reinterpret_cast<const double *>(S_saved), flags, p->nnodes,
                                                 p->adj_part);
        k_adj_gather<double><<<kAdjParts, 256, 0, st>>>(p->D, K, p->pt_key, p->pt_lc, (int)p->N[0], (int)p->N[1],
                                                        (int)p->nb[0], (int)p->nb[1],
                                                        reinterpret_cast<const double *>(p->adj_planes), p->nnodes,
                                                        dL_dY, p->adj_part + kAdjParts);
    } else {
        k_wsum<float><<<kAdjParts, 256, 0, st>>>(reinterpret_cast<const float *>(w),
                                                reinterpret_cast<const float *>(S_saved), flags, p->nnodes,
                                                p->adj_part);
        k_adj_gather<float><<<kAdjParts, 256, 0, st>>>(p->D, K, p->pt_key, p->pt_lc, (int)p->N[0], (int)p->N[1],
                                                       (int)p->nb[0], (int)p->nb[1],
                                                       reinterpret_cast<const float *>(p->adj_planes), p->nnodes,
                                                       dL_dY, p->adj_part + kAdjParts);
    }
    k_adj_final<<<1, 256, 0, st>>>(p->adj_part, 1.0 / p->tau, dL_dtau);
    prof_end(p, st);
    return cudaGetLastError();
}

}  // namespace sdf
