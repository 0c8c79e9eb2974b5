// curvature.cu -- curvature fields from an execute's grad S and Hessian.
// Sec. 5 notes that, with the first and second derivatives on the grid, the
// Gaussian, mean and principal curvatures of the surface S(X) follow.
//   2D: the graph z = S(x, y) (Monge patch, upward normal), W = 1 + |grad S|^2:
//       K = (S_xx S_yy - S_xy^2) / W^2,
//       H = ((1 + S_y^2) S_xx - 2 S_x S_y S_xy + (1 + S_x^2) S_yy) / (2 W^{3/2}).
//   3D: the level surfaces of S (the paper is silent), g = |grad S|:
//       H = (g^2 tr(Hess) - grad S^T Hess grad S) / (2 g^3),
//       K = grad S^T adj(Hess) grad S / g^4.
//   Principal curvatures k1 >= k2 = H +- sqrt(max(H^2 - K, 0)).
// One grid-stride pass, HBM-bound: reads D + D(D+1)/2 planes and the flags,
// writes 4 planes.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "sdf_internal.cuh"

namespace sdf {

template <typename T, int D>
__global__ void __launch_bounds__(256) k_curvature(const T *__restrict__ dS, const T *__restrict__ d2S,
                                                   const uint8_t *__restrict__ flags, T *__restrict__ curv,
                                                   int64_t n) {
    constexpr int NH = D * (D + 1) / 2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T g[D], h[NH];
#pragma unroll
        for (int a = 0; a < D; ++a) g[a] = dS[a * n + i];
#pragma unroll
        for (int a = 0; a < NH; ++a) h[a] = d2S[a * n + i];
        T K = T(0), H = T(0);
        const bool capped = flags && (flags[i] & SDF_FLAG_CAPPED);
        if (!capped) {
            if (D == 2) {
                const T sx = g[0], sy = g[D > 1 ? 1 : 0], sxx = h[0], syy = h[NH > 1 ? 1 : 0], sxy = h[NH - 1];
                const T W = T(1) + sx * sx + sy * sy;
                K = (sxx * syy - sxy * sxy) / (W * W);
                H = ((T(1) + sy * sy) * sxx - T(2) * sx * sy * sxy + (T(1) + sx * sx) * syy) / (T(2) * W * sqrt(W));
            } else {
                const T sx = g[0], sy = g[1 % D], sz = g[2 % D];
                const T a = h[0], b = h[1 % NH], c = h[2 % NH], d = h[3 % NH], e = h[4 % NH], f = h[5 % NH];
                const T g2 = sx * sx + sy * sy + sz * sz;
                if (g2 > T(0)) {
                    const T gHg = sx * (a * sx + d * sy + e * sz) + sy * (d * sx + b * sy + f * sz) +
                                  sz * (e * sx + f * sy + c * sz);
                    H = (g2 * (a + b + c) - gHg) / (T(2) * g2 * sqrt(g2));
                    const T gAg = sx * sx * (b * c - f * f) + sy * sy * (a * c - e * e) + sz * sz * (a * b - d * d) +
                                  T(2) * (sx * sy * (e * f - c * d) + sx * sz * (d * f - b * e) +
                                          sy * sz * (d * e - a * f));
                    K = gAg / (g2 * g2);
                }
            }
        }
        const T disc = H * H - K;
        const T sq = disc > T(0) ? sqrt(disc) : T(0);
        curv[i] = K;
        curv[n + i] = H;
        curv[2 * n + i] = H + sq;
        curv[3 * n + i] = H - sq;
    }
}

}  // namespace sdf

using namespace sdf;

extern "C" sdf_status sdf_curvature(sdf_plan p, const void *dS, const void *d2S, const uint8_t *flags, void *curv) {
    if (!p || !dS || !d2S || !curv) {
        set_last_error("sdf_curvature: null plan or plane");
        return SDF_ERR_INVALID_ARG;
    }
    if (p->D == 1) {
        set_last_error("sdf_curvature: 2D and 3D plans only");
        return SDF_ERR_UNSUPPORTED;
    }
    const int64_t n = p->nnodes;
    const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 8);
    prof_begin(p, "curvature", p->stream);
    if (p->prec == SDF_FP64) {
        if (p->D == 2)
            k_curvature<double, 2><<<grid, 256, 0, p->stream>>>((const double *)dS, (const double *)d2S, flags,
                                                                 (double *)curv, n);
        else
            k_curvature<double, 3><<<grid, 256, 0, p->stream>>>((const double *)dS, (const double *)d2S, flags,
                                                                 (double *)curv, n);
    } else {
        if (p->D == 2)
            k_curvature<float, 2><<<grid, 256, 0, p->stream>>>((const float *)dS, (const float *)d2S, flags,
                                                                (float *)curv, n);
        else
            k_curvature<float, 3><<<grid, 256, 0, p->stream>>>((const float *)dS, (const float *)d2S, flags,
                                                                (float *)curv, n);
    }
    prof_end(p, p->stream);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return SDF_ERR_CUDA;
    }
    return SDF_OK;
}
