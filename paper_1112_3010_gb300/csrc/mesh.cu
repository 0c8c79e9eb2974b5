// mesh.cu -- point sources of a triangle mesh for the 3D degree (Sec. 4.2 and
// Example 5): each triangle contributes its incentre Y_k (the vertices
// weighted by the opposite side lengths) with the normal P_k = (B - A) x
// (C - A) / 2, the edge cross product scaled to the triangle's area, so that
// the normalized flux (eq. normflux) sums area-weighted normals.  Orientation
// comes from the faces' vertex order, or, given a centre c, from the rule of
// Example 5: P_k is negated where <Y_k - c, P_k> < 0.  One thread per
// triangle; the result feeds sdf_execute as points and weights.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sdf_internal.cuh"

namespace sdf {

__global__ void k_mesh_sources(int64_t nf, int64_t nv, const double *__restrict__ V, const int64_t *__restrict__ F,
                               int use_center, double c0, double c1, double c2, double *__restrict__ Y,
                               double *__restrict__ P, DevScalars *dsc) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nf) return;
    const int64_t ia = F[3 * k], ib = F[3 * k + 1], ic = F[3 * k + 2];
    if (ia < 0 || ib < 0 || ic < 0 || ia >= nv || ib >= nv || ic >= nv) {
        atomicCAS(&dsc->status, 0, (int)SDF_ERR_INVALID_ARG);  // a face names a missing vertex
        for (int a = 0; a < 3; ++a) Y[3 * k + a] = P[3 * k + a] = 0.0;
        return;
    }
    double A[3], B[3], C[3], ab[3], ac[3], bc[3];
    for (int a = 0; a < 3; ++a) {
        A[a] = V[3 * ia + a];
        B[a] = V[3 * ib + a];
        C[a] = V[3 * ic + a];
        ab[a] = B[a] - A[a];
        ac[a] = C[a] - A[a];
        bc[a] = C[a] - B[a];
    }
    const double la = sqrt(bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]);
    const double lb = sqrt(ac[0] * ac[0] + ac[1] * ac[1] + ac[2] * ac[2]);
    const double lc = sqrt(ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2]);
    const double sum = la + lb + lc;
    double y[3], n[3];
    for (int a = 0; a < 3; ++a) y[a] = (la * A[a] + lb * B[a] + lc * C[a]) / sum;
    n[0] = 0.5 * (ab[1] * ac[2] - ab[2] * ac[1]);
    n[1] = 0.5 * (ab[2] * ac[0] - ab[0] * ac[2]);
    n[2] = 0.5 * (ab[0] * ac[1] - ab[1] * ac[0]);
    if (use_center) {
        const double dot = (y[0] - c0) * n[0] + (y[1] - c1) * n[1] + (y[2] - c2) * n[2];
        if (dot < 0.0)
            for (int a = 0; a < 3; ++a) n[a] = -n[a];
    }
    for (int a = 0; a < 3; ++a) {
        Y[3 * k + a] = y[a];
        P[3 * k + a] = n[a];
    }
}

}  // namespace sdf

using namespace sdf;

extern "C" sdf_status sdf_mesh_sources(sdf_plan p, int64_t nf, int64_t nv, const double *V, const int64_t *F,
                                       const double *center, double *points, double *weights) {
    if (!p || nf < 0 || nv < 0 || (nf > 0 && (!V || !F || !points || !weights))) {
        set_last_error("sdf_mesh_sources: null plan or buffer, or negative count");
        return SDF_ERR_INVALID_ARG;
    }
    if (p->D != 3) {
        set_last_error("sdf_mesh_sources: 3D plans only");
        return SDF_ERR_UNSUPPORTED;
    }
    if (nf == 0) return SDF_OK;
    const unsigned grid = (unsigned)((nf + 255) / 256);
    prof_begin(p, "mesh_sources", p->stream);
    k_mesh_sources<<<grid, 256, 0, p->stream>>>(nf, nv, V, F, center ? 1 : 0, center ? center[0] : 0.0,
                                                 center ? center[1] : 0.0, center ? center[2] : 0.0, points, weights,
                                                 p->dsc);
    prof_end(p, p->stream);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return SDF_ERR_CUDA;
    }
    return SDF_OK;
}
