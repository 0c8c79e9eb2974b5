// passes_fwd.cu -- launchers of the forward x-pass and (3D) y-pass (Table 1
// steps 2-3 of the paper); the fused pass that follows is in passes_fused.cu.
#include "passes.cuh"

namespace sdf {

template <typename T>
cudaError_t fwd_T_launch(const cx<T> *in, cx<T> *out, int logL, int n_in, int64_t n_lines, int nfield, int64_t in_fs,
                         int64_t out_fs, const cx<T> *tw, cudaStream_t st, sdf_plan_impl *p) {
    const int R = tuned_R<T>(p, logL);
    LineCfg c = line_cfg(logL, R);
    const size_t smem = line_smem(R, c.L, (int)sizeof(cx<T>));
    cudaError_t e;
    const int64_t grid = (n_lines + R - 1) / R;
    if (p) prof_begin(p, "fwd_y", st);
#define SDF_FWDT(LG) \
    SDF_LAUNCH_MT(k_fwd_T, T, LG, R * c.TPL, grid, smem, st, in, out, logL, n_in, R, n_lines, nfield, in_fs, out_fs, tw)
    SDF_BY_LOGL(T, logL, SDF_FWDT);
#undef SDF_FWDT
    if (p) prof_end(p, st);
    return cudaGetLastError();
}
template cudaError_t fwd_T_launch<double>(const double2 *, double2 *, int, int, int64_t, int, int64_t, int64_t,
                                          const double2 *, cudaStream_t, sdf_plan_impl *);
template cudaError_t fwd_T_launch<float>(const float2 *, float2 *, int, int, int64_t, int, int64_t, int64_t,
                                         const float2 *, cudaStream_t, sdf_plan_impl *);

// The forward transforms up to the fused pass's input (x-pass, and the
// y-pass in 3D): they depend on the points and the grid, not on tau or the
// kernels.  With `shared` (another plan of the same shape and precision that
// ran them for the same points), p skips them and its fused pass reads that
// plan's buffer.
template <typename T>
static cudaError_t forward_impl(sdf_plan_impl *p, bool with_weights, const void *dense_in, const uint8_t *flags_in,
                                const sdf_plan_impl *shared = nullptr, bool shared_only = false,
                                bool skip_mu = false, const sdf_plan_impl *pair = nullptr) {
    using V = cx<T>;
    cudaStream_t st = p->stream;
    cudaError_t e;
    const int D = p->D;
    const int nfield = dense_in ? 1 : (with_weights ? p->nfield : 1);
    V *A = reinterpret_cast<V *>(p->bufA);
    V *B = reinterpret_cast<V *>(p->bufB);
    const int64_t N0 = p->N[0], N1 = p->N[1], N2 = p->N[2];
    const int64_t M0 = p->M[0], M1 = p->M[1];
    if (shared) {
        // 2D: the fused input is the x-pass output (bufA); 3D: the y-pass output (bufB)
        const V *fin = reinterpret_cast<const V *>(D == 2 ? shared->bufA : shared->bufB);
        V *fout = D == 2 ? B : A;
        V *fout1 = pair ? reinterpret_cast<V *>(D == 2 ? pair->bufB : pair->bufA) : nullptr;
        if (D == 2) return fused_step<T>(p, fin, fout, p->logM[1], (int)N1, M0, M0 * N1, false, skip_mu, pair, fout1);
        return fused_step<T>(p, fin, fout, p->logM[2], (int)N2, M1 * M0, M1 * M0 * N2, false, skip_mu, pair, fout1);
    }
    // ---- x-pass
    {
        const int logL = p->logM[0];
        const int R = dense_in ? pick_R(logL, sizeof(V), max_threads<T>(), 16, kSmemBudget)
                               : tuned_R<T>(p, logL, xpass_max_threads<T>(logL));
        LineCfg c = line_cfg(logL, R);
        const int64_t n_lines = N1 * (D == 3 ? N2 : 1);
        const size_t smem = line_smem(R, c.L, (int)sizeof(V));
        const int64_t grid = (n_lines + R - 1) / R;
        const V *tw0 = reinterpret_cast<const V *>(p->tw[0]);
        if (dense_in) {
            const T *const *pair = reinterpret_cast<const T *const *>(dense_in);
            prof_begin(p, "xpass_dense", st);
#define SDF_XD(LG)                                                                                         \
    do {                                                                                                   \
        if ((e = set_smem<T>((const void *)k_xpass_dense<T, LG>, smem)) != cudaSuccess) return e;          \
        k_xpass_dense<T, LG><<<(unsigned)grid, R * c.TPL, smem, st>>>(pair[0], pair[1], flags_in, 1.0 / p->tau, \
                                                                     (int)N0, logL, R, n_lines, A, tw0);   \
    } while (0)
            SDF_BY_LOGL(T, logL, SDF_XD);
#undef SDF_XD
            prof_end(p, st);
        } else {
            prof_begin(p, "xpass", st);
#define SDF_XC_MT(MTT, LG)                                                                                \
    do {                                                                                                  \
        if ((e = set_smem<T>((const void *)k_xpass_cells<T, MTT, LG>, smem)) != cudaSuccess) return e;   \
        k_xpass_cells<T, MTT, LG><<<(unsigned)grid, R * c.TPL, smem, st>>>(                              \
            p->bin_start, p->bin_nuniq, p->ucell, p->ucount, p->uw, (int)N1, (int)p->nb[0], (int)p->nb[1], \
            logL, R, nfield, n_lines, A, M0 * n_lines, tw0);                                              \
    } while (0)
#define SDF_XC(LG)                                              \
    do {                                                        \
        if constexpr (LG > 0) {                                 \
            if (R * c.TPL > 512) {                              \
                SDF_XC_MT(1024, LG);                            \
                break;                                          \
            }                                                   \
        }                                                       \
        SDF_XC_MT(512, LG);                                     \
    } while (0)
            SDF_BY_LOGL(T, logL, SDF_XC);
#undef SDF_XC
#undef SDF_XC_MT
            prof_end(p, st);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const V *fin = A;
    V *fout = B;
    int64_t fused_lines = M0;
    int fused_logL = p->logM[1];
    int fused_nin = (int)N1;
    int64_t in_fs = M0 * N1;
    if (D == 3) {
        // ---- y-pass: T1[u][z][y] (lines (u,z), contiguous y) -> T2[v][u][z]
        const int64_t n_lines = M0 * N2;
        if ((e = fwd_T_launch<T>(A, B, p->logM[1], (int)N1, n_lines, nfield, M0 * N2 * N1, M1 * n_lines,
                                 reinterpret_cast<const V *>(p->tw[1]), st, p)) != cudaSuccess)
            return e;
        fin = B;
        fout = A;
        fused_lines = M1 * M0;
        fused_logL = p->logM[2];
        fused_nin = (int)N2;
        in_fs = M1 * M0 * N2;
    }
    if (shared_only) return cudaSuccess;
    // ---- fused: forward along the last axis, multiply, inverse
    return fused_step<T>(p, fin, fout, fused_logL, fused_nin, fused_lines, in_fs, dense_in != nullptr);
}

cudaError_t launch_forward(sdf_plan_impl *p, bool with_weights, const void *dense_in, int /*dense_mode*/,
                           const uint8_t *flags_in) {
    if (p->prec == SDF_FP64) return forward_impl<double>(p, with_weights, dense_in, flags_in);
    return forward_impl<float>(p, with_weights, dense_in, flags_in);
}

// The tau-independent forward transforms only (x-pass, 3D y-pass) into p's buffers.
cudaError_t launch_forward_shared_part(sdf_plan_impl *p, bool with_weights) {
    if (p->prec == SDF_FP64) return forward_impl<double>(p, with_weights, nullptr, nullptr, nullptr, true);
    return forward_impl<float>(p, with_weights, nullptr, nullptr, nullptr, true);
}

// The fused pass of p on the forward transforms `shared` computed (without
// the sign group when skip_mu: another plan computes the same sign); with
// `pair`, the same launch also runs that plan's groups (sign group excepted)
// on the same forward transform of field 0.
cudaError_t launch_forward_from(sdf_plan_impl *p, const sdf_plan_impl *shared, bool skip_mu,
                                const sdf_plan_impl *pair) {
    if (p->prec == SDF_FP64) return forward_impl<double>(p, true, nullptr, nullptr, shared, false, skip_mu, pair);
    return forward_impl<float>(p, true, nullptr, nullptr, shared, false, skip_mu, pair);
}


}  // namespace sdf
