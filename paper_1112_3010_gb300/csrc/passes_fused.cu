// passes_fused.cu -- launcher of the fused pass (Table 1 steps 3-5 of the
// paper): forward transform along the last axis, multiply by every kernel
// spectrum, inverse transform along the same axis.  The kernel variants are
// compiled in passes_fused_f2.cu, passes_fused_f3.cu and passes_fused_d.cu
// (in parallel); this file only chooses and launches them.
#include "passes.cuh"

namespace sdf {

template <typename T>
cudaError_t fused_step(sdf_plan_impl *p, const cx<T> *fin, cx<T> *fout, int logL, int n_in, int64_t n_lines,
                       int64_t in_fs, bool dense, bool skip_mu, const sdf_plan_impl *p1, cx<T> *fout1) {
    using V = cx<T>;
    cudaStream_t st = p->stream;
    cudaError_t e;
    const int D = p->D;
    const int64_t N1 = p->N[1], N2 = p->N[2], M0 = p->M[0];
    {
        const int TPL = line_len(logL) >> 4;
        int R = 1;
        while (R * 2 * TPL <= 256) R *= 2;
        if (p->tune_RF > 0) {
            R = p->tune_RF;
            while (R > 1 && R * TPL > 512) R >>= 1;
        }
        // the two-CTAs-per-SM variant needs <= 256 threads
        const bool fv = p->tune_FV == 1 && R * TPL <= 256;
        LineCfg c = line_cfg(logL, R);
        const size_t smem = line_smem(R, c.L, (int)sizeof(V));
        FusedParams F = make_fused_params(p, dense);
        if (dense) F.nfield = 1;
        // the sign group (the last) left to another plan on the same points
        if (skip_mu && !dense && F.ngroup > 0 && p->gch[F.ngroup - 1][0] == CH_MU) --F.ngroup;
        // a second plan on the same transforms (per-line kernel only): its
        // groups without the sign group, which reads the other fields
        FusedParams F1;
        memset(&F1, 0, sizeof(F1));
        if (p1) {
            F1 = make_fused_params(p1, false);
            if (F1.ngroup > 0 && p1->gch[F1.ngroup - 1][0] == CH_MU) --F1.ngroup;
        }
        const int64_t n_out = (D == 2) ? N1 : N2;
        const int64_t out_fs = n_lines * n_out;
        const int64_t grid = (n_lines + R - 1) / R;
        const V *twl = reinterpret_cast<const V *>(p->tw[D - 1]);
        prof_begin(p, "fused", st);
        // paired-column variant (2D float plans that fit), on request: the
        // per-line variant below measured faster on GB300 and is the default
        const size_t smem2p = (!dense && sizeof(T) == 4) ? fused2p_smem(p) : 0;
        if (smem2p && p->tune_FV == 3 && !p1) {
#define SDF_F2P(LG)                                                                                     \
    do {                                                                                                \
        if ((e = run_fused2p<T, LG>((unsigned)(M0 / 2 + 1), 2 * TPL, smem2p, st, fin, fout, logL, n_in,  \
                                    (int)n_out, in_fs, out_fs, F, (int)p->kernels.size(), twl)) !=      \
            cudaSuccess)                                                                                \
            return e;                                                                                   \
    } while (0)
            if constexpr (sizeof(T) == 4) SDF_BY_LOGL(T, logL, SDF_F2P);
#undef SDF_F2P
            prof_end(p, st);
            return cudaGetLastError();
        }
#define SDF_FUSED(DD, FVV, LG)                                                                               \
    do {                                                                                                     \
        if ((e = run_fused<T, DD, FVV, LG>((unsigned)grid, R * c.TPL, smem, st, fin, fout, logL, n_in,        \
                                           (int)n_out, R, n_lines, in_fs, out_fs, F, twl, F1, fout1)) !=     \
            cudaSuccess)                                                                                     \
            return e;                                                                                        \
    } while (0)
#define SDF_FUSED2(LG) SDF_FUSED(2, 0, LG)
#define SDF_FUSED3(LG) SDF_FUSED(3, 0, LG)
        if (fv) {
            if (D == 2) SDF_FUSED(2, 1, 0);
            else SDF_FUSED(3, 1, 0);
        } else if (D == 2) {
            SDF_BY_LOGL(T, logL, SDF_FUSED2);
        } else {
            SDF_BY_LOGL(T, logL, SDF_FUSED3);
        }
#undef SDF_FUSED2
#undef SDF_FUSED3
#undef SDF_FUSED
        prof_end(p, st);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template cudaError_t fused_step<float>(sdf_plan_impl *, const float2 *, float2 *, int, int, int64_t, int64_t, bool,
                                       bool, const sdf_plan_impl *, float2 *);
template cudaError_t fused_step<double>(sdf_plan_impl *, const double2 *, double2 *, int, int, int64_t, int64_t,
                                        bool, bool, const sdf_plan_impl *, double2 *);

}  // namespace sdf
