// passes_inv.cu -- launchers of the inverse passes after the fused pass:
// the 3D inverse y-pass, the epilogue (Table 1 step 6 of the paper: S, its
// derivatives and the sign) and the adjoint's last pass.
#include <cudaTypedefs.h>

#include <mutex>

#include "passes.cuh"

namespace sdf {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); null when unavailable.
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
        cudaGetLastError();
    });
    return fn;
}

// The epilogue input as a 3D float tensor: x = 2 n_lines floats (re, im of
// each line, lines contiguous), y = M0 elements (stride n_lines complex), z =
// the groups (stride in_fs); box 2R floats x kTmaBoxRows x 1.  Cached in the
// plan per (buffer, n_lines, M0, groups, R).  False when it cannot be made.
static bool epilogue_tmap(sdf_plan_impl *p, const float2 *in, int64_t n_lines, int64_t M0, int64_t in_fs, int ngroup,
                          int R) {
    const int64_t key[5] = {(int64_t)(uintptr_t)in, n_lines, M0, ngroup, R};
    bool same = true;
    for (int i = 0; i < 5; ++i) same = same && key[i] == p->epi_tmap_key[i];
    if (same) return true;
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)(2 * n_lines), (cuuint64_t)M0, (cuuint64_t)ngroup};
    const cuuint64_t strides[2] = {(cuuint64_t)(n_lines * sizeof(float2)), (cuuint64_t)(in_fs * sizeof(float2))};
    const cuuint32_t box[3] = {(cuuint32_t)(2 * R), (cuuint32_t)kTmaBoxRows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (fn(&p->epi_tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2 *>(in), dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
        for (int i = 0; i < 5; ++i) p->epi_tmap_key[i] = 0;
        return false;
    }
    for (int i = 0; i < 5; ++i) p->epi_tmap_key[i] = key[i];
    return true;
}

// Inverse passes after the fused pass; the result of the fused pass is in
// bufB (2D) or bufA (3D).  For 3D the inverse y-pass goes bufA -> bufB.
template <typename T>
static cudaError_t inverse_mid(sdf_plan_impl *p, int ngroup, const cx<T> **last_in) {
    using V = cx<T>;
    const int D = p->D;
    if (D == 2) {
        *last_in = reinterpret_cast<const V *>(p->bufB);
        return cudaSuccess;
    }
    const int64_t N1 = p->N[1], N2 = p->N[2], M0 = p->M[0], M1 = p->M[1];
    const int logL = p->logM[1];
    const int R = tuned_R<T>(p, logL);
    LineCfg c = line_cfg(logL, R);
    const size_t smem = line_smem(R, c.L, (int)sizeof(V));
    cudaError_t e;
    const int64_t n_lines = M0 * N2;  // lines (u, z')
    const int64_t grid = (n_lines + R - 1) / R;
    prof_begin(p, "inv_y", p->stream);
#define SDF_INVT(LG)                                                                                 \
    SDF_LAUNCH_MT(k_inv_T, T, LG, R * c.TPL, grid, smem, p->stream, reinterpret_cast<const V *>(p->bufA), \
                  reinterpret_cast<V *>(p->bufB), logL, (int)N1, R, n_lines, ngroup, M1 * n_lines,      \
                  n_lines * N1, reinterpret_cast<const V *>(p->tw[1]))
    SDF_BY_LOGL(T, logL, SDF_INVT);
#undef SDF_INVT
    prof_end(p, p->stream);
    *last_in = reinterpret_cast<const V *>(p->bufB);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t inverse_epilogue_impl(sdf_plan_impl *p, bool with_weights, void *S, void *dS, void *d2S,
                                         int8_t *sign, uint8_t *flags, const int8_t *sign_in) {
    using V = cx<T>;
    const int D = p->D;
    // groups actually computed: the sign group only with weights, and not
    // when the sign comes from another plan
    int ng = p->ngroup;
    if (!with_weights || sign_in) {
        while (ng > 0 && p->gch[ng - 1][0] == CH_MU) --ng;
    }
    const V *lin = nullptr;
    cudaError_t e = inverse_mid<T>(p, ng, &lin);
    if (e != cudaSuccess) return e;
    EpiParams E;
    memset(&E, 0, sizeof(E));
    E.ngroup = ng;
    int k = 0;
    for (int g = 0; g < ng; ++g)
        if (p->gch[g][0] == CH_MU) E.order[k++] = g;
    for (int g = 0; g < ng; ++g)
        if (p->gch[g][0] != CH_MU) E.order[k++] = g;
    for (int g = 0; g < ng; ++g) {
        E.gch[g][0] = p->gch[g][0];
        E.gch[g][1] = p->gch[g][1];
    }
    const int64_t N0 = p->N[0], N1 = p->N[1], N2 = p->N[2], M0 = p->M[0];
    const int64_t n_lines = N1 * (D == 3 ? N2 : 1);
    E.in_fs = M0 * n_lines;
    E.S = S;
    E.dS = dS;
    E.d2S = d2S;
    E.sign = with_weights ? sign : nullptr;
    E.sign_in = with_weights ? sign_in : nullptr;
    E.flags = flags;
    E.tile_flag = p->tile_flag;
    E.dsc = p->dsc;
    E.dsc_w = p->dsc;
    E.tau = p->tau;
    {
        const double n = (double)p->M[0] * (double)p->M[1] * (D == 3 ? (double)p->M[2] : 1.0);
        const double base = sqrt(log2(n)) / sqrt(n) * p->q_factor / kTrustEps;
        E.coef64 = p->noise_c64 * ldexp(1.0, -53) * base;
        E.coef32 = p->noise_c32 * ldexp(1.0, -24) * base;
    }
    E.nnodes = p->nnodes;
    E.N0 = (int)N0;
    E.N1 = (int)N1;
    E.nb0 = (int)p->nb[0];
    E.nb1 = (int)p->nb[1];
    E.D = D;
    E.fixup = (p->prec == SDF_FP32) ? 1 : 0;
    E.hs_inv = 1.0 / hessian_scale(p);
    E.tau_f = (float)p->tau;
    E.itau_f = (float)(1.0 / p->tau);
    E.hs_inv_f = (float)E.hs_inv;
    const int logL = p->logM[0];
    const int R = tuned_R<T>(p, logL);
    LineCfg c = line_cfg(logL, R);
    size_t smem = line_smem(R, c.L, (int)sizeof(V));
    const int64_t grid = (n_lines + R - 1) / R;
    const V *tw0 = reinterpret_cast<const V *>(p->tw[0]);
    // TMA staging of the transposed input: float lines of a compiled length
    // that is a multiple of the box rows, at least two lines per CTA (16-byte
    // rows), an even line count (16-byte strides), the staging buffer beside
    // the line buffers within the shared memory of a CTA
    CUtensorMap tmap;
    memset(&tmap, 0, sizeof(tmap));
    bool tma = false;
    if constexpr (sizeof(T) == 4) {
        const bool compiled = (logL >= 8 && logL <= 12) || (logL >= (8 | kLineR3) && logL <= (10 | kLineR3));
        const size_t off = smem;
        const size_t tot = off + 1024 + (size_t)R * c.L * sizeof(V);
        if (p->tune_EV == 0 && compiled && R >= 2 && c.L % kTmaBoxRows == 0 && n_lines % 2 == 0 &&
            tot <= 227 * 1024 &&
            epilogue_tmap(p, reinterpret_cast<const float2 *>(lin), n_lines, M0, E.in_fs, p->ngroup, R)) {
            tma = true;
            E.stage_off = (unsigned)off;
            E.wait_polls = tma_wait_polls();
            smem = tot;
            tmap = p->epi_tmap;
        }
    }
    // the TMA kernel is persistent: as many CTAs as fit on the device at once
#define SDF_EPI(DD, LG, TM)                                                                                      \
    do {                                                                                                         \
        const void *fn_ = (const void *)k_epilogue<T, DD, 512, LG, TM>;                                          \
        if ((e = set_smem<T>(fn_, smem)) != cudaSuccess) return e;                                               \
        int64_t g_ = grid;                                                                                       \
        if (TM) {                                                                                                \
            int per_sm = 0;                                                                                      \
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn_, R * c.TPL, smem)) != cudaSuccess) \
                return e;                                                                                        \
            g_ = std::min<int64_t>(grid, (int64_t)std::max(per_sm, 1) * sm_count());                             \
        }                                                                                                        \
        k_epilogue<T, DD, 512, LG, TM><<<(unsigned)g_, R * c.TPL, smem, p->stream>>>(lin, logL, R, n_lines, E,  \
                                                                                     tw0, tmap);                \
    } while (0)
    prof_begin(p, "epilogue", p->stream);
#define SDF_EPI2(LG) SDF_EPI(2, LG, false)
#define SDF_EPI3(LG) SDF_EPI(3, LG, false)
#define SDF_EPI2T(LG) SDF_EPI(2, LG, true)
#define SDF_EPI3T(LG) SDF_EPI(3, LG, true)
    if constexpr (sizeof(T) == 4) {
        if (tma) {
            if (D == 2) SDF_BY_LOGL_COMPILED(logL, SDF_EPI2T);
            else SDF_BY_LOGL_COMPILED(logL, SDF_EPI3T);
        } else if (D == 2) {
            SDF_BY_LOGL(T, logL, SDF_EPI2);
        } else {
            SDF_BY_LOGL(T, logL, SDF_EPI3);
        }
    } else {
        if (D == 2) SDF_BY_LOGL(T, logL, SDF_EPI2);
        else SDF_BY_LOGL(T, logL, SDF_EPI3);
    }
#undef SDF_EPI2
#undef SDF_EPI3
#undef SDF_EPI2T
#undef SDF_EPI3T
#undef SDF_EPI
    prof_end(p, p->stream);
    (void)N2;
    return cudaGetLastError();
}

cudaError_t launch_inverse_epilogue(sdf_plan_impl *p, bool with_weights, void *S, void *dS, void *d2S, int8_t *sign,
                                    uint8_t *flags, const int8_t *sign_in) {
    if (p->prec == SDF_FP64) return inverse_epilogue_impl<double>(p, with_weights, S, dS, d2S, sign, flags, sign_in);
    return inverse_epilogue_impl<float>(p, with_weights, S, dS, d2S, sign, flags, sign_in);
}

// ---------------------------------------------------------------- adjoint epilogue
// Last inverse pass of the adjoint: the real / imaginary part of each group
// goes to dense plane plane[g][0|1] (-1: dropped), node order x fastest.
struct DenseParams {
    int ngroup;
    int plane[2][2];
    int64_t in_fs, nnodes;
    int N0;
};

template <typename T, int LOGL = 0>
__global__ void SDF_LB(T) k_epi_dense(const cx<T> *__restrict__ in, int logL, int R, int64_t n_lines, DenseParams P,
                                      T *planes, const cx<T> *__restrict__ tw) {
    using V = cx<T>;
    if constexpr (LOGL > 0) logL = LOGL;  // line length fixed at compile time
    extern __shared__ unsigned char smraw[];
    V *sm = reinterpret_cast<V *>(smraw);
    const int L = line_len(logL), TPL = L >> 4, PL = pad16(L);
    const int tid = threadIdx.x, lr = tid % R, t = tid / R;
    const int64_t line = (int64_t)blockIdx.x * R + lr;
    const bool valid = line < n_lines;
    V *my = sm + lr * line_stride(PL, R, (int)sizeof(V));
    const V *tws = stage_twiddles(sm + R * line_stride(PL, R, (int)sizeof(V)), tw, L);
    for (int g = 0; g < P.ngroup; ++g) {
        V v[16];
        const V *src = in + g * P.in_fs + line;
#pragma unroll
        for (int m = 0; m < 16; ++m) v[m] = valid ? src[(int64_t)(t + m * TPL) * n_lines] : mk<V>(T(0), T(0));
        __syncthreads();
        fft_line<true, LOGL>(v, my, t, logL, tws);
        if (!valid) continue;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int x = t + m * TPL;
            if (x >= P.N0) continue;
            const int64_t node = line * P.N0 + x;
            if (P.plane[g][0] >= 0) planes[P.plane[g][0] * P.nnodes + node] = v[m].x;
            if (P.plane[g][1] >= 0) planes[P.plane[g][1] * P.nnodes + node] = v[m].y;
        }
    }
}

// Transform a = w/phi (dense x-pass, [y-pass], fused pass with the adjoint
// programme, [inverse y-pass]) and write the D+1 convolution planes
// (a * k_x, a * k_y[, a * k_z], a * (|X| f)) to p->adj_planes.
template <typename T>
static cudaError_t adjoint_transforms_impl(sdf_plan_impl *p, const void *w, const void *S_saved,
                                           const uint8_t *flags) {
    using V = cx<T>;
    const void *pair[2] = {w, S_saved};
    cudaError_t e = launch_forward(p, false, pair, 0, flags);
    if (e != cudaSuccess) return e;
    const V *lin = nullptr;
    if ((e = inverse_mid<T>(p, p->adj_ngroup, &lin)) != cudaSuccess) return e;
    const int D = p->D;
    const int64_t N1 = p->N[1], N2 = p->N[2], M0 = p->M[0];
    const int64_t n_lines = N1 * (D == 3 ? N2 : 1);
    DenseParams P;
    memset(&P, 0, sizeof(P));
    P.ngroup = p->adj_ngroup;
    for (int g = 0; g < p->adj_ngroup; ++g)
        for (int hh = 0; hh < 2; ++hh) {
            const int ch = p->adj_gch[g][hh];
            P.plane[g][hh] = ch == CH_AGX ? 0 : ch == CH_AGY ? 1 : ch == CH_AGZ ? 2 : ch == CH_ARF ? D : -1;
        }
    P.in_fs = M0 * n_lines;
    P.nnodes = p->nnodes;
    P.N0 = (int)p->N[0];
    const int logL = p->logM[0];
    const int R = pick_R(logL, sizeof(V), max_threads<T>(), 16, kSmemBudget);
    LineCfg c = line_cfg(logL, R);
    const size_t smem = line_smem(R, c.L, (int)sizeof(V));
    prof_begin(p, "epi_dense", p->stream);
#define SDF_ED(LG)                                                                                          \
    do {                                                                                                    \
        if ((e = set_smem<T>((const void *)k_epi_dense<T, LG>, smem)) != cudaSuccess) return e;             \
        k_epi_dense<T, LG><<<(unsigned)((n_lines + R - 1) / R), R * c.TPL, smem, p->stream>>>(              \
            lin, logL, R, n_lines, P, reinterpret_cast<T *>(p->adj_planes), reinterpret_cast<const V *>(p->tw[0])); \
    } while (0)
    SDF_BY_LOGL(T, logL, SDF_ED);
#undef SDF_ED
    prof_end(p, p->stream);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_transforms(sdf_plan_impl *p, const void *w, const void *S_saved, const uint8_t *flags) {
    if (p->prec == SDF_FP64) return adjoint_transforms_impl<double>(p, w, S_saved, flags);
    return adjoint_transforms_impl<float>(p, w, S_saved, flags);
}

}  // namespace sdf
