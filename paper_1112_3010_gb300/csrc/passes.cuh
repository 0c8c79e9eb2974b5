// passes.cuh -- kernels and launch helpers of the FFT passes of one execute
// (Table 1 steps 2-6 of the paper, and the same steps for the derivative
// kernels of Sec. 5 and the sign kernels of Sec. 4).  The launchers live in
// passes_fwd.cu (x-pass, 3D y-pass), passes_fused.cu (fused pass) and
// passes_inv.cu (inverse y-pass, epilogue, adjoint epilogue), which compile
// in parallel.
//
// Grid layouts (x fastest unless stated; N_a nodes, M_a padded, M_a >= 2 N_a):
//   2D:  x-pass   cells      -> T1[u][y]      (u < M0, y < N1)
//        fused    T1[u][.]   -> O[g][u][y']   (forward along y, multiply, inverse, y' < N1)
//        epilogue O[g][.][y']-> out[y'][x]    (inverse along x, x < N0)
//   3D:  x-pass   cells      -> T1[u][z][y]
//        y-pass   T1[u][z][.]-> T2[v][u][z]
//        fused    T2[v][u][.]-> O[g][v][u][z']
//        inv-y    O[g][.][u][z'] -> O2[g][u][z'][y']
//        epilogue O2[g][.][z'][y'] -> out[z'][y'][x]
// A "transposed" side reads or writes element i of line l at i*n_lines + l; a
// CTA handles R consecutive lines so those accesses are R-element segments.
// Input pruning: only the first N of M inputs of a forward line are nonzero.
// Output pruning: only the first N outputs of an inverse line are kept.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "sdf_internal.cuh"

namespace sdf {

template <typename T> using cx = typename cplx_t<T>::type;

// Line kernels run at most 512 threads per CTA: each thread holds 16 complex
// values plus transform state, and 1024-thread CTAs (64 registers) spill.
#define SDF_LB(T) __launch_bounds__(512)
template <typename T> constexpr int max_threads() { return 512; }

struct LineCfg {
    int logL, L, TPL, PL, R;
};

static inline LineCfg line_cfg(int logL, int R) {
    LineCfg c;
    c.logL = logL;
    c.L = line_len(logL);
    c.TPL = c.L >> 4;
    c.PL = pad16(c.L);
    c.R = R;
    return c;
}

// Lines per CTA: the largest power of two with R*TPL <= max_threads,
// line_smem(R, L) <= smem budget and R <= r_cap.
static inline int pick_R(int logL, size_t vbytes, int max_threads, int r_cap, size_t smem_budget) {
    const int L = line_len(logL), TPL = L >> 4;
    int R = 1;
    while (R * 2 <= r_cap && (R * 2) * TPL <= max_threads && line_smem(R * 2, L, (int)vbytes) <= smem_budget) R *= 2;
    return R;
}

// ---------------------------------------------------------------- x-pass
// Builds each line of the point fields from the deduplicated node list
// (bin-grouped), transforms it along x and writes it transposed.
// Field 0: (count, 0); field 1: (w_0, w_1); field 2: (w_2, 0).
template <typename T, int MT, int LOGL = 0>
__global__ void __launch_bounds__(MT) k_xpass_cells(const int *__restrict__ bin_start, const int *__restrict__ bin_nuniq,
                                                      const int *__restrict__ ucell, const int *__restrict__ ucount,
                                                      const double *__restrict__ uw, int N1, int nb0, int nb1,
                                                      int logL, int R, int nfield, int64_t n_lines, cx<T> *out,
                                                      int64_t out_fs, const cx<T> *__restrict__ tw) {
    using V = cx<T>;
    if constexpr (LOGL > 0) logL = LOGL;  // line length fixed at compile time
    extern __shared__ unsigned char smraw[];
    V *sm = reinterpret_cast<V *>(smraw);
    const int L = line_len(logL), TPL = L >> 4, PL = pad16(L);
    const int tid = threadIdx.x, lr = tid % R, t = tid / R;
    const int64_t line = (int64_t)blockIdx.x * R + lr;
    const bool valid = line < n_lines;
    const int y = valid ? (int)(line % N1) : 0;
    const int z = valid ? (int)(line / N1) : 0;
    const int by = y >> 3, bz = z >> 3, ly = y & 7, lz = z & 7;
    const int64_t brow = (int64_t)nb0 * (by + (int64_t)nb1 * bz);
    V *my = sm + lr * line_stride(PL, R, (int)sizeof(V));
    const V *tws = stage_twiddles(sm + R * line_stride(PL, R, (int)sizeof(V)), tw, L);
    for (int f = 0; f < nfield; ++f) {
        if (f > 0) __syncthreads();
#pragma unroll
        for (int m = 0; m < 8; ++m) my[pad16(t + m * TPL)] = mk<V>(T(0), T(0));
        __syncthreads();
        bool hit = false;  // this thread placed a point on one of the CTA's lines
        if (valid) {
            for (int bx = t; bx < nb0; bx += TPL) {
                const int64_t b = brow + bx;
                const int n = bin_nuniq[b];
                const int s = bin_start[b];
                for (int i = 0; i < n; ++i) {
                    const int lc = ucell[s + i];
                    if (((lc >> 3) & 7) != ly || (lc >> 6) != lz) continue;
                    const int x = bx * 8 + (lc & 7);
                    V val;
                    if (f == 0) val = mk<V>(T(ucount[s + i]), T(0));
                    else if (f == 1) val = mk<V>(T(uw[3 * (int64_t)(s + i)]), T(uw[3 * (int64_t)(s + i) + 1]));
                    else val = mk<V>(T(uw[3 * (int64_t)(s + i) + 2]), T(0));
                    my[pad16(x)] = val;
                    hit = true;
                }
            }
        }
        // lines without points (a quarter of the rows of a typical shape
        // set) transform to zero: the CTA writes zeros and skips the FFT
        if (!__syncthreads_or(hit)) {
            if (valid) {
                V *o = out + f * out_fs + line;
#pragma unroll
                for (int m = 0; m < 16; ++m) o[(int64_t)(t + m * TPL) * n_lines] = mk<V>(T(0), T(0));
            }
            continue;
        }
        V v[16];
#pragma unroll
        for (int m = 0; m < 8; ++m) v[m] = my[pad16(t + m * TPL)];
#pragma unroll
        for (int m = 8; m < 16; ++m) v[m] = mk<V>(T(0), T(0));
        fft_line<false, LOGL>(v, my, t, logL, tws);
        if (valid) {
            V *o = out + f * out_fs + line;
#pragma unroll
            for (int m = 0; m < 16; ++m) o[(int64_t)(t + m * TPL) * n_lines] = v[m];
        }
    }
}

// x-pass of a dense real grid a(X) = w(X)/phi(X) (the adjoint's input), with
// phi = exp(-S/tau) from the forward's unsigned S; nodes flagged CAPPED give 0.
template <typename T, int LOGL = 0>
__global__ void SDF_LB(T) k_xpass_dense(const T *__restrict__ w, const T *__restrict__ Ssaved,
                                                      const uint8_t *__restrict__ flags, double inv_tau, int N0,
                                                      int logL, int R, int64_t n_lines, cx<T> *out,
                                                      const cx<T> *__restrict__ tw) {
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
    V v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const int x = t + m * TPL;
        T a = T(0);
        if (m < 8 && valid && x < N0) {
            const int64_t node = line * N0 + x;
            if (!(flags && (flags[node] & SDF_FLAG_CAPPED))) {
                // a = w / phi = w exp(S/tau)
                a = w[node] * exp(Ssaved[node] * T(inv_tau));
            }
        }
        v[m] = mk<V>(a, T(0));
    }
    __syncthreads();
    fft_line<false, LOGL>(v, my, t, logL, tws);
    if (valid) {
#pragma unroll
        for (int m = 0; m < 16; ++m) out[(int64_t)(t + m * TPL) * n_lines + line] = v[m];
    }
}

// ---------------------------------------------------------------- generic forward
// Contiguous lines of n_in stored values (the rest of the L inputs are zero),
// forward transform, transposed output.  Used for the 3D y-pass and for the
// plan-time kernel transforms (n_in = L).
template <typename T, int MT, int LOGL = 0>
__global__ void __launch_bounds__(MT) k_fwd_T(const cx<T> *__restrict__ in, cx<T> *out, int logL, int n_in, int R,
                                                int64_t n_lines, int nfield, int64_t in_fs, int64_t out_fs,
                                                const cx<T> *__restrict__ tw) {
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
    for (int f = 0; f < nfield; ++f) {
        V v[16];
        const V *src = in + f * in_fs + line * n_in;
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            const int e = t + m * TPL;
            v[m] = (valid && e < n_in) ? src[e] : mk<V>(T(0), T(0));
        }
        __syncthreads();
        fft_line<false, LOGL>(v, my, t, logL, tws);
        if (valid) {
            V *o = out + f * out_fs + line;
#pragma unroll
            for (int m = 0; m < 16; ++m) o[(int64_t)(t + m * TPL) * n_lines] = v[m];
        }
    }
}

// ---------------------------------------------------------------- fused pass
struct FusedParams {
    int ngroup;
    int nterm[kMaxGroups];
    int tk[kMaxGroups][3];     // kernel slot
    int tf[kMaxGroups][3];     // field
    double br[kMaxGroups][3], bi[kMaxGroups][3];
    float brf[kMaxGroups][3], bif[kMaxGroups][3];  // the same in float (no FP64 work in float kernels)
    const void *kc[kMaxKernels];  // compressed spectra
    int kpar[kMaxKernels];        // parity bits
    int D;
    int M0, M1;                   // padded sizes of the line axes (3D: M0 = axis0, M1 = axis1)
    int nfield;
    int64_t Hp;                   // compressed spectrum row length
};

// Bijection of [0, M) (M even): 2j -> j, 1 -> M/2, 2j+1 -> M-j.
__device__ __forceinline__ int pair_index(int i, int M) {
    const int j = i >> 1;
    return (i & 1) ? (j == 0 ? M / 2 : M - j) : j;
}

template <typename T, int D>
__device__ __forceinline__ void line_fold(int64_t line, const FusedParams &P, int64_t &cbase, int &flips) {
    // flips bit a: frequency on axis a is above M_a/2
    if (D == 2) {
        const int u = (int)line;
        const int fu = u <= P.M0 / 2 ? u : P.M0 - u;
        flips = (u > P.M0 / 2) ? 1 : 0;
        cbase = (int64_t)fu;  // times (M1/2+1) added by caller
    } else {
        const int u = (int)(line % P.M0), vv = (int)(line / P.M0);
        const int fu = u <= P.M0 / 2 ? u : P.M0 - u;
        const int fv = vv <= P.M1 / 2 ? vv : P.M1 - vv;
        flips = ((u > P.M0 / 2) ? 1 : 0) | ((vv > P.M1 / 2) ? 2 : 0);
        cbase = (int64_t)fv * (P.M0 / 2 + 1) + fu;
    }
}

// v[m] += beta * khat(w) * s[m] over a thread's 16 elements w = t + m*TPL of
// a line of length L, where khat is the folded (real) kernel spectrum row c:
// khat(w) = sg(w) c[w] for w <= L/2 and sg(w) c[L - w] above, the sign being
// alo below the fold and ahi above it (odd kernels change sign across it;
// w = L/2 takes alo).  beta is real (imag = false) or imaginary: every term
// coefficient of the programme is a real multiple of 1 or i, and alo, ahi
// carry that multiple.
template <bool LDG, typename T, typename V>
__device__ __forceinline__ void mac_term(V (&v)[16], const V (&s)[16], const T *c, int t, int TPL, int L, T alo, T ahi,
                                         bool imag) {
    const T *cp = c + t, *cn = c + (L - t);
    auto coef = [&](int m) {
        const T *q = (m < 8) ? cp + m * TPL : cn - m * TPL;
        T val;
        if constexpr (LDG) val = __ldg(q);
        else val = *q;
        return ((m < 8 || (m == 8 && t == 0)) ? alo : ahi) * val;
    };
    if (!imag) {
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            const T a = coef(m);
            v[m].x = fma(a, s[m].x, v[m].x);
            v[m].y = fma(a, s[m].y, v[m].y);
        }
    } else {
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            const T a = coef(m);
            v[m].x = fma(-a, s[m].y, v[m].x);
            v[m].y = fma(a, s[m].x, v[m].y);
        }
    }
}

// The signs below and above the fold of a term's spectrum row, with its
// coefficient folded in: lflip = the row's own fold flips an odd axis,
// wodd = the kernel is odd along the line axis.
template <typename T>
__device__ __forceinline__ void term_coef(const FusedParams &P, int g, int k, bool lflip, bool wodd, T &alo, T &ahi,
                                          bool &imag) {
    T br, bi;
    if constexpr (sizeof(T) == 4) {
        br = P.brf[g][k];
        bi = P.bif[g][k];
    } else {
        br = P.br[g][k];
        bi = P.bi[g][k];
    }
    imag = (br == T(0));
    const T cf = imag ? bi : br;
    alo = lflip ? -cf : cf;
    ahi = (lflip != wodd) ? -cf : cf;
}

// Forward along the last axis, multiply by the kernel spectra, inverse along the
// same axis, keep the first n_out outputs.  Field spectra stay in registers.
// P1 (P1.ngroup > 0): a second plan of the same shape on the same points (a
// different tau or kernel set), whose groups all read field 0: its products
// and inverses reuse this CTA's forward transform of field 0 and go to out1.
template <typename T, int D, int FV, int LOGL = 0>
__global__ void __launch_bounds__(FV ? 256 : 512, FV ? 2 : 1) k_fused(const cx<T> *__restrict__ in, cx<T> *out, int logL, int n_in, int n_out,
                                               int R, int64_t n_lines, int64_t in_fs, int64_t out_fs, FusedParams P,
                                               const cx<T> *__restrict__ tw, FusedParams P1, cx<T> *out1) {
    using V = cx<T>;
    if constexpr (LOGL > 0) logL = LOGL;  // line length fixed at compile time
    extern __shared__ unsigned char smraw[];
    V *sm = reinterpret_cast<V *>(smraw);
    const int L = line_len(logL), TPL = L >> 4, PL = pad16(L);
    const int tid = threadIdx.x, lr = tid % R, t = tid / R;
    // consecutive line ids visit frequency pairs (k, M-k), which read the same
    // folded spectrum row: the second read hits L2
    const int64_t lid = (int64_t)blockIdx.x * R + lr;
    const bool valid = lid < n_lines;
    int64_t line = 0;
    if (valid) {
        if (D == 2) {
            line = pair_index((int)lid, P.M0);
        } else {
            line = (int64_t)pair_index((int)(lid / P.M0), P.M1) * P.M0 + pair_index((int)(lid % P.M0), P.M0);
        }
    }
    V *my = sm + lr * line_stride(PL, R, (int)sizeof(V));
    const V *tws = stage_twiddles(sm + R * line_stride(PL, R, (int)sizeof(V)), tw, L);
    int64_t cb;
    int flips;
    line_fold<T, D>(line, P, cb, flips);
    cb *= P.Hp;
    const int waxis = D - 1;

    V F0[16], F1[16], F2[16];
    auto load_fwd = [&](int f, V (&v)[16]) {
        const V *src = in + f * in_fs + line * n_in;
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            const int e = t + m * TPL;
            v[m] = (valid && m < 8 && e < n_in) ? src[e] : mk<V>(T(0), T(0));
        }
        __syncthreads();
        fft_line<false, LOGL>(v, my, t, logL, tws);
    };
    auto run_group = [&](const FusedParams &Q, V *qout, int g, const V (&A)[16], const V (&B)[16], const V (&C)[16]) {
        V v[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) v[m] = mk<V>(T(0), T(0));
        for (int k = 0; k < Q.nterm[g]; ++k) {
            const int slot = Q.tk[g][k];
            const T *c = reinterpret_cast<const T *>(Q.kc[slot]);
            const int par = Q.kpar[slot];
            const int f = Q.tf[g][k];
            const bool lflip = (__popc(par & flips) & 1) != 0;
            const bool wodd = (par >> waxis) & 1;
            T alo, ahi;
            bool imag;
            term_coef<T>(Q, g, k, lflip, wodd, alo, ahi, imag);
            if (f == 2) mac_term<true>(v, C, c + cb, t, TPL, L, alo, ahi, imag);
            else if (f == 1) mac_term<true>(v, B, c + cb, t, TPL, L, alo, ahi, imag);
            else mac_term<true>(v, A, c + cb, t, TPL, L, alo, ahi, imag);
        }
        __syncthreads();
        fft_line<true, LOGL>(v, my, t, logL, tws);
        if (valid) {
            V *o = qout + g * out_fs + line * n_out;
#pragma unroll
            for (int m = 0; m < 16; ++m) {
                const int e = t + m * TPL;
                if (m < 8 && e < n_out) o[e] = v[m];
            }
        }
    };
    // groups that use field 0 only come first; the sign group (fields 1[,2]) last
    load_fwd(0, F0);
    int g = 0;
    for (; g < P.ngroup; ++g) {
        bool only0 = true;
        for (int k = 0; k < P.nterm[g]; ++k) only0 &= (P.tf[g][k] == 0);
        if (!only0) break;
        run_group(P, out, g, F0, F0, F0);
    }
    // the second plan's groups, while F0 is still live
    for (int g1 = 0; g1 < P1.ngroup; ++g1) run_group(P1, out1, g1, F0, F0, F0);
    if (g < P.ngroup) {
        load_fwd(1, F1);
        if (P.nfield > 2) load_fwd(2, F2);
        else {
#pragma unroll
            for (int m = 0; m < 16; ++m) F2[m] = mk<V>(T(0), T(0));
        }
        // no sign-group term reads field 0, so F0 is dead here
        for (; g < P.ngroup; ++g) run_group(P, out, g, F1, F1, F2);
    }
}

// ---------------------------------------------------------------- fused, paired columns (2D)
// One CTA, two halves of TPL threads: columns u = j and u = M0 - j, whose
// folded spectrum rows are the same row j.  All the plan's rows for j are
// copied to shared memory with 16-byte cp.async while the forward transform
// of field 0 runs, then every multiply reads shared memory.  j = 0 and
// j = M0/2 have no partner (the second half idles).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <typename T, int LOGL = 0>
__global__ void __launch_bounds__(512, 1) k_fused2p(const cx<T> *__restrict__ in, cx<T> *out, int logL, int n_in,
                                                    int n_out, int64_t in_fs, int64_t out_fs, FusedParams P, int nker,
                                                    const cx<T> *__restrict__ tw) {
    using V = cx<T>;
    if constexpr (LOGL > 0) logL = LOGL;  // line length fixed at compile time
    extern __shared__ __align__(16) unsigned char smraw_p[];
    const int L = line_len(logL), TPL = L >> 4, PL = pad16(L);
    const int64_t Hp = P.Hp;
    T *crow = reinterpret_cast<T *>(smraw_p);                      // nker rows of Hp
    V *sm = reinterpret_cast<V *>(smraw_p + sizeof(T) * nker * Hp);  // two exchange lines
    const int tid = threadIdx.x, hh = tid / TPL, t = tid % TPL;
    const int j = blockIdx.x;
    const int M0 = P.M0;
    const bool valid = (hh == 0) || (j > 0 && j < M0 / 2);
    const int u = hh == 0 ? j : M0 - j;
    const int flips = (u > M0 / 2) ? 1 : 0;
    V *my = sm + hh * PL;
    const V *tws = stage_twiddles(sm + 2 * PL, tw, L);
    // stage the spectrum rows of j
    {
        const int per_row = (int)(Hp * sizeof(T) / 16);
        const int total = nker * per_row;
        for (int i = tid; i < total; i += blockDim.x) {
            const int k = i / per_row, o = i % per_row;
            const T *src = reinterpret_cast<const T *>(P.kc[k]) + (int64_t)j * Hp;
            cp_async16(reinterpret_cast<unsigned char *>(crow + (int64_t)k * Hp) + 16 * o,
                       reinterpret_cast<const unsigned char *>(src) + 16 * o);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    V F0[16], F1[16];
    auto load_fwd = [&](int f, V (&v)[16]) {
        const V *src = in + f * in_fs + (int64_t)u * n_in;
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            const int e = t + m * TPL;
            v[m] = (valid && m < 8 && e < n_in) ? src[e] : mk<V>(T(0), T(0));
        }
        __syncthreads();
        fft_line<false, LOGL>(v, my, t, logL, tws);
    };
    auto run_group = [&](int g, const V (&A)[16], const V (&B)[16]) {
        V v[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) v[m] = mk<V>(T(0), T(0));
        for (int k = 0; k < P.nterm[g]; ++k) {
            const int slot = P.tk[g][k];
            const T *c = crow + (int64_t)slot * Hp;
            const int par = P.kpar[slot];
            const bool lflip = (par & flips & 1) != 0;
            const bool wodd = (par >> 1) & 1;
            T alo, ahi;
            bool imag;
            term_coef<T>(P, g, k, lflip, wodd, alo, ahi, imag);
            if (P.tf[g][k] != 0) mac_term<false>(v, B, c, t, TPL, L, alo, ahi, imag);
            else mac_term<false>(v, A, c, t, TPL, L, alo, ahi, imag);
        }
        __syncthreads();
        fft_line<true, LOGL>(v, my, t, logL, tws);
        if (valid) {
            V *o = out + g * out_fs + (int64_t)u * n_out;
#pragma unroll
            for (int m = 0; m < 16; ++m) {
                const int e = t + m * TPL;
                if (m < 8 && e < n_out) o[e] = v[m];
            }
        }
    };
    load_fwd(0, F0);
    cp_async_wait_all();
    __syncthreads();
    int g = 0;
    for (; g < P.ngroup; ++g) {
        bool only0 = true;
        for (int k = 0; k < P.nterm[g]; ++k) only0 &= (P.tf[g][k] == 0);
        if (!only0) break;
        run_group(g, F0, F0);
    }
    if (g < P.ngroup) {
        load_fwd(1, F1);
        for (; g < P.ngroup; ++g) run_group(g, F1, F1);
    }
}

// Shared memory of k_fused2p (0 when the 2D float plan does not fit).
static inline size_t fused2p_smem(const sdf_plan_impl *p) {
    if (p->D != 2 || p->prec != SDF_FP32 || p->nfield > 2) return 0;
    const size_t b = sizeof(float) * p->kernels.size() * spec_row_len(p) +
                     sizeof(float2) * (2 * pad16((int)p->M[1]) + p->M[1]);  // rows, two lines, twiddles
    const int TPL = (int)(p->M[1] >> 4);
    return (b <= 220 * 1024 && 2 * TPL <= 512) ? b : 0;
}

// ---------------------------------------------------------------- inverse (3D y)
// Transposed input (all L elements), inverse transform, contiguous output of
// the first n_out elements.
template <typename T, int MT, int LOGL = 0>
__global__ void __launch_bounds__(MT) k_inv_T(const cx<T> *__restrict__ in, cx<T> *out, int logL, int n_out, int R,
                                                int64_t n_lines, int nfield, int64_t in_fs, int64_t out_fs,
                                                const cx<T> *__restrict__ tw) {
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
    for (int f = 0; f < nfield; ++f) {
        V v[16];
        const V *src = in + f * in_fs + line;
#pragma unroll
        for (int m = 0; m < 16; ++m) v[m] = valid ? src[(int64_t)(t + m * TPL) * n_lines] : mk<V>(T(0), T(0));
        __syncthreads();
        fft_line<true, LOGL>(v, my, t, logL, tws);
        if (valid) {
            V *o = out + f * out_fs + line * n_out;
#pragma unroll
            for (int m = 0; m < 16; ++m) {
                const int e = t + m * TPL;
                if (m < 8 && e < n_out) o[e] = v[m];
            }
        }
    }
}

// ---------------------------------------------------------------- epilogue
struct EpiParams {
    int ngroup;
    int order[kMaxGroups];
    int gch[kMaxGroups][2];
    int64_t in_fs;
    void *S, *dS, *d2S;
    int8_t *sign;
    const int8_t *sign_in;  // the sign from another plan on the same points (no mu group then)
    uint8_t *flags;
    uint8_t *tile_flag;
    const DevScalars *dsc;
    DevScalars *dsc_w;  // the same scalars, for the count of capped nodes
    double tau, coef64, coef32;
    int64_t nnodes;
    int N0, N1;
    int nb0, nb1;
    int D;
    int fixup;  // FP32 plan: nodes below theta32 go to the fix-up
    double hs_inv;  // 1 / scale of the stored Hessian kernels
    float tau_f, itau_f, hs_inv_f;  // tau, 1/tau, hs_inv in float (float kernels stay off the FP64 pipe)
    unsigned stage_off;  // TMA variant: staging buffer at or after this byte offset (1 KB of slack)
    unsigned wait_polls; // TMA variant: 0, or the test hook's polls of a barrier that never completes
};

// ---------------------------------------------------------------- TMA staging (epilogue)
// One thread arms an mbarrier with the bytes it expects and issues 3D tiled
// tensor copies (cp.async.bulk.tensor) of a group's lines into shared memory;
// every thread waits on the barrier's phase.  Waits are bounded: on expiry
// the caller records SDF_ERR_TIMEOUT and stops.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// true once phase `parity` of the barrier has completed; false after `limit` polls
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, unsigned limit) {
    for (unsigned i = 0; i < limit; ++i) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
// as mbar_wait with non-blocking polls (mbarrier.test_wait): `limit` polls
// cover a few nanoseconds each (the test hook of the expiry path)
__device__ __forceinline__ bool mbar_test(unsigned bar, unsigned parity, unsigned limit) {
    for (unsigned i = 0; i < limit; ++i) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap *map, int x, int y, int z, unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}
constexpr unsigned kTmaWaitLimit = 1u << 22;  // polls of a barrier before a wait counts as expired
constexpr int kTmaBoxRows = 256;               // rows (transform elements) per tensor copy

// TMA: the lines of a group reach shared memory by tensor copies (map
// `tmap`, box 2R floats x kTmaBoxRows rows x 1 group) into a staging buffer
// at P.stage_off, the next group's copy issued as soon as every thread has
// read the current one; otherwise each thread loads its elements itself.
template <typename T, int D, int MT, int LOGL = 0, bool TMA = false>
__global__ void __launch_bounds__(MT) k_epilogue(const cx<T> *__restrict__ in, int logL, int R, int64_t n_lines,
                                                   EpiParams P, const cx<T> *__restrict__ tw,
                                                   const __grid_constant__ CUtensorMap tmap) {
    using V = cx<T>;
    if constexpr (LOGL > 0) logL = LOGL;  // line length fixed at compile time
    extern __shared__ unsigned char smraw[];
    V *sm = reinterpret_cast<V *>(smraw);
    const int L = line_len(logL), TPL = L >> 4, PL = pad16(L);
    const int tid = threadIdx.x, lr = tid % R, t = tid / R;
    V *my = sm + lr * line_stride(PL, R, (int)sizeof(V));
    const V *tws = stage_twiddles(sm + R * line_stride(PL, R, (int)sizeof(V)), tw, L);
    const int N0 = P.N0;
    // trust threshold and capped S: one thread works them out in double (the
    // FP64 pipe is slow), the CTA reads them from shared memory
    __shared__ T s_thr[2];
    if (threadIdx.x == 0) {
        if constexpr (sizeof(T) == 4) {
            // thresholds: float is enough
            const float gn = sqrtf((float)P.dsc->sum_c2);
            const float theta64 = (float)P.coef64 * gn;
            s_thr[0] = P.fixup ? (float)P.coef32 * gn : theta64;
            s_thr[1] = -P.tau_f * logf(theta64);
        } else {
            const double gn = sqrt((double)P.dsc->sum_c2);
            const double theta64 = P.coef64 * gn;
            s_thr[0] = T(P.fixup ? P.coef32 * gn : theta64);
            s_thr[1] = T(-P.tau * log(theta64));
        }
    }
    __syncthreads();
    const T theta = s_thr[0], scap = s_thr[1];
    T tau, itau, hs_inv;
    if constexpr (sizeof(T) == 4) {
        tau = P.tau_f;
        itau = P.itau_f;
        hs_inv = P.hs_inv_f;
    } else {
        tau = P.tau;
        itau = 1.0 / P.tau;
        hs_inv = P.hs_inv;
    }
    constexpr int NH = D * (D + 1) / 2;
    T *Sout = reinterpret_cast<T *>(P.S);
    T *dS = reinterpret_cast<T *>(P.dS);
    T *d2S = reinterpret_cast<T *>(P.d2S);
    unsigned ncap = 0;      // nodes of this thread flagged CAPPED

    // TMA staging: the barrier, the buffer, the copies.  The TMA kernel is
    // persistent (CTAs stride over the blocks of R lines), and the copy of the
    // next block's first group is issued while the current block's last
    // group is transformed.
    // s_never: a barrier nothing arrives on, which the test hook's waits poll
    // (wait_polls > 0) so that they expire on their first group, whatever the
    // copies' timing
    __shared__ __align__(8) unsigned long long s_bar, s_never;
    // the buffer starts at the first 1024-byte boundary at or after stage_off
    const unsigned sbase = smem_u32(smraw);
    V *stage = reinterpret_cast<V *>(smraw + (((sbase + P.stage_off + 1023u) & ~1023u) - sbase));
    const unsigned bar = smem_u32(&s_bar), never = smem_u32(&s_never);
    const unsigned stage_bytes = (unsigned)(R * L * sizeof(V));
    const int64_t nblk = (n_lines + R - 1) / R;
    auto issue = [&](int64_t blk, int g) {  // one thread: copy group g of block blk
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, stage_bytes);
        for (int u0 = 0; u0 < L; u0 += kTmaBoxRows)
            tma_load_3d(smem_u32(stage + u0 * R), &tmap, 2 * (int)(blk * R), u0, g, bar);
    };
    bool expired = false;
    unsigned nwait = 0;  // copies waited for so far: the barrier phase
    if constexpr (TMA) {
        if (threadIdx.x == 0) {
            mbar_init(bar, 1);
            if (P.wait_polls) mbar_init(never, 1);
            if (blockIdx.x < nblk) issue(blockIdx.x, P.order[0]);
        }
        __syncthreads();
    }

    for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int64_t line = blk * R + lr;
    const bool valid = line < n_lines;
    // bin row of this line, for the fix-up's tile flags
    const int64_t brow = valid ? (int64_t)P.nb0 * (((int)(line % P.N1) >> 3) + (int64_t)P.nb1 * ((int)(line / P.N1) >> 3))
                               : 0;
    T phi[8];  // 1/phi per node, once the phi group is done
    T gs[D][8];
    unsigned sgn = 0xffu;   // bit m: +1 (no sign requested: all +1)
    unsigned trusted = 0;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        phi[m] = T(1);
#pragma unroll
        for (int a = 0; a < D; ++a) gs[a][m] = T(0);
    }
    if (P.sign_in && valid) {
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int x = t + m * TPL;
            if (x >= N0) continue;
            const int64_t node = line * N0 + x;
            const int8_t sv = P.sign_in[node];
            if (sv < 0) sgn &= ~(1u << m);
            if (P.sign) P.sign[node] = sv;
        }
    }

    for (int gi = 0; gi < P.ngroup; ++gi) {
        const int g = P.order[gi];
        V v[16];
        if constexpr (TMA) {
            const bool ok = P.wait_polls ? mbar_test(never, 0u, P.wait_polls)
                                         : mbar_wait(bar, nwait & 1u, kTmaWaitLimit);
            ++nwait;
            if (__syncthreads_or(!ok)) {  // every thread takes the same way out
                expired = true;
                break;
            }
#pragma unroll
            for (int m = 0; m < 16; ++m) v[m] = stage[(t + m * TPL) * R + lr];
            __syncthreads();  // the buffer is free again: the next copy
            if (threadIdx.x == 0) {
                if (gi + 1 < P.ngroup) issue(blk, P.order[gi + 1]);
                else if (blk + gridDim.x < nblk) issue(blk + gridDim.x, P.order[0]);
            }
        } else {
            const V *src = in + g * P.in_fs + line;
#pragma unroll
            for (int m = 0; m < 16; ++m) v[m] = valid ? src[(int64_t)(t + m * TPL) * n_lines] : mk<V>(T(0), T(0));
            __syncthreads();
        }
        fft_line<true, LOGL>(v, my, t, logL, tws);
        if (!valid) continue;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int ch = P.gch[g][half];
            if (ch == CH_NONE) continue;
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const int x = t + m * TPL;
                if (x >= N0) continue;
                const int64_t node = line * N0 + x;
                const T val = half ? v[m].y : v[m].x;
                const bool tr = (trusted >> m) & 1;
                switch (ch) {
                    case CH_MU: {
                        const bool inside = fabs(val) >= T(0.5);
                        if (!inside) sgn &= ~(1u << m);
                        if (P.sign) P.sign[node] = inside ? 1 : -1;
                        break;
                    }
                    case CH_PHI: {
                        phi[m] = T(1) / val;  // kept as 1/phi: every other channel divides by it
                        const bool ok = val >= theta;
                        if (ok) trusted |= 1u << m;
                        const T s = ok ? -tau * log(val) : scap;
                        const T sv = ((sgn >> m) & 1) ? s : -s;
                        if (Sout) Sout[node] = sv;
                        if (P.flags) P.flags[node] = ok ? 0 : SDF_FLAG_CAPPED;
                        ncap += ok ? 0u : 1u;
                        if (!ok && P.fixup && P.tile_flag) P.tile_flag[brow + (x >> 3)] = 1;
                        break;
                    }
                    case CH_GX:
                    case CH_GY:
                    case CH_GZ: {
                        const int a = ch - CH_GX;
                        const T gv = tr ? val * phi[m] : T(0);
                        if (a == 0) gs[0][m] = gv;
                        if (D > 1 && a == 1) gs[1][m] = gv;
                        if (D > 2 && a == 2) gs[D - 1][m] = gv;
                        if (dS) dS[a * P.nnodes + node] = gv;
                        break;
                    }
                    default: {
                        // Hessian channel: num/phi + S_a S_b / tau
                        int a = 0, b = 0, c = 0;
                        switch (ch) {
                            case CH_HXX: a = 0; b = 0; c = 0; break;
                            case CH_HYY: a = 1; b = 1; c = 1; break;
                            case CH_HZZ: a = 2; b = 2; c = 2; break;
                            case CH_HXY: a = 0; b = 1; c = D; break;
                            case CH_HXZ: a = 0; b = 2; c = 4; break;
                            default: a = 1; b = 2; c = 5; break;
                        }
                        T ga = gs[0][m], gb = gs[0][m];
                        if (a == 1) ga = gs[1][m];
                        if (D > 2 && a == 2) ga = gs[D - 1][m];
                        if (b == 1) gb = gs[1][m];
                        if (D > 2 && b == 2) gb = gs[D - 1][m];
                        const T hv = tr ? (val * hs_inv) * phi[m] + ga * gb * itau : T(0);
                        if (d2S && c < NH) d2S[c * P.nnodes + node] = hv;
                        break;
                    }
                }
            }
        }
    }
    if (expired) break;
    }  // blocks of lines
    if constexpr (TMA) {
        if (expired) {
            // record the expiry; let the copy in flight land (bounded) before
            // the CTA leaves: one copy at a time, the one the failed wait
            // (number nwait - 1) was for
            if (threadIdx.x == 0) atomicCAS(&P.dsc_w->status, 0, (int)SDF_ERR_TIMEOUT);
            mbar_wait(bar, (nwait - 1u) & 1u, kTmaWaitLimit);
            return;
        }
    }
    // capped nodes (the FP32 fix-up takes back the ones it recomputes)
    ncap = __reduce_add_sync(__activemask(), ncap);  // the last warp of a CTA may be partial
    if ((threadIdx.x & 31) == 0 && ncap) atomicAdd(&P.dsc_w->n_capped, (unsigned long long)ncap);
}

// ---------------------------------------------------------------- launch helpers
template <typename T>
static inline cudaError_t set_smem(const void *fn, size_t bytes) {
    if (bytes > 48 * 1024) return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return cudaSuccess;
}

constexpr size_t kSmemBudget = 200 * 1024;

// Lines per CTA of a transposed pass: the plan's tuning when set and valid,
// else pick_R.
template <typename T>
static inline int tuned_R(const sdf_plan_impl *p, int logL, int maxthr = max_threads<T>()) {
    const int def = pick_R(logL, sizeof(cx<T>), maxthr, 16, kSmemBudget);
    if (!p || p->tune_RT <= 0) return def;
    const int TPL = line_len(logL) >> 4;
    int R = p->tune_RT;
    while (R > 1 && (R * TPL > maxthr || line_smem(R, line_len(logL), (int)sizeof(cx<T>)) > kSmemBudget)) R >>= 1;
    return R;
}

// The x-pass may run 1024-thread CTAs for float lines of a compile-time
// length (those variants fit 64 registers): four 4096-point lines per CTA
// write whole 32-byte sectors of the transposed output.
template <typename T>
static inline int xpass_max_threads(int logL) {
    return (sizeof(T) == 4 && logL >= 8 && logL <= 12) ? 1024 : max_threads<T>();
}

// Launch kern<T, 512, LG> (nthr <= 512).  Needs `cudaError_t e` in scope.
#define SDF_LAUNCH_MT(kern, T, LG, nthr, grid, smem, st, ...)                                   \
    do {                                                                                      \
        if ((e = set_smem<T>((const void *)kern<T, 512, LG>, smem)) != cudaSuccess) return e; \
        kern<T, 512, LG><<<(unsigned)(grid), (nthr), (smem), (st)>>>(__VA_ARGS__);             \
    } while (0)

// CALL(LG) with LG = logL for the float line lengths compiled with a fixed
// size (256 to 4096 points, and 768, 1536, 3072 = 3 * 2^k: every length the
// workloads use) and LG = 0 (the length read at run time) for the rest and
// for double.
#define SDF_BY_LOGL(T, logL, CALL)                                  \
    do {                                                            \
        if constexpr (sizeof(T) == 4) {                             \
            switch (logL) {                                         \
                case 8: CALL(8); break;                             \
                case 9: CALL(9); break;                             \
                case 10: CALL(10); break;                           \
                case 11: CALL(11); break;                           \
                case 12: CALL(12); break;                           \
                case 8 | kLineR3: CALL(8 | kLineR3); break;         \
                case 9 | kLineR3: CALL(9 | kLineR3); break;         \
                case 10 | kLineR3: CALL(10 | kLineR3); break;       \
                default: CALL(0); break;                            \
            }                                                       \
        } else {                                                    \
            CALL(0);                                                \
        }                                                           \
    } while (0)

// CALL(LG) over the compiled float line lengths only (the TMA epilogue).
#define SDF_BY_LOGL_COMPILED(logL, CALL)                      \
    do {                                                      \
        switch (logL) {                                       \
            case 8: CALL(8); break;                           \
            case 9: CALL(9); break;                           \
            case 10: CALL(10); break;                         \
            case 11: CALL(11); break;                         \
            case 12: CALL(12); break;                         \
            case 8 | kLineR3: CALL(8 | kLineR3); break;       \
            case 9 | kLineR3: CALL(9 | kLineR3); break;       \
            default: CALL(10 | kLineR3); break;               \
        }                                                     \
    } while (0)

// adj: the adjoint programme (transform of a = w/phi) instead of the forward one
static inline FusedParams make_fused_params(const sdf_plan_impl *p, bool adj = false) {
    FusedParams F;
    memset(&F, 0, sizeof(F));
    const int ng = adj ? p->adj_ngroup : p->ngroup;
    const Group *grp = adj ? p->adj_group : p->group;
    F.ngroup = ng;
    for (int g = 0; g < ng; ++g) {
        F.nterm[g] = grp[g].nterm;
        for (int k = 0; k < grp[g].nterm; ++k) {
            F.tk[g][k] = grp[g].term[k].kslot;
            F.tf[g][k] = grp[g].term[k].field;
            F.br[g][k] = grp[g].term[k].br;
            F.bi[g][k] = grp[g].term[k].bi;
            F.brf[g][k] = (float)grp[g].term[k].br;
            F.bif[g][k] = (float)grp[g].term[k].bi;
        }
    }
    for (size_t s = 0; s < p->kernels.size() && s < (size_t)kMaxKernels; ++s) {
        F.kc[s] = p->kernels[s].c;
        F.kpar[s] = p->kernels[s].parity;
    }
    F.D = p->D;
    F.M0 = (int)p->M[0];
    F.M1 = (int)p->M[1];
    F.nfield = p->nfield;
    F.Hp = spec_row_len(p);
    return F;
}

// Launch one variant of the fused pass (defined, and explicitly instantiated
// for every variant fused_step launches, in passes_fused_kern.cuh's users).
template <typename T, int DD, int FVV, int LG>
cudaError_t run_fused(unsigned grid, int nthr, size_t smem, cudaStream_t st, const cx<T> *fin, cx<T> *fout, int logL,
                      int n_in, int n_out, int R, int64_t n_lines, int64_t in_fs, int64_t out_fs, const FusedParams &F,
                      const cx<T> *twl, const FusedParams &F1, cx<T> *fout1);
template <typename T, int LG>
cudaError_t run_fused2p(unsigned grid, int nthr, size_t smem, cudaStream_t st, const cx<T> *fin, cx<T> *fout,
                        int logL, int n_in, int n_out, int64_t in_fs, int64_t out_fs, const FusedParams &F, int nker,
                        const cx<T> *twl);

// The fused pass (passes_fused.cu): forward along the last axis, multiply by
// the kernel spectra, inverse; dense: the adjoint programme.
template <typename T>
cudaError_t fused_step(sdf_plan_impl *p, const cx<T> *fin, cx<T> *fout, int logL, int n_in, int64_t n_lines,
                       int64_t in_fs, bool dense, bool skip_mu = false, const sdf_plan_impl *p1 = nullptr,
                       cx<T> *fout1 = nullptr);

}  // namespace sdf
