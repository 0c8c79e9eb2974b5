// line1d.cu -- the whole path for D = 1 in one CTA (Sec. 2.1 treats 1D like
// 2D and 3D; Table 1 with a single axis).  The padded line (M <= 4096 nodes)
// lives in shared memory, so the steps need no trip through HBM:
//   snap + count     the points to node counts m_j (Sec. 6 rounding)
//   forward FFT      of the count line (Table 1 step 3)
//   multiply         phi and d phi packed in one complex product: the kernel
//                    f is even and its derivative kernel n E odd, so with the
//                    compressed real spectra c_f, c_g,
//                    F (c_f + s(k) c_g), s(k) = +1 for k <= M/2, -1 above,
//                    inverts to phi + i (n E * m)  (Table 1 step 4)
//   inverse FFTs     that one, and F c_h for the Hessian kernel
//   epilogue         S = -tau log phi, S' = (n E * m)/phi,
//                    S'' = (h * m)/phi + S'^2/tau  (eqs. STilde, SxSy, Sxx)
//   fix-up           SDF_FP32 plans: nodes below theta_32 from the shifted
//                    direct sum over the occupied nodes (eq. Bound1), in the
//                    same CTA.
// One thread per 16 line elements (the FFT's layout), so the CTA has M/16
// threads.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sdf_internal.cuh"

namespace sdf {

struct Line1dParams {
    int64_t K;
    const double *pts;
    double h, tau;
    int N, logM;
    const void *c_phi, *c_gx, *c_hxx;  // compressed spectra, M/2 + 1 values (plan precision)
    const void *tw;                    // twiddles of the M-point line (plan precision)
    double coef64, coef32;             // theta_p = coef_p * ||m||_2
    double hs_inv;                     // 1 / stored scale of the Hessian kernel
    int fixup;                         // SDF_FP32 plan: nodes below theta_32 go to the direct sum
    int full_range;                    // ... and nodes below theta_64 too
    void *S, *dS, *d2S;
    uint8_t *flags;
    DevScalars *dsc;
};

template <typename T> using cx1 = typename cplx_t<T>::type;

__device__ __forceinline__ void line1d_status(DevScalars *d, int code) { atomicCAS(&d->status, 0, code); }

template <typename T>
__global__ void k_line1d(Line1dParams P) {
    using V = cx1<T>;
    extern __shared__ unsigned char smraw[];
    const int M = 1 << P.logM, TPL = M >> 4, N = P.N;
    V *sm = reinterpret_cast<V *>(smraw);
    int *cnt = reinterpret_cast<int *>(smraw + sizeof(V) * pad16(M));  // node counts
    int *fix = cnt + N;                                                 // nodes for the direct sum
    __shared__ int s_nfix, s_ncap, s_ncapfix;
    __shared__ unsigned long long s_c2;
    __shared__ int s_nu;
    __shared__ double s_thr[3];  // theta64, theta32, S_cap
    const int t = threadIdx.x, nt = blockDim.x;
    const V *tw = reinterpret_cast<const V *>(P.tw);

    for (int i = t; i < N; i += nt) cnt[i] = 0;
    if (t == 0) {
        s_nfix = s_ncap = s_ncapfix = s_nu = 0;
        s_c2 = 0;
    }
    __syncthreads();
    // snap: nearest node, ties up
    for (int64_t k = t; k < P.K; k += nt) {
        const double q = floor(P.pts[k] / P.h + 0.5);
        if (!(q >= 0.0 && q < (double)N)) {
            line1d_status(P.dsc, SDF_ERR_POINT_OUT_OF_GRID);
            continue;
        }
        atomicAdd(&cnt[(int)q], 1);
    }
    __syncthreads();
    // ||m||_2^2 and the occupied-node count (shared atomics: the CTA may be
    // narrower than a warp)
    unsigned long long c2 = 0;
    int nu = 0;
    for (int i = t; i < N; i += nt) {
        const unsigned long long c = (unsigned)cnt[i];
        c2 += c * c;
        nu += c > 0;
    }
    atomicAdd(&s_c2, c2);
    atomicAdd(&s_nu, nu);
    __syncthreads();
    if (t == 0) {
        P.dsc->sum_c2 = s_c2;
        P.dsc->n_unique = s_nu;
        const double gn = sqrt((double)s_c2);
        s_thr[0] = P.coef64 * gn;
        s_thr[1] = P.coef32 * gn;
        s_thr[2] = -P.tau * log(s_thr[0]);
    }
    // forward transform of the counts (the barrier inside orders the reads
    // of s_thr and cnt after the writes above)
    V v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const int x = t + m * TPL;
        v[m] = mk<V>(x < N ? T(cnt[x]) : T(0), T(0));
    }
    __syncthreads();
    fft_line<false>(v, sm, t, P.logM, tw);
    // v[m] = F(k), k = t + m TPL
    const T *cf = reinterpret_cast<const T *>(P.c_phi);
    const T *cg = reinterpret_cast<const T *>(P.c_gx);
    const T *ch = reinterpret_cast<const T *>(P.c_hxx);
    T hv[16];
    if (ch) {
        V w[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            const int k = t + m * TPL;
            const T c = ch[k <= M / 2 ? k : M - k];
            w[m] = mk<V>(v[m].x * c, v[m].y * c);
        }
        fft_line<true>(w, sm, t, P.logM, tw);
#pragma unroll
        for (int m = 0; m < 16; ++m) hv[m] = w[m].x * T(P.hs_inv);
    }
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const int k = t + m * TPL;
        const int f = k <= M / 2 ? k : M - k;
        T c = cf[f];
        if (cg) c += (k <= M / 2 ? cg[f] : -cg[f]);
        v[m] = mk<V>(v[m].x * c, v[m].y * c);
    }
    fft_line<true>(v, sm, t, P.logM, tw);

    const T theta64 = T(s_thr[0]), theta32 = T(s_thr[1]), scap = T(s_thr[2]);
    const T tau = T(P.tau), itau = T(1.0 / P.tau);
    const T theta = P.fixup ? theta32 : theta64;
    T *Sout = reinterpret_cast<T *>(P.S);
    T *dS = reinterpret_cast<T *>(P.dS);
    T *d2S = reinterpret_cast<T *>(P.d2S);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const int x = t + m * TPL;
        if (x >= N) continue;
        const T phi = v[m].x;
        uint8_t fl = cnt[x] > 0 ? SDF_FLAG_SOURCE : 0;
        if (phi >= theta) {
            const T g = v[m].y / phi;
            if (Sout) Sout[x] = -tau * log(phi);
            if (dS) dS[x] = g;
            if (d2S) d2S[x] = hv[m] / phi + g * g * itau;
        } else if (P.fixup) {
            // the float transform cannot tell phi from noise here: the direct
            // sum below decides (and caps below theta_64 unless full range)
            fix[atomicAdd(&s_nfix, 1)] = x;
            fl |= SDF_FLAG_FIXUP;
        } else {
            atomicAdd(&s_ncap, 1);
            if (Sout) Sout[x] = scap;
            if (dS) dS[x] = T(0);
            if (d2S) d2S[x] = T(0);
            fl |= SDF_FLAG_CAPPED;
        }
        if (P.flags) P.flags[x] = fl;
    }
    __syncthreads();
    const int nfix = s_nfix;
    if (t == 0) P.dsc->n_fixup_tiles = nfix > 0 ? 1ull : 0ull;
    if (nfix == 0) {
        if (t == 0) P.dsc->n_capped = (unsigned long long)s_ncap;
        return;
    }
    // the occupied nodes in order, as (position, count) pairs: each thread
    // lists one contiguous chunk, thread 0 turns the chunk sizes into offsets
    int2 *occ = reinterpret_cast<int2 *>(fix + N);
    __shared__ int s_part[256];
    const int chunk = (N + nt - 1) / nt, i0 = min(N, t * chunk), i1 = min(N, i0 + chunk);
    int mine = 0;
    for (int i = i0; i < i1; ++i) mine += cnt[i] > 0;
    s_part[t] = mine;
    __syncthreads();
    if (t == 0) {
        int acc = 0;
        for (int w = 0; w < nt; ++w) {
            const int c = s_part[w];
            s_part[w] = acc;
            acc += c;
        }
    }
    __syncthreads();
    for (int i = i0, o = s_part[t]; i < i1; ++i)
        if (cnt[i] > 0) occ[o++] = make_int2(i, cnt[i]);
    __syncthreads();
    const int nocc = s_nu;
    // direct sum, shifted by the distance R to the nearest occupied node
    // (eq. Bound1): phi e^{R/tau} = sum_j m_j e^{-(r_j - R)/tau}, in units of h
    const float hf = (float)P.h, itf = (float)(P.h / P.tau), tf = (float)P.tau;
    unsigned long long terms = 0;
    for (int i = t; i < nfix; i += nt) {
        const int x = fix[i];
        // nearest occupied node: the first position >= x or the one before it
        int lo = 0, hi = nocc;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (occ[mid].x < x) lo = mid + 1;
            else hi = mid;
        }
        int dmin = 1 << 30;
        if (lo < nocc) dmin = occ[lo].x - x;
        if (lo > 0) dmin = min(dmin, x - occ[lo - 1].x);
        // outward from there while a term can still matter: past 60 tau
        // beyond the nearest node it is below e^-60 of the leading term
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        auto add = [&](const int2 q) {
            const int d = x - q.x;
            const float e = (float)q.y * __expf(-(float)(abs(d) - dmin) * itf);
            s0 += e;
            if (d != 0) {
                s1 += d > 0 ? e : -e;  // n E with n = sign(x - y)
                s2 += e;               // the Hessian kernel is -E/tau off the origin
            }
            ++terms;
        };
        const float cut = 60.f / itf;  // 60 tau in nodes
        const unsigned long long terms0 = terms;
        for (int j = lo; j < nocc && (float)(occ[j].x - x - dmin) <= cut; ++j) add(occ[j]);
        for (int j = lo - 1; j >= 0 && (float)(x - occ[j].x - dmin) <= cut; --j) add(occ[j]);
        atomicMax(&P.dsc->fix_nmax, terms - terms0);  // for the error report
        const float Sx = (float)dmin * hf - tf * logf(s0);
        if (!P.full_range && Sx > (float)scap) {  // phi below theta_64
            atomicAdd(&s_ncap, 1);
            atomicAdd(&s_ncapfix, 1);
            if (Sout) Sout[x] = scap;
            if (dS) dS[x] = T(0);
            if (d2S) d2S[x] = T(0);
            if (P.flags) P.flags[x] = (cnt[x] > 0 ? SDF_FLAG_SOURCE : 0) | SDF_FLAG_CAPPED;
            continue;
        }
        const float g = s1 / s0;
        if (Sout) Sout[x] = T(Sx);
        if (dS) dS[x] = T(g);
        if (d2S) d2S[x] = T((g * g - s2 / s0) / tf);
    }
    __syncthreads();
    if (t == 0) {
        // as in 2D: the nodes the direct sum wrote, and every capped node
        P.dsc->n_fixup_nodes = (unsigned long long)(nfix - s_ncapfix);
        P.dsc->n_capped = (unsigned long long)s_ncap;
    }
    if (terms) atomicAdd(&P.dsc->n_fixup_terms, terms);
}

cudaError_t launch_line1d(sdf_plan_impl *p, int64_t K, const double *points, void *S, void *dS, void *d2S,
                          uint8_t *flags) {
    cudaError_t e;
    cudaStream_t st = p->stream;
    // clear the per-execute scalars but keep `status` (reported by sdf_sync)
    if ((e = cudaMemsetAsync(reinterpret_cast<char *>(p->dsc) + offsetof(DevScalars, wmax), 0,
                             sizeof(DevScalars) - offsetof(DevScalars, wmax), st)) != cudaSuccess)
        return e;
    Line1dParams P;
    P.K = K;
    P.pts = points;
    P.h = p->h;
    P.tau = p->tau;
    P.N = (int)p->N[0];
    P.logM = p->logM[0];
    auto spec = [&](int id) -> const void * { return p->kslot[id] >= 0 ? p->kernels[p->kslot[id]].c : nullptr; };
    P.c_phi = spec(KER_PHI);
    P.c_gx = (p->outputs & SDF_OUT_DS) ? spec(KER_GX) : nullptr;
    P.c_hxx = (p->outputs & SDF_OUT_D2S) && d2S ? spec(KER_HXX) : nullptr;
    P.tw = p->tw[0];
    P.coef64 = theta_coef(p, SDF_FP64);
    P.coef32 = theta_coef(p, SDF_FP32);
    P.hs_inv = 1.0 / hessian_scale(p);
    P.fixup = p->prec == SDF_FP32;
    P.full_range = p->full_range;
    P.S = S;
    P.dS = dS;
    P.d2S = d2S;
    P.flags = flags;
    P.dsc = p->dsc;
    const int M = 1 << P.logM, nt = M >> 4;
    prof_begin(p, "line1d", st);
    if (p->prec == SDF_FP64) {
        const size_t smem = sizeof(double2) * pad16(M) + (sizeof(int) * 2 + sizeof(int2)) * P.N;
        if ((e = cudaFuncSetAttribute(k_line1d<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        k_line1d<double><<<1, nt, smem, st>>>(P);
    } else {
        const size_t smem = sizeof(float2) * pad16(M) + (sizeof(int) * 2 + sizeof(int2)) * P.N;
        if ((e = cudaFuncSetAttribute(k_line1d<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        k_line1d<float><<<1, nt, smem, st>>>(P);
    }
    prof_end(p, st);
    return cudaGetLastError();
}

}  // namespace sdf
