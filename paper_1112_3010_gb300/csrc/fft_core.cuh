// fft_core.cuh -- the FFT building block shared by every transform pass.
//
// One CTA transforms R lines of length L = 2^k (16 <= L <= 8192) or
// L = 3 * 2^k (48 <= L <= 6144; see fft_line_r3) at once.
// Each line gets TPL = L/16 threads; thread t of a line owns the 16 elements
// t + m*TPL (m = 0..15) both on entry and on exit, so a forward transform's
// output registers feed an inverse transform's input registers directly (the
// fused spectrum multiply relies on this).
//
// The transform is a radix-16 Stockham auto-sort FFT: stage s (span Ns =
// 16^s) reads x[j + r*L/16], multiplies by w_{16 Ns}^{r (j mod Ns)}, does a
// 16-point DFT in registers (radix-4 x radix-4) and writes
// y[(j/Ns)*16*Ns + (j mod Ns) + q*Ns].  When log2 L is not a multiple of 4 the
// last stage has radix 2, 4 or 8 and each thread runs 16/radix butterflies.
// Between stages data goes through shared memory with one pad element per 16
// (index e -> e + e/16), which makes the stride-16 writes of the first stage
// conflict-free.  Twiddles come from a per-length table computed in long
// double on the host (conjugated for the inverse): radix-16 stage s >= 1
// (span Ns = 16^s) keeps w_{16 Ns}^{r k} at entry r*Ns + k - 16 (r = 1..15,
// k < Ns), and a final radix-P stage (span Ns = L/P) keeps w_L^{r j} at
// r*Ns + j - 16 (r < P, j < Ns).  Neighbouring k sit side by side, so the
// lanes of a warp read neighbouring entries (no bank conflicts when the table
// is in shared memory); L - 16 entries in all.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace sdf {

template <typename T> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };

template <typename V> __device__ __forceinline__ V mk(decltype(V::x) a, decltype(V::x) b) {
    V r; r.x = a; r.y = b; return r;
}
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
    return mk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) {
    return mk<V>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename V> __device__ __forceinline__ V cscale(V a, decltype(V::x) s) { return mk<V>(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename V> __device__ __forceinline__ V mul_mi(V a) {
    return INV ? mk<V>(-a.y, a.x) : mk<V>(a.y, -a.x);
}

__host__ __device__ __forceinline__ int pad16(int e) { return e + (e >> 4); }

// log2 of a power of two.
__host__ __device__ __forceinline__ int ilog2(int64_t L) {
    int k = 0;
    while (((int64_t)1 << k) < L) ++k;
    return k;
}

// Line codes.  A line of L = 2^k points has code k; a line of L = 3 * 2^k
// points has code k | kLineR3 (its transform starts with a radix-3 stage).
constexpr int kLineR3 = 1 << 8;
__host__ __device__ __forceinline__ int line_len(int lc) { return ((lc & kLineR3) ? 3 : 1) << (lc & 0xff); }
__host__ __device__ __forceinline__ bool line_r3(int lc) { return (lc & kLineR3) != 0; }
// Code of a length 2^k or 3 * 2^k (-1 for any other length).
inline int line_code(int64_t L) {
    int k = 0;
    int64_t q = L;
    const bool r3 = (q % 3) == 0;
    if (r3) q /= 3;
    while (((int64_t)1 << k) < q) ++k;
    return (((int64_t)1 << k) == q) ? (k | (r3 ? kLineR3 : 0)) : -1;
}

// Host: the twiddle table of a line with code lc, in the layout above (h
// holds L entries, the unused tail stays zero).  Lines of L = 3Q points (Q =
// 2^k): the radix-16 and radix-P stages of Q come first and keep the table
// of a Q-point line (entries below Q - 16); the last stage, radix 3 with span
// Q, keeps w_L^{r j} (r = 1, 2; j < Q) at Q - 16 + (r - 1) Q + j.
template <typename V> inline void fill_twiddle_table(int lc, V *h) {
    using T = decltype(V::x);
    const int64_t L = line_len(lc);
    for (int64_t e = 0; e < L; ++e) h[e].x = h[e].y = T(0);
    auto put_n = [&](int64_t e, int64_t i, int64_t n) {  // w_n^i
        const long double ang = -2.0L * 3.141592653589793238462643383279502884L * (long double)i / (long double)n;
        h[e].x = (T)cosl(ang);
        h[e].y = (T)sinl(ang);
    };
    const int logQ = lc & 0xff;
    const int64_t Q = (int64_t)1 << logQ;
    const int nst = logQ >> 2, rem = logQ & 3;
    for (int s = 1; s < nst; ++s) {
        const int64_t Ns = (int64_t)1 << (4 * s);
        for (int64_t r = 1; r < 16; ++r)
            for (int64_t k = 0; k < Ns; ++k) put_n(r * Ns + k - 16, r * k * (Q / (16 * Ns)), Q);
    }
    if (rem) {
        const int64_t Ns = (int64_t)1 << (4 * nst), P = (int64_t)1 << rem;
        for (int64_t r = 1; r < P; ++r)
            for (int64_t j = 0; j < Ns; ++j) put_n(r * Ns + j - 16, r * j, Q);
    }
    if (line_r3(lc))
        for (int64_t r = 1; r < 3; ++r)
            for (int64_t j = 0; j < Q; ++j) put_n(Q - 16 + (r - 1) * Q + j, r * j, L);
}

// Shared-memory stride between the R lines of a CTA.  Threads of a warp
// interleave lines (line = tid % R), and pad16(L) is a multiple of 16, so
// without an offset all R lines would hit the same banks; an offset of
// (elements per 128 bytes)/R staggers them across the banks.
__host__ __device__ __forceinline__ int line_stride(int PL, int R, int vbytes) {
    if (R <= 1) return PL;
    const int per = 128 / vbytes;
    return PL + (per / R > 0 ? per / R : 1);
}

// Float lines keep their L-entry twiddle table in shared memory, after the
// line buffers; double lines (whose table would not fit beside an 8192-point
// line) read it from global memory.
__host__ __device__ __forceinline__ constexpr bool twiddles_in_smem(int vbytes) { return vbytes == 8; }

// Shared memory of a CTA of R lines: the R staggered line buffers, then the
// twiddle table when it is staged.
__host__ __device__ __forceinline__ size_t line_smem(int R, int L, int vbytes) {
    return ((size_t)R * line_stride(pad16(L), R, vbytes) + (twiddles_in_smem(vbytes) ? (size_t)L : 0)) *
           (size_t)vbytes;
}

// The twiddle table fft_line reads: for float, copied to dst (shared memory
// following the line buffers) -- fft_line reads twiddles only after its first
// barrier, so no barrier is needed here; for double, the global table.
template <typename V>
__device__ __forceinline__ const V *stage_twiddles(V *dst, const V *__restrict__ tw, int L) {
    if constexpr (!twiddles_in_smem((int)sizeof(V))) {
        return tw;
    } else {
        for (int i = threadIdx.x; i < L; i += blockDim.x) dst[i] = tw[i];
        return dst;
    }
}

// Multiply by w16^K = exp(-+2 pi i K/16) for a compile-time K in [0, 16).
template <int K, bool INV, typename V> __device__ __forceinline__ V mul_w16(V a) {
    using T = decltype(V::x);
    constexpr int k = K & 15;
    const T c1 = T(0.92387953251128675613), s1 = T(0.38268343236508977173), c2 = T(0.70710678118654752440);
    if constexpr (k == 0) return a;
    else if constexpr (k == 4) return mul_mi<INV>(a);
    else if constexpr (k == 8) return mk<V>(-a.x, -a.y);
    else if constexpr (k == 12) return mul_mi<!INV>(a);
    else {
        // forward w16^k = cos(pi k/8) - i sin(pi k/8)
        constexpr int kk = k;
        T c, s;
        if constexpr (kk == 1) { c = c1; s = s1; }
        else if constexpr (kk == 2) { c = c2; s = c2; }
        else if constexpr (kk == 3) { c = s1; s = c1; }
        else if constexpr (kk == 5) { c = -s1; s = c1; }
        else if constexpr (kk == 6) { c = -c2; s = c2; }
        else if constexpr (kk == 7) { c = -c1; s = s1; }
        else if constexpr (kk == 9) { c = -c1; s = -s1; }
        else if constexpr (kk == 10) { c = -c2; s = -c2; }
        else if constexpr (kk == 11) { c = -s1; s = -c1; }
        else if constexpr (kk == 13) { c = s1; s = -c1; }
        else if constexpr (kk == 14) { c = c2; s = -c2; }
        else { c = c1; s = -s1; } // 15
        if (INV) s = -s;
        // (a.x + i a.y)(c - i s)
        return mk<V>(a.x * c + a.y * s, a.y * c - a.x * s);
    }
}

// 4-point DFT in place, natural order.
template <bool INV, typename V> __device__ __forceinline__ void dft4(V &a, V &b, V &c, V &d) {
    V t0 = cadd(a, c), t1 = csub(a, c), t2 = cadd(b, d), t3 = mul_mi<INV>(csub(b, d));
    a = cadd(t0, t2);
    c = csub(t0, t2);
    b = cadd(t1, t3);
    d = csub(t1, t3);
}

// 3-point DFT in place, natural order: y_q = sum_r x_r w3^{rq}, w3 = e^{-+2 pi i/3}.
template <bool INV, typename V> __device__ __forceinline__ void dft3(V &a, V &b, V &c) {
    using T = decltype(V::x);
    const T h3 = T(0.86602540378443864676);  // sqrt(3)/2
    const V s = cadd(b, c), d = csub(b, c);
    const V m = mk<V>(a.x - T(0.5) * s.x, a.y - T(0.5) * s.y);
    // forward: y1 = m - i h3 d, y2 = m + i h3 d (inverse: the other way)
    const V id = INV ? mk<V>(-h3 * d.y, h3 * d.x) : mk<V>(h3 * d.y, -h3 * d.x);
    a = cadd(a, s);
    b = cadd(m, id);
    c = csub(m, id);
}

template <bool INV, typename V> __device__ __forceinline__ void dft2(V &a, V &b) {
    V t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

// 16-point DFT of a[0..15] in place, natural order.
// n = 4 n1 + n2, k = k1 + 4 k2:  X[k] = sum_n2 w4^{n2 k2} w16^{n2 k1} sum_n1 x[4 n1 + n2] w4^{n1 k1}
template <bool INV, typename V> __device__ __forceinline__ void dft16(V (&a)[16]) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(a[n2], a[4 + n2], a[8 + n2], a[12 + n2]);
    // now a[4 k1 + n2] = Y[n2][k1]; twiddle by w16^{n2 k1}
    a[5] = mul_w16<1, INV>(a[5]);
    a[9] = mul_w16<2, INV>(a[9]);
    a[13] = mul_w16<3, INV>(a[13]);
    a[6] = mul_w16<2, INV>(a[6]);
    a[10] = mul_w16<4, INV>(a[10]);
    a[14] = mul_w16<6, INV>(a[14]);
    a[7] = mul_w16<3, INV>(a[7]);
    a[11] = mul_w16<6, INV>(a[11]);
    a[15] = mul_w16<9, INV>(a[15]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(a[4 * k1], a[4 * k1 + 1], a[4 * k1 + 2], a[4 * k1 + 3]);
    // a[4 k1 + k2] = X[k1 + 4 k2]; transpose to natural order
    V b[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) b[q] = a[4 * (q & 3) + (q >> 2)];
#pragma unroll
    for (int q = 0; q < 16; ++q) a[q] = b[q];
}

// 8-point DFT of x[e] = a[b0 + e*S] (e = 0..7), in place, natural order.
template <bool INV, int S, typename V> __device__ __forceinline__ void dft8s(V *a) {
    // n = 2 n1 + n2, k = k1 + 4 k2
#pragma unroll
    for (int n2 = 0; n2 < 2; ++n2) dft4<INV>(a[n2 * S], a[(2 + n2) * S], a[(4 + n2) * S], a[(6 + n2) * S]);
    // a[(2 k1 + n2) S] = Y[n2][k1]; twiddle n2 = 1 by w8^{k1} = w16^{2 k1}
    a[3 * S] = mul_w16<2, INV>(a[3 * S]);
    a[5 * S] = mul_w16<4, INV>(a[5 * S]);
    a[7 * S] = mul_w16<6, INV>(a[7 * S]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft2<INV>(a[(2 * k1) * S], a[(2 * k1 + 1) * S]);
    // a[(2 k1 + k2) S] = X[k1 + 4 k2]
    V b[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) b[q] = a[(2 * (q & 3) + (q >> 2)) * S];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q * S] = b[q];
}

// Float lines: the butterflies' complex adds as packed FP32x2 on the (re, im)
// pair a register already holds (sm_100+); a product by -i or +i becomes a
// component swap with a +-1 packed multiply-add.  Each lane rounds exactly as
// the scalar add it replaces.
__device__ __forceinline__ float2 p2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p2sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
// a + (sx b.y, sy b.x)
__device__ __forceinline__ float2 p2addsw(float2 a, float2 b, float sx, float sy) {
    return __ffma2_rn(make_float2(b.y, b.x), make_float2(sx, sy), a);
}
template <> __device__ __forceinline__ void dft4<false, float2>(float2 &a, float2 &b, float2 &c, float2 &d) {
    const float2 t0 = p2add(a, c), t1 = p2sub(a, c), t2 = p2add(b, d), t3 = p2sub(b, d);
    a = p2add(t0, t2);
    c = p2sub(t0, t2);
    b = p2addsw(t1, t3, 1.f, -1.f);  // t1 + (-i) t3
    d = p2addsw(t1, t3, -1.f, 1.f);  // t1 - (-i) t3
}
template <> __device__ __forceinline__ void dft4<true, float2>(float2 &a, float2 &b, float2 &c, float2 &d) {
    const float2 t0 = p2add(a, c), t1 = p2sub(a, c), t2 = p2add(b, d), t3 = p2sub(b, d);
    a = p2add(t0, t2);
    c = p2sub(t0, t2);
    b = p2addsw(t1, t3, -1.f, 1.f);  // t1 + i t3
    d = p2addsw(t1, t3, 1.f, -1.f);  // t1 - i t3
}
template <> __device__ __forceinline__ void dft2<false, float2>(float2 &a, float2 &b) {
    const float2 t = a;
    a = p2add(t, b);
    b = p2sub(t, b);
}
template <> __device__ __forceinline__ void dft2<true, float2>(float2 &a, float2 &b) {
    const float2 t = a;
    a = p2add(t, b);
    b = p2sub(t, b);
}

template <typename V> __device__ __forceinline__ V ldtw(const V *tw, int i) { return tw[i]; }

// Final stage of radix P (2, 4 or 8): Ns = L/P, thread t runs butterflies
// j = t + b*TPL (b < 16/P) on registers v[b + r*(16/P)].
template <int P, bool INV, typename V>
__device__ __forceinline__ void final_stage(V (&v)[16], int t, int TPL, int Ns, const V *__restrict__ tw) {
    constexpr int B = 16 / P;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = t + b * TPL;  // < Ns, so k = j
#pragma unroll
        for (int r = 1; r < P; ++r) {
            V w = ldtw(tw, r * Ns + j - 16);
            v[b + r * B] = INV ? cmulc(v[b + r * B], w) : cmul(v[b + r * B], w);
        }
        if constexpr (P == 2) {
            dft2<INV>(v[b], v[b + B]);
        } else if constexpr (P == 4) {
            dft4<INV>(v[b], v[b + B], v[b + 2 * B], v[b + 3 * B]);
        } else {
            dft8s<INV, B>(&v[b]);
        }
    }
}

// One radix-16 stage (span Ns = 2^logNs) of an L-point line, then the
// exchange through shared memory.  Addresses use pad16(a + 16 c) =
// pad16(a) + 17 c: the stores of stage 0 go to 17 t + q, those of later
// stages (Ns a multiple of 16) to pad16(base) + q * 17 Ns/16, and the loads to
// pad16(t) + m * 17 TPL/16 when TPL is a multiple of 16.  Returns false when
// this was the last stage (the result stays in v).
template <bool INV, typename V>
__device__ __forceinline__ bool fft_stage16(V (&v)[16], V *sm, int t, int logL, int logNs, bool last,
                                            const V *__restrict__ tw) {
    const int TPL = (1 << logL) >> 4;
    const int Ns = 1 << logNs;
    const int k = t & (Ns - 1);
    if (logNs > 0) {
        const V *ts = tw + (k - 16);  // w_{16 Ns}^{r k} at ts[r * Ns]
#pragma unroll
        for (int r = 1; r < 16; ++r) {
            V w = ldtw(ts, r * Ns);
            v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
        }
    }
    dft16<INV>(v);
    if (last) return false;  // Ns*16 == L: v[q] = X[t + q*TPL]
    __syncthreads();
    if (logNs == 0) {
        V *d = sm + 17 * t;
#pragma unroll
        for (int q = 0; q < 16; ++q) d[q] = v[q];
    } else {
        const int base = ((t - k) << 4) + k;
        const int st = Ns + (Ns >> 4);
        V *d = sm + pad16(base);
#pragma unroll
        for (int q = 0; q < 16; ++q) d[q * st] = v[q];
    }
    __syncthreads();
    if (TPL >= 16) {
        const V *s = sm + pad16(t);
        const int st = TPL + (TPL >> 4);
#pragma unroll
        for (int m = 0; m < 16; ++m) v[m] = s[m * st];
    } else {
#pragma unroll
        for (int m = 0; m < 16; ++m) v[m] = sm[pad16(t + m * TPL)];
    }
    return true;
}

// L = 3Q point line, Q = 2^lg.  The radix-16 stages of Q (spans 1, 16, ...)
// and, when lg is not a multiple of 4, a radix-P stage (P = 2, 4, 8) run as
// for a Q-point line -- the Stockham stage formula holds for any L the radix
// divides -- but the last of them stores its outputs to shared memory
// instead of the registers; the radix-3 stage (span Q, twiddles w_L^{r j})
// then works in place there, one butterfly (y[j], y[j + Q], y[j + 2Q]) at a
// time (Q butterflies over L/16 threads: up to 6 each), and every thread
// loads its 16 outputs X[t + m L/16].  LG > 0 fixes lg at compile time.
template <bool INV, int LG = 0, typename V>
__device__ __forceinline__ void fft_line_r3(V (&v)[16], V *sm, int t, int lg, const V *__restrict__ tw) {
    if constexpr (LG > 0) lg = LG;
    const int L = 3 << lg, TPL = L >> 4, Q = 1 << lg;
    const int nst = lg >> 2, rem = lg & 3;
    auto load_canon = [&]() {
        __syncthreads();
        if (TPL % 16 == 0) {
            const V *s0 = sm + pad16(t);
            const int st = TPL + (TPL >> 4);
#pragma unroll
            for (int m = 0; m < 16; ++m) v[m] = s0[m * st];
        } else {
#pragma unroll
            for (int m = 0; m < 16; ++m) v[m] = sm[pad16(t + m * TPL)];
        }
    };
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        if (s >= nst) break;
        const int Ns = 1 << (4 * s);
        const int k = t & (Ns - 1);
        if (s > 0) {
            const V *ts = tw + (k - 16);  // w_{16 Ns}^{r k} at ts[r * Ns]
#pragma unroll
            for (int r = 1; r < 16; ++r) {
                V w = ldtw(ts, r * Ns);
                v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
            }
        }
        dft16<INV>(v);
        __syncthreads();
        const int base = ((t - k) << 4) + k;
#pragma unroll
        for (int q = 0; q < 16; ++q) sm[pad16(base + q * Ns)] = v[q];
        if (s + 1 < nst || rem) load_canon();
    }
    if (rem) {
        // radix-P stage, span Ns = 16^nst (not the last): butterflies j = t + b TPL
        const int P = 1 << rem, B = 16 / P, Ns = 1 << (4 * nst);
#pragma unroll
        for (int b = 0; b < 16; ++b) {
            if (b >= B) break;
            const int j = t + b * TPL, k = j & (Ns - 1);
#pragma unroll
            for (int r = 1; r < 8; ++r) {
                if (r >= P) break;
                V w = ldtw(tw, r * Ns + k - 16);  // w_{P Ns}^{r k}
                v[b + r * B] = INV ? cmulc(v[b + r * B], w) : cmul(v[b + r * B], w);
            }
        }
        if (P == 2) {
#pragma unroll
            for (int b = 0; b < 8; ++b) dft2<INV>(v[b], v[b + 8]);
        } else if (P == 4) {
#pragma unroll
            for (int b = 0; b < 4; ++b) dft4<INV>(v[b], v[b + 4], v[b + 8], v[b + 12]);
        } else {
#pragma unroll
            for (int b = 0; b < 2; ++b) dft8s<INV, 2>(&v[b]);
        }
        __syncthreads();
#pragma unroll
        for (int b = 0; b < 16; ++b) {
            if (b >= B) break;
            const int j = t + b * TPL, k = j & (Ns - 1);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (q >= P) break;
                sm[pad16((j - k) * P + k + q * Ns)] = v[b + q * B];
            }
        }
    }
    __syncthreads();
    // radix 3 in place: X[j + q Q] = sum_r w3^{rq} w_L^{rj} y[j + r Q]
    const V *t1 = tw + (Q - 16), *t2 = tw + (2 * Q - 16);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const int j = t + i * TPL;
        if (j < Q) {
            V a0 = sm[pad16(j)], a1 = sm[pad16(j + Q)], a2 = sm[pad16(j + 2 * Q)];
            const V w1 = ldtw(t1, j), w2 = ldtw(t2, j);
            a1 = INV ? cmulc(a1, w1) : cmul(a1, w1);
            a2 = INV ? cmulc(a2, w2) : cmul(a2, w2);
            dft3<INV>(a0, a1, a2);
            sm[pad16(j)] = a0;
            sm[pad16(j + Q)] = a1;
            sm[pad16(j + 2 * Q)] = a2;
        }
    }
    load_canon();
}

// L-point FFT (forward: exp(-2 pi i nk/L); inverse: exp(+2 pi i nk/L), not
// normalised) of one line.  On entry v[m] = x[t + m*TPL]; on exit
// v[m] = X[t + m*TPL].  `sm` is this line's shared buffer of pad16(L) elements.
// logL is a line code (line_len): L = 2^logL, or 3 * 2^k for k | kLineR3.
// Every thread of the CTA must call this with the same logL (it synchronises).
// `tw` is the table of L twiddles (shared memory for float, global for double).
// LOGL > 0 fixes log2 L at compile time (logL is then ignored): every stage is
// unrolled, addresses become immediates, and inputs known to be zero or
// outputs never read cost nothing.
template <bool INV, int LOGL = 0, typename V>
__device__ __forceinline__ void fft_line(V (&v)[16], V *sm, int t, int logL, const V *__restrict__ tw) {
    if constexpr (LOGL > 0 && (LOGL & kLineR3) != 0) {
        fft_line_r3<INV, (LOGL & 0xff)>(v, sm, t, LOGL & 0xff, tw);
    } else if constexpr (LOGL > 0) {
        constexpr int nst = LOGL >> 2, rem = LOGL & 3;
#pragma unroll
        for (int s = 0; s < nst; ++s)
            if (!fft_stage16<INV>(v, sm, t, LOGL, 4 * s, s == nst - 1 && rem == 0, tw)) return;
        constexpr int TPL = (1 << LOGL) >> 4, Ns = 1 << (4 * nst);
        if constexpr (rem == 1) final_stage<2, INV>(v, t, TPL, Ns, tw);
        else if constexpr (rem == 2) final_stage<4, INV>(v, t, TPL, Ns, tw);
        else if constexpr (rem == 3) final_stage<8, INV>(v, t, TPL, Ns, tw);
    } else {
        if (line_r3(logL)) {
            fft_line_r3<INV>(v, sm, t, logL & 0xff, tw);
            return;
        }
        const int TPL = (1 << logL) >> 4;
        const int nst = logL >> 2, rem = logL & 3;
        for (int s = 0; s < nst; ++s)
            if (!fft_stage16<INV>(v, sm, t, logL, 4 * s, s == nst - 1 && rem == 0, tw)) return;
        const int Ns = 1 << (4 * nst);
        if (rem == 1) final_stage<2, INV>(v, t, TPL, Ns, tw);
        else if (rem == 2) final_stage<4, INV>(v, t, TPL, Ns, tw);
        else if (rem == 3) final_stage<8, INV>(v, t, TPL, Ns, tw);
    }
}

}  // namespace sdf
