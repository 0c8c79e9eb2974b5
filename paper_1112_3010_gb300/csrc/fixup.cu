// fixup.cu -- step A6 (SDF_FP32 plans): nodes where the float transform's phi
// fell below its trust threshold theta_32 but may lie inside the FP64 trust
// region are recomputed by a direct sum over the occupied nodes near them,
// with the log-sum-exp shift of Sec. 2.4 (eq. Bound1):
//   S = m - tau log sum_k c_k exp(-(r_k - m)/tau),   m = min_k r_k,
// plus grad S (eq. SxSy) and the Hessian (eqs. Sxx, Syy, Sxy).  The shift makes
// float arithmetic sufficient: there is no dynamic-range floor.  The paper
// motivates the problem (Sec. 3.3, double precision fails far from the points)
// but gives no mechanism; this one is ours.
//
// One CTA per flagged tile (2x2 bins of 8x8 nodes in 2D, one 8^3 bin in 3D),
// two nodes per thread so that each staged point feeds two sums; the two
// nodes are the two lanes of packed FP32x2 arithmetic (fma/mul/add.f32x2),
// which halves the FMA-pipe instructions of the summing loop.  Candidate
// bins are visited in rings of Chebyshev distance k = 0, 1, 2, ... around the
// tile (a batch of rings is listed row by row from per-row lists of the
// occupied bins, so empty bins cost nothing); every occupied node of ring k'
// lies at least (8(k'-1)+1)h from every
// node of the tile, so after ring k the unvisited points add at most
// T = sum_{k'>k} n_k' exp(-(8(k'-1)+1)h/tau), with the ring counts n_k' read
// from the bins' prefix sums for a few rings ahead (the rest all at the next
// distance).  A node stops summing once T is below 1e-5 of its sum, or once
// even its sum plus T is below theta_64 (it stays capped).  Rings go in
// batches that end at the first ring where every node of some warp could meet
// one of these tests (a bound from its sums so far): the summing loop is
// warp-uniform, so a finished warp is what saves work, and batches stay few.
// In 3D a warp also skips a staged bin when, for each of its active nodes,
// the bin's whole box lies so far out that all the batch's points there add
// under 1e-6 of the node's sum so far (the cube of rings holds many points
// outside that sphere); over a node's batches that leaves out at most 1e-6
// per batch of its final sum.  The log-sum-exp shift
// m is the nearest point found by a cheap pass over the first batch of points
// (and over a later batch only if it could hold a point so much nearer that a
// term would exceed 2^60), so the summing loop itself has no branch.  A
// tile whose nearest occupied bin is so far that K exp(-d/tau) < theta_64
// keeps the capped value.  In full-range mode nothing is capped: every node
// the float transform does not trust gets the sum, however small phi is (the
// regime the paper reaches only with multiple-precision arithmetic).  Visiting order is fixed, so the sums are
// deterministic.
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <stdint.h>

#include "sdf_internal.cuh"

namespace sdf {

struct FixParams {
    const int *bin_start, *bin_nuniq, *ucell, *ucount;
    const int *occ_start, *occ_x;  // occupied bins per bin row, x ascending
    const int *sat;  // summed-area table of the points per bin
    const unsigned char *cheb, *tile_flag;
    const DevScalars *dsc;
    DevScalars *dsc_w;
    void *S, *dS, *d2S;
    const int8_t *sign;
    uint8_t *flags;
    int N0, N1, N2;
    int nb0, nb1, nb2;
    int64_t nnodes;
    double coef64;
    float log_coef64;
    float h, tau, l2e_th, logK;  // spacing, tau, h log2(e)/tau, log K
    int full;  // full range: no capping at theta_64 (every untrusted node is summed)
};

constexpr int kFixCap = 1024;  // cells staged in shared memory at once
// bin rows listed per pass (a batch's rows are those of the box of its last ring)
template <int D> constexpr int kRowCap = (D == 2) ? 256 : 1024;

// First index in occ_x[a, b) (ascending) that is >= v.
__device__ __forceinline__ int occ_lower(const int *__restrict__ occ_x, int a, int b, int v) {
    while (a < b) {
        const int m = (a + b) >> 1;
        if (occ_x[m] < v) a = m + 1;
        else b = m;
    }
    return a;
}
constexpr int kTB2 = 2;       // 2D tile: kTB2 x kTB2 bins (16 x 16 nodes)

// Hardware approximations (PTX ex2.approx / rsqrt.approx, relative error
// about 2^-22): arguments here are never denormal (exponents lie in
// [-40, 0], squared distances are integers >= 1).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// The two nodes of a thread are the two lanes of packed FP32x2 arithmetic
// (sm_100+): lane j of an accumulator is node j's.
__device__ __forceinline__ float lane(const float2 &v, int j) { return j ? v.y : v.x; }
__device__ __forceinline__ void lane_scale(float2 &v, int j, float s) {
    if (j) v.y *= s;
    else v.x *= s;
}
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }

// Index of the pair (a, b), a <= b, in the row-by-row upper triangle.
template <int D> __device__ __forceinline__ constexpr int sym_index(int a, int b) {
    return a * D - a * (a - 1) / 2 + (b - a);
}

// LVL: 0 = S only, 1 = S and grad S, 2 = S, grad S and the Hessian (only the
// sums the requested outputs need are accumulated).
template <int D, typename TO, int LVL>
__global__ void __launch_bounds__(D == 2 ? 32 * kTB2 * kTB2 : 256, D == 2 ? 7 : (LVL == 2 ? 2 : 3)) k_fixup(FixParams P) {
    constexpr int TB = (D == 2) ? kTB2 : 1;  // tile edge in bins
    constexpr int NT = (D == 2) ? 32 * kTB2 * kTB2 : 256;
    constexpr int NH = D * (D + 1) / 2;
    constexpr int NPT = 2;                    // nodes per thread
    constexpr float kOff = (D == 2) ? 8.f : 4.f;  // second node: +kOff along the last axis
    __shared__ float4 cell[kFixCap];  // (x, y, z, count) of staged occupied nodes
    __shared__ int soff[NT + 1];      // first staged cell of each taken bin, then the total
    __shared__ int ssrc[NT];          // the bin's first entry in ucell / ucount
    __shared__ int sbin[NT];          // the bin's index
    __shared__ float4 sbox[NT];       // the bin's first node (x, y, z) and whether it holds points
    __shared__ int wtot[32];
    __shared__ int4 s_row[kRowCap<D>];  // per listed row: (first, count) of up to two runs in occ_x
    __shared__ int s_rpre[kRowCap<D>];  // per listed row: its first bin in the pass's list
    const int tid = threadIdx.x;
    const int nt0 = (P.nb0 + TB - 1) / TB, nt1 = (P.nb1 + TB - 1) / TB;
    const int64_t tile = blockIdx.x;
    const int bx = (int)(tile % nt0) * TB, by = (int)((tile / nt0) % nt1) * TB,
              bz = (int)(tile / ((int64_t)nt0 * nt1)) * TB;
    // the tile's bins: any flagged?  nearest occupied bin over all of them
    int c = 255;
    bool flagged = false;
    for (int j = 0; j < TB * TB; ++j) {
        const int qx = bx + (j % TB), qy = by + (j / TB);
        if (qx >= P.nb0 || qy >= P.nb1) continue;
        const int64_t q = qx + (int64_t)P.nb0 * (qy + (int64_t)P.nb1 * bz);
        flagged |= P.tile_flag[q] != 0;
        c = min(c, (int)P.cheb[q]);
    }
    if (!flagged) return;
    // log theta_64 = log(coef64) + log(sum c^2)/2, a threshold: float is
    // enough (the FP64 pipe is slow); one thread, read from shared memory
    __shared__ float s_lt;
    if (tid == 0) s_lt = P.log_coef64 + 0.5f * logf((float)P.dsc->sum_c2);
    __syncthreads();
    const float lt = s_lt;
    const float dlo = (c >= 1) ? (8.f * (c - 1) + 1.f) * P.h : 0.f;
    // every node of the tile: phi <= K exp(-dlo/tau) < theta64 -> stays capped
    if (!P.full && (c >= 255 || P.logK - dlo / P.tau < lt)) return;

    // this thread's nodes: (x, y, z) and the same plus kOff along y (2D) or z (3D)
    const int x = (D == 2) ? bx * 8 + (tid % (8 * TB)) : bx * 8 + (tid & 7);
    const int y = (D == 2) ? by * 8 + (tid / (8 * TB)) : by * 8 + ((tid >> 3) & 7);
    const int z = (D == 2) ? 0 : bz * 8 + (tid >> 6);
    int64_t node[NPT];
    bool mine[NPT], active[NPT], early_cap[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const int yj = (D == 2) ? y + 8 * j : y, zj = (D == 2) ? 0 : z + 4 * j;
        const bool inb = x < P.N0 && yj < P.N1 && (D == 2 || zj < P.N2);
        node[j] = (int64_t)x + (int64_t)P.N0 * (yj + (int64_t)P.N1 * zj);
        mine[j] = inb && (P.flags[node[j]] & SDF_FLAG_CAPPED) != 0;
        active[j] = mine[j];   // still summing
        early_cap[j] = false;  // shown below theta_64 before the sum finished
    }
    const float h = P.h, tau = P.tau, itau = 1.f / tau, ih = 1.f / h;
    // distances are kept in grid units (node spacing 1); exp(-(r - m)/tau) =
    // 2^((m - r) * l2e_th) with l2e_th = h log2(e)/tau
    const float l2e_th = P.l2e_th;
    // node and cell coordinates are integers below 2^13, so the squared
    // distances that matter (below 2^24) are exact in float
    const float xf = (float)x, yf = (float)y, zf = (float)z;
    // running sums per node, relative to exp(-m/tau), m the nearest occupied
    // node seen so far: sE = sum c e, sA = sum c e/r, sG_a = sum c e d_a/r,
    // sB_ab = sum c e d_a d_b (1/r_w + 1/tau)/r^2 (r in grid units, r_w = h r
    // the distance, d = node - point); then H_ab = (delta_ab sA/h - sB_ab)/sE
    // + g_a g_b/tau (eqs. Sxx, Syy, Sxy) and grad S = sG/sE (eq. SxSy)
    static_assert(NPT == 2, "two nodes per thread: the two lanes of float2");
    float mg[NPT];
    float2 mk = dup2(INFINITY), sE = dup2(0.f), sA = dup2(0.f), sG[D], sB[NH];
#pragma unroll
    for (int j = 0; j < NPT; ++j) mg[j] = INFINITY;
#pragma unroll
    for (int a = 0; a < D; ++a) sG[a] = dup2(0.f);
#pragma unroll
    for (int a = 0; a < NH; ++a) sB[a] = dup2(0.f);
    unsigned nterm = 0;

    const int kmax = max(max(P.nb0, P.nb1), (D == 3) ? P.nb2 : 0);
    // Rings are visited in batches: {0,1,2}, then up to the first ring at
    // whose end every active node of some warp could stop or be capped (a
    // lower bound worked out from its sums after the previous batch, s_kev).
    __shared__ int s_kev[2];
    // points in the box of rings <= k1 + j (j <= kLook) and the log of the
    // bound on what lies beyond ring k1 + i (i < kLook): ring k' holds
    // n_k' points, all at least 8(k'-1)+1 nodes away
    constexpr int kLook = 8;
    __shared__ int s_cnt[kLook + 1];
    __shared__ float s_logT[kLook];
    const int ktot = P.bin_start[(int64_t)P.nb0 * P.nb1 * ((D == 3) ? P.nb2 : 1)];  // points binned
    // points in the box of rings <= k around the tile, from the table
    auto box_count = [&](int k) {
        const int x0 = max(bx - k, 0) - 1, x1 = min(bx + TB - 1 + k, P.nb0 - 1);
        const int y0 = max(by - k, 0) - 1, y1 = min(by + TB - 1 + k, P.nb1 - 1);
        const int z0 = (D == 3) ? max(bz - k, 0) - 1 : -1, z1 = (D == 3) ? min(bz + k, P.nb2 - 1) : 0;
        auto at = [&](int x, int y, int z) -> int {
            return (x < 0 || y < 0 || z < 0) ? 0 : P.sat[x + (int64_t)P.nb0 * (y + (int64_t)P.nb1 * z)];
        };
        int n = at(x1, y1, z1) - at(x0, y1, z1) - at(x1, y0, z1) + at(x0, y0, z1);
        if (D == 3) n -= at(x1, y1, z0) - at(x0, y1, z0) - at(x1, y0, z0) + at(x0, y0, z0);
        return n;
    };
    if (tid == 0) s_kev[0] = s_kev[1] = INT_MAX;
    int round = 0;
    unsigned nsum = 0;  // cells this thread's loop ran over: no node of it summed more terms
    for (int k0 = 0; k0 <= kmax; ++round) {
        if (!__syncthreads_or(active[0] || active[1])) break;
        const int k1 = (k0 == 0) ? min(kmax, 2) : min(kmax, max(k0, s_kev[round & 1]));
        if (tid == 0) s_kev[(round + 1) & 1] = INT_MAX;  // this batch's checks go here
        if (tid <= kLook) s_cnt[tid] = box_count(min(k1 + tid, kmax));
        // every node of ring k0 or beyond lies at least 8(k0-1)+1 from the tile
        const float lb_in = (k0 == 0) ? 0.f : 8.f * (k0 - 1) + 1.f;
        // The batch's bins are those of rings k0..k1: the occupied bins of the
        // rows (y[, z]) of ring k1's box, whole x runs for rows at ring
        // distance >= k0 in (y, z), else the two x runs at distance k0..k1.
        // Rows go in passes of at most kRowCap; each thread lists a run of
        // consecutive rows, so the bins come in row order (deterministic).
        const int ylo = max(by - k1, 0), yhi = min(by + TB - 1 + k1, P.nb1 - 1);
        const int zlo = (D == 3) ? max(bz - k1, 0) : 0, zhi = (D == 3) ? min(bz + k1, P.nb2 - 1) : 0;
        const int ny = yhi - ylo + 1, nrow_all = ny * (zhi - zlo + 1);
        for (int r0 = 0; r0 < nrow_all; r0 += kRowCap<D>) {
        const int npass = min(kRowCap<D>, nrow_all - r0);
        const int rpt = (npass + NT - 1) / NT;
        int cnt_t = 0;
        for (int q = 0; q < rpt; ++q) {
            const int lr = tid * rpt + q;
            if (lr >= npass) break;
            const int r = r0 + lr;
            const int qy = ylo + r % ny, qz = zlo + r / ny;
            const int row = qy + P.nb1 * qz;
            int dyz = max(max(by - qy, qy - (by + TB - 1)), 0);
            if (D == 3) dyz = max(dyz, max(bz - qz, qz - bz));
            const int a = P.occ_start[row], b = P.occ_start[row + 1];
            int4 rg = make_int4(a, 0, a, 0);
            if (a < b) {
                if (dyz >= k0) {
                    const int lo = occ_lower(P.occ_x, a, b, bx - k1);
                    rg.x = lo;
                    rg.y = occ_lower(P.occ_x, lo, b, bx + TB + k1) - lo;
                } else {
                    const int lo = occ_lower(P.occ_x, a, b, bx - k1);
                    rg.x = lo;
                    rg.y = occ_lower(P.occ_x, lo, b, bx - k0 + 1) - lo;
                    const int lo2 = occ_lower(P.occ_x, lo + rg.y, b, bx + TB - 1 + k0);
                    rg.z = lo2;
                    rg.w = occ_lower(P.occ_x, lo2, b, bx + TB + k1) - lo2;
                }
            }
            s_row[lr] = rg;
            s_rpre[lr] = cnt_t;
            cnt_t += rg.y + rg.w;
        }
        int nlist = 0;
        {
            // block exclusive scan of the threads' bin counts
            const int lane = tid & 31, wid = tid >> 5;
            int incl = cnt_t;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            __syncthreads();  // wtot is free (its last readers are past a barrier)
            if (lane == 31) wtot[wid] = incl;
            __syncthreads();
            int woff = 0;
            for (int w = 0; w < NT / 32; ++w) {
                const int t = wtot[w];
                if (w < wid) woff += t;
                nlist += t;
            }
            const int off = woff + incl - cnt_t;
            for (int q = 0; q < rpt; ++q) {
                const int lr = tid * rpt + q;
                if (lr >= npass) break;
                s_rpre[lr] += off;
            }
            __syncthreads();
        }
        for (int i0 = 0; i0 < nlist;) {
            // one listed bin per thread: the last row whose first bin is <= i
            const int i = i0 + tid;
            int nb = 0, gb = -1, s0 = 0, cx = 0, cy = 0, cz = 0;
            if (i < nlist) {
                int lo = 0, hi = npass - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_rpre[mid] <= i) lo = mid;
                    else hi = mid - 1;
                }
                const int4 rg = s_row[lo];
                const int kk = i - s_rpre[lo];
                const int idx = (kk < rg.y) ? rg.x + kk : rg.z + (kk - rg.y);
                const int r = r0 + lo;
                cx = P.occ_x[idx];
                cy = ylo + r % ny;
                cz = zlo + r / ny;
                gb = cx + P.nb0 * (cy + P.nb1 * cz);
                nb = P.bin_nuniq[gb];
                s0 = P.bin_start[gb];
            }
            // block exclusive scan of nb
            const int lane = tid & 31, wid = tid >> 5;
            int incl = nb;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (lane == 31) wtot[wid] = incl;
            __syncthreads();
            if (wid == 0) {
                const int v = (lane < NT / 32) ? wtot[lane] : 0;
                int i2 = v;
                for (int o = 1; o < 32; o <<= 1) {
                    const int u = __shfl_up_sync(0xffffffffu, i2, o);
                    if (lane >= o) i2 += u;
                }
                wtot[lane] = i2 - v;
            }
            __syncthreads();
            const int off = wtot[wid] + incl - nb;
            const bool take = (i < nlist) && (off + nb <= kFixCap);
            const int taken = __syncthreads_count(take);  // taken bins form a prefix
            if (take) {
                soff[tid] = off;
                ssrc[tid] = s0;
                sbin[tid] = gb;
                sbox[tid] = make_float4(8.f * cx, 8.f * cy, 8.f * cz, nb > 0 ? 1.f : 0.f);
            }
            if (tid == taken - 1) soff[taken] = off + nb;
            __syncthreads();
            const int ncell = (taken > 0) ? soff[taken] : 0;
            // all threads copy: staged cell j belongs to the last taken bin
            // whose first cell is <= j (empty bins share their successor's)
            for (int j = tid; j < ncell; j += NT) {
                int lo = 0, hi = taken - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (soff[mid] <= j) lo = mid;
                    else hi = mid - 1;
                }
                const int g = sbin[lo], src = ssrc[lo] + (j - soff[lo]);
                const int qx = g % P.nb0, qy = (g / P.nb0) % P.nb1, qz = g / (P.nb0 * P.nb1);
                const int lc = P.ucell[src];
                cell[j] = make_float4((float)(qx * 8 + (lc & 7)), (float)(qy * 8 + ((lc >> 3) & 7)),
                                      (float)(qz * 8 + (lc >> 6)), (float)P.ucount[src]);
            }
            __syncthreads();
            // every lane of a warp with an active node runs the loops below
            // (warp-uniform control flow; in 3D the bin votes need the whole
            // warp).  A lane whose nodes stopped keeps adding terms beyond its
            // stopping ring: they are positive and only make its sums more
            // complete (the term count below leaves them out)
            const bool me = active[0] || active[1];
            const bool run = __any_sync(0xffffffffu, me);
            if (run && ncell > 0) {
                // the shift m need not be the exact minimum, only keep every
                // term in range: no shift yet, or a batch point that could
                // be nearer than m by more than 60 tau ln 2 (term > 2^60),
                // calls for the nearest point of the batch first
                const float lim = 60.f / l2e_th;
                // bin boxes are close enough unless tau is below ~0.3 h: the
                // nearest point may then lie a bin diagonal (7 sqrt(D) nodes)
                // beyond the box bound, its term 2^(-7 sqrt(D) l2e_th)
                const bool by_bins = 7.f * ((D == 2) ? 1.4143f : 1.7321f) * l2e_th < 60.f;
                if (me && (mg[0] - lb_in > lim || mg[1] - lb_in > lim)) {
                    float mn[NPT] = {INFINITY, INFINITY};
                    if (by_bins) {
                        // distance to the nearest occupied bin's box: a lower
                        // bound on the nearest point within one bin diagonal
                        for (int b = 0; b < taken; ++b) {
                            const float4 bq = sbox[b];
                            if (bq.w == 0.f) continue;
                            const float ex = fmaxf(fmaxf(bq.x - xf, xf - (bq.x + 7.f)), 0.f);
                            const float ey = (D == 2) ? 0.f : fmaxf(fmaxf(bq.y - yf, yf - (bq.y + 7.f)), 0.f);
                            const float base = fmaf(ex, ex, ey * ey);
#pragma unroll
                            for (int j = 0; j < NPT; ++j) {
                                const float c = (D == 2) ? yf + kOff * j : zf + kOff * j;
                                const float lo = (D == 2) ? bq.y : bq.z;
                                const float ec = fmaxf(fmaxf(lo - c, c - (lo + 7.f)), 0.f);
                                mn[j] = fminf(mn[j], fmaf(ec, ec, base));
                            }
                        }
                    } else {
                    for (int e = 0; e < ncell; ++e) {
                        const float4 q = cell[e];
                        const float d0 = xf - q.x, d1 = yf - q.y;
                        const float cl = (D == 2) ? d1 : zf - q.z;
                        const float base = (D == 2) ? d0 * d0 : fmaf(d0, d0, d1 * d1);
#pragma unroll
                        for (int j = 0; j < NPT; ++j) {
                            const float cj = cl + kOff * j;
                            mn[j] = fminf(mn[j], fmaf(cj, cj, base));
                        }
                    }
                    }
#pragma unroll
                    for (int j = 0; j < NPT; ++j) {
                        const float r = sqrtf(mn[j]);
                        if (r < mg[j]) {
                            const float sc = (mg[j] < INFINITY) ? ex2_approx((r - mg[j]) * l2e_th) : 0.f;
                            lane_scale(sE, j, sc);
                            lane_scale(sA, j, sc);
#pragma unroll
                            for (int a = 0; a < D; ++a) lane_scale(sG[a], j, sc);
#pragma unroll
                            for (int a = 0; a < NH; ++a) lane_scale(sB[a], j, sc);
                            mg[j] = r;
                            if (j) mk.y = r * l2e_th;
                            else mk.x = r * l2e_th;
                        }
                    }
                }
                const unsigned nmine = me ? (mine[0] ? 1u : 0u) + (mine[1] ? 1u : 0u) : 0u;
                // 3D: a bin whose points all lie at least rho_j from node j adds
                // at most n e^{-(rho_j - m_j)/tau} to its sum (relative to
                // e^{-m_j/tau}), n <= the points in the box of rings <= k1.
                // rho_j makes all the batch's skipped points together add at
                // most 1e-6 of the sum so far (2^-19.93), so over a node's
                // batches the skipped terms stay below (batches) x 1e-6 of
                // its final sum; the warp skips the bin when none of its
                // active nodes needs it.  No sum yet: nothing is skipped.  (The points of
                // a 2D tile's bins are few, and the per-bin loop measured
                // slower there: 2D sums every staged point in one loop.)
                float rho2[NPT] = {INFINITY, INFINITY};
                bool cull = false;
                if constexpr (D == 3) {
#pragma unroll
                    for (int j = 0; j < NPT; ++j) {
                        const float sj = j ? sE.y : sE.x;
                        const float rho = mg[j] + (__log2f((float)s_cnt[0]) + 19.94f - __log2f(sj)) / l2e_th;
                        rho2[j] = (active[j] && sj > 0.f && mg[j] < INFINITY) ? rho * rho : INFINITY;
                    }
                    cull = __any_sync(0xffffffffu, rho2[0] < INFINITY || rho2[1] < INFINITY);
                }
                const float2 nl2e = dup2(-l2e_th), ih2 = dup2(ih), itau2 = dup2(itau);
                const int nloop = (D == 3) ? taken : 1;
                for (int b = 0; b < nloop; ++b) {
                    const int e0 = (D == 3) ? soff[b] : 0, e1 = (D == 3) ? soff[b + 1] : ncell;
                    if (e0 == e1) continue;
                    if (cull) {
                        // squared distance from each node to the bin's box
                        const float4 bq = sbox[b];
                        const float ex = fmaxf(fmaxf(bq.x - xf, xf - (bq.x + 7.f)), 0.f);
                        const float ey = (D == 2) ? 0.f : fmaxf(fmaxf(bq.y - yf, yf - (bq.y + 7.f)), 0.f);
                        const float base = fmaf(ex, ex, ey * ey);
                        bool skip = true;
#pragma unroll
                        for (int j = 0; j < NPT; ++j) {
                            const float c = (D == 2) ? yf + kOff * j : zf + kOff * j;
                            const float lo = (D == 2) ? bq.y : bq.z;
                            const float ec = fmaxf(fmaxf(lo - c, c - (lo + 7.f)), 0.f);
                            skip = skip && (!active[j] || fmaf(ec, ec, base) >= rho2[j]);
                        }
                        if (__all_sync(0xffffffffu, skip)) continue;
                    }
                    nterm += (unsigned)(e1 - e0) * nmine;
                    nsum += (unsigned)(e1 - e0);
#pragma unroll 4
                for (int e = e0; e < e1; ++e) {
                    const float4 q = cell[e];
                    const float d0 = xf - q.x, d1 = yf - q.y;
                    const float cl = (D == 2) ? d1 : zf - q.z;
                    const float base = (D == 2) ? d0 * d0 : fmaf(d0, d0, d1 * d1);
                    // node offsets per axis, lanes = the two nodes (they differ along the last axis)
                    float2 dv[D];
                    dv[0] = dup2(d0);
                    if (D == 3) dv[1] = dup2(d1);
                    dv[D - 1] = make_float2(cl, cl + kOff);
                    const float2 r2 = __ffma2_rn(dv[D - 1], dv[D - 1], dup2(base));
                    // 1/r from one reciprocal square root; r2 is an integer,
                    // and the point under the node itself (r2 = 0) gets
                    // 1/r = 0: it adds to the sum only
                    const float2 ir = make_float2(fminf(rsqrt_approx(r2.x), r2.x), fminf(rsqrt_approx(r2.y), r2.y));
                    const float2 arg = __ffma2_rn(__fmul2_rn(r2, ir), nl2e, mk);
                    const float2 E = __fmul2_rn(dup2(q.w), make_float2(ex2_approx(arg.x), ex2_approx(arg.y)));
                    sE = __fadd2_rn(sE, E);
                    if constexpr (LVL >= 1) {
                        const float2 Eir = __fmul2_rn(E, ir);
#pragma unroll
                        for (int a = 0; a < D; ++a) sG[a] = __ffma2_rn(Eir, dv[a], sG[a]);
                        if constexpr (LVL >= 2) {
                            const float2 F = __fmul2_rn(__fmul2_rn(Eir, ir), __ffma2_rn(ir, ih2, itau2));
                            sA = __fadd2_rn(sA, Eir);
                            // every moment but the last diagonal one, which
                            // the trace gives at the end
                            int qh = 0;
#pragma unroll
                            for (int a = 0; a < D - 1; ++a) {
                                const float2 Fd = __fmul2_rn(F, dv[a]);
#pragma unroll
                                for (int bb = a; bb < D; ++bb, ++qh) sB[qh] = __ffma2_rn(Fd, dv[bb], sB[qh]);
                            }
                        }
                    }
                }
                }
            }
            __syncthreads();
            i0 += max(taken, 1);
        }
        }  // row passes
        if (tid < kLook) {
            // log T_i, T_i = sum_{k'=k1+i+1}^{k1+kLook} n_k' e^{-lb(k'-1)/tau}
            //                + (points beyond ring k1+kLook) e^{-lb(k1+kLook)/tau},
            // summed relative to e^{-lb(k1)/tau} (every factor <= 1)
            const float q = __expf(-8.f * h * itau);  // one ring further out
            float w = 1.f, acc = 0.f;
            for (int i = 0; i < kLook; ++i) {
                if (i >= tid) acc += (float)(s_cnt[i + 1] - s_cnt[i]) * w;
                w *= q;
            }
            acc += (float)(ktot - s_cnt[kLook]) * w;
            s_logT[tid] = __logf(acc) - (8.f * k1 + 1.f) * h * itau;
        }
        __syncthreads();
        // phi = e^{-m/tau} sE + (rest), rest <= T_0; in logs A = log(e^{-m/tau} sE)
        const float tail0 = s_logT[0];
        // The next batch ends where some whole warp could be done: the
        // summing loop is warp-uniform, so a node that stops early saves
        // nothing while its warp runs on; per warp the latest ring at which
        // its nodes could stop (or be capped), then the earliest over warps.
        int kev = -1;
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            if (!active[j]) continue;
            const float A = (mg[j] < INFINITY) ? -mg[j] * h * itau + __logf(lane(sE, j)) : -INFINITY;
            // the rest adds less than 1e-5 of the sum: final
            if (tail0 <= A - 11.512925f) {
                active[j] = false;
                continue;
            }
            // phi < theta_64 whatever the rest adds: capped
            const float hi = fmaxf(A, tail0), lo = fminf(A, tail0);
            const float lphi = hi + __logf(1.f + __expf(lo - hi));  // log of the bound on phi
            if (!P.full && lphi < lt - 1e-4f) {
                active[j] = false;
                early_cap[j] = true;
                continue;
            }
            // the first later ring end (within the look-ahead) at which this
            // node could stop (its sum can only grow to e^{lphi}) or be capped
            int ev = kLook;
            for (int i = 1; i < kLook; ++i) {
                const float Ti = s_logT[i];
                if (Ti <= lphi - 11.512925f || (!P.full && A < lt - 1e-4f && Ti < lt - 1e-4f)) {
                    ev = i;
                    break;
                }
            }
            kev = max(kev, min(k1 + ev, kmax));
        }
        kev = __reduce_max_sync(0xffffffffu, kev);
        if ((tid & 31) == 0 && kev >= 0) atomicMin(&s_kev[(round + 1) & 1], kev);
        k0 = k1 + 1;
    }
    int fixed = 0;
    float rinv = 0.f;  // largest 1/max(m, 1) over the nodes written here
    TO *So = reinterpret_cast<TO *>(P.S);
    TO *dS = reinterpret_cast<TO *>(P.dS);
    TO *d2S = reinterpret_cast<TO *>(P.d2S);
    const float scap = -tau * lt;
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        if (!mine[j]) continue;
        const int64_t nd = node[j];
        const float S = fmaf(mg[j], h, -tau * logf(lane(sE, j)));
        const float sg = (P.sign && P.sign[nd] < 0) ? -1.f : 1.f;
        if (!P.full && (early_cap[j] || !(S <= scap))) {
            P.flags[nd] = SDF_FLAG_CAPPED | SDF_FLAG_FIXUP;
            continue;
        }
        ++fixed;
        rinv = fmaxf(rinv, 1.f / fmaxf(mg[j], 1.f));
        if (So) So[nd] = (TO)(sg * S);
        if constexpr (LVL == 0) {
            P.flags[nd] = SDF_FLAG_FIXUP;
            continue;
        }
        const float inv = 1.f / lane(sE, j);
        float g[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            g[a] = lane(sG[a], j) * inv;
            if (dS) dS[a * P.nnodes + nd] = (TO)g[a];
        }
        if (LVL >= 2 && d2S) {
            // sB is stored row by row (xx, xy, [xz,] yy, ...); d2S is
            // diagonal first, then the pairs a < b.  The last diagonal
            // moment was not summed: per term F r^2 = E/(h r) + E/tau, so
            // sum_a sB_aa = sA/h + (sE - E0)/tau, E0 the term of a point at
            // the node itself (its 1/r is taken as 0; it is the only point
            // at distance 0, so the shift makes E0 its multiplicity), and
            // H_last = sum_{a<last} sB_aa/sE - (1 - E0/sE)/tau + g_last^2/tau
            const float Ad = lane(sA, j) * ih * inv;
            float e0 = 0.f;
            if (mg[j] == 0.f) {
                const int xj = x, yj = (D == 2) ? y + 8 * j : y, zj = (D == 2) ? 0 : z + 4 * j;
                const int64_t gb = (xj >> 3) + (int64_t)P.nb0 * ((yj >> 3) + (int64_t)P.nb1 * (zj >> 3));
                const int lc = (xj & 7) + 8 * (yj & 7) + 64 * (zj & 7);
                const int u0 = P.bin_start[gb], u1 = u0 + P.bin_nuniq[gb];
                for (int u = u0; u < u1; ++u)
                    if (P.ucell[u] == lc) e0 = (float)P.ucount[u];
            }
            float tr = 0.f;
#pragma unroll
            for (int a = 0; a < D - 1; ++a) tr += lane(sB[sym_index<D>(a, a)], j) * inv;
            int q = 0;
#pragma unroll
            for (int a = 0; a < D; ++a, ++q) {
                const float Baa = (a < D - 1) ? Ad - lane(sB[sym_index<D>(a, a)], j) * inv
                                              : tr - (1.f - e0 * inv) * itau;
                d2S[q * P.nnodes + nd] = (TO)(Baa + g[a] * g[a] * itau);
            }
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
                for (int bb = a + 1; bb < D; ++bb, ++q)
                    d2S[q * P.nnodes + nd] = (TO)(-lane(sB[sym_index<D>(a, bb)], j) * inv + g[a] * g[bb] * itau);
        }
        P.flags[nd] = SDF_FLAG_FIXUP;
    }
    // statistics
    unsigned fx = fixed;
    unsigned long long nt64 = nterm;
    for (int o = 16; o > 0; o >>= 1) {
        fx += __shfl_down_sync(0xffffffffu, fx, o);
        nt64 += __shfl_down_sync(0xffffffffu, nt64, o);
    }
    // for the error report: the most terms a written node summed, its 1/r bound
    const unsigned nmx = __reduce_max_sync(0xffffffffu, fixed ? nsum : 0u);
    const unsigned rmx = __reduce_max_sync(0xffffffffu, __float_as_uint(rinv));
    if ((tid & 31) == 0) {
        if (nmx) atomicMax(&P.dsc_w->fix_nmax, (unsigned long long)nmx);
        if (rmx) atomicMax(&P.dsc_w->fix_rinv_bits, rmx);
        if (fx) {
            atomicAdd(&P.dsc_w->n_fixup_nodes, (unsigned long long)fx);
            // the epilogue counted these as capped; they are not any more
            atomicAdd(&P.dsc_w->n_capped, (unsigned long long)(-(long long)fx));
        }
        if (nt64) atomicAdd(&P.dsc_w->n_fixup_terms, nt64);
    }
    if (tid == 0) {
        atomicAdd(&P.dsc_w->n_fixup_tiles, 1ull);
        atomicMax(&P.dsc_w->fix_rounds, (unsigned long long)round);  // for the error report
    }
}

cudaError_t launch_fixup(sdf_plan_impl *p, bool /*with_sign*/, void *S, void *dS, void *d2S, const int8_t *sign,
                         uint8_t *flags) {
    FixParams F;
    F.bin_start = p->bin_start;
    F.occ_start = p->occ_start;
    F.occ_x = p->occ_x;
    F.sat = p->bin_count;  // launch_cheb wrote the table there
    F.bin_nuniq = p->bin_nuniq;
    F.ucell = p->ucell;
    F.ucount = p->ucount;
    F.cheb = p->cheb;
    F.tile_flag = p->tile_flag;
    F.dsc = p->dsc;
    F.dsc_w = p->dsc;
    F.S = S;
    F.dS = dS;
    F.d2S = d2S;
    F.sign = sign;
    F.flags = flags;
    F.N0 = (int)p->N[0];
    F.N1 = (int)p->N[1];
    F.N2 = (int)p->N[2];
    F.nb0 = (int)p->nb[0];
    F.nb1 = (int)p->nb[1];
    F.nb2 = (int)p->nb[2];
    F.nnodes = p->nnodes;
    F.h = (float)p->h;
    F.tau = (float)p->tau;
    F.l2e_th = (float)(p->h * 1.4426950408889634 / p->tau);
    const int D = p->D;
    const double n = (double)p->M[0] * (double)p->M[1] * (D == 3 ? (double)p->M[2] : 1.0);
    F.coef64 = p->noise_c64 * ldexp(1.0, -53) * sqrt(log2(n)) / sqrt(n) * p->q_factor / kTrustEps;
    F.logK = (float)log((double)p->last_K);
    F.log_coef64 = (float)log(F.coef64);
    F.full = p->full_range ? 1 : 0;
    prof_begin(p, "fixup", p->stream);
    // only the derivatives the caller asked for are summed
    const int lvl = d2S ? 2 : (dS ? 1 : 0);
#define SDF_FIX(DD, LV)                                                                          \
    do {                                                                                         \
        if (DD == 2) {                                                                           \
            const int64_t nt = ((p->nb[0] + kTB2 - 1) / kTB2) * ((p->nb[1] + kTB2 - 1) / kTB2);  \
            k_fixup<2, float, LV><<<(unsigned)nt, 32 * kTB2 * kTB2, 0, p->stream>>>(F);           \
        } else {                                                                                 \
            k_fixup<3, float, LV><<<(unsigned)p->nbins, 256, 0, p->stream>>>(F);                  \
        }                                                                                        \
    } while (0)
    if (lvl == 2) SDF_FIX(D, 2);
    else if (lvl == 1) SDF_FIX(D, 1);
    else SDF_FIX(D, 0);
#undef SDF_FIX
    prof_end(p, p->stream);
    return cudaGetLastError();
}

}  // namespace sdf
