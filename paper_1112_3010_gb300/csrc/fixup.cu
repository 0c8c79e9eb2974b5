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
// One CTA per flagged 8^D tile (one thread per node).  Candidate bins are
// visited in rings of Chebyshev distance k = 0, 1, 2, ... around the tile;
// after ring k every unvisited occupied node lies at least lb = (8k+1)h from
// every node of the tile, so a node stops summing once K exp(-(lb - m)/tau)
// is below 1e-5 of its sum, or once even its sum plus K exp(-lb/tau) is below
// theta_64 (it stays capped).  Terms beyond m + tau ln(K 1e5) are skipped.  A
// tile whose nearest occupied bin is so far that K exp(-d/tau) < theta_64
// keeps the capped value.  Visiting order is fixed, so the sums are
// deterministic.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sdf_internal.cuh"

namespace sdf {

struct FixParams {
    const int *bin_start, *bin_nuniq, *ucell, *ucount;
    const unsigned char *cheb, *tile_flag;
    const DevScalars *dsc;
    DevScalars *dsc_w;
    void *S, *dS, *d2S;
    const int8_t *sign;
    uint8_t *flags;
    int N0, N1, N2;
    int nb0, nb1, nb2;
    int64_t nnodes;
    double h, tau, coef64;
    double logK;
    int fp64_out;
};

constexpr int kFixCap = 1024;  // cells staged in shared memory at once
constexpr int kTB2 = 2;       // 2D tile: kTB2 x kTB2 bins (16 x 16 nodes)

// Bin offset of ring element i (ring k > 0) in 2D: walk the square's border.
__device__ __forceinline__ void ring2(int k, int i, int &dx, int &dy) {
    const int side = 2 * k;
    const int s = i / side, o = i % side;
    switch (s) {
        case 0: dx = -k + o; dy = -k; break;
        case 1: dx = k; dy = -k + o; break;
        case 2: dx = k - o; dy = k; break;
        default: dx = -k; dy = k - o; break;
    }
}

// 3D ring element i: enumerate the (2k+1)^3 cube and skip the interior by
// index arithmetic: layers z = -k and z = k are full squares, the others are
// square borders.
__device__ __forceinline__ void ring3(int k, int i, int &dx, int &dy, int &dz) {
    const int w = 2 * k + 1, full = w * w, border = 8 * k;
    if (i < full) {
        dz = -k;
        dx = i % w - k;
        dy = i / w - k;
        return;
    }
    i -= full;
    const int nmid = 2 * k - 1;
    if (i < nmid * border) {
        dz = -k + 1 + i / border;
        ring2(k, i % border, dx, dy);
        return;
    }
    i -= nmid * border;
    dz = k;
    dx = i % w - k;
    dy = i / w - k;
}

// Border of a square of side s (s >= 2): element i of 4(s-1), as offsets
// from its corner.
__device__ __forceinline__ void square_border(int s, int i, int &dx, int &dy) {
    const int side = i / (s - 1), o = i % (s - 1);
    switch (side) {
        case 0: dx = o; dy = 0; break;
        case 1: dx = s - 1; dy = o; break;
        case 2: dx = s - 1 - o; dy = s - 1; break;
        default: dx = 0; dy = s - 1 - o; break;
    }
}

template <int D, typename TO>
__global__ void __launch_bounds__(D == 2 ? 256 : 512) k_fixup(FixParams P) {
    constexpr int TB = (D == 2) ? kTB2 : 1;  // tile edge in bins
    constexpr int NT = (D == 2) ? 64 * kTB2 * kTB2 : 512;
    constexpr int NH = D * (D + 1) / 2;
    __shared__ int4 cell[kFixCap];  // (x, y, z, count) of staged occupied nodes
    __shared__ int soff[1];
    __shared__ int wtot[32];
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
    const double theta64 = P.coef64 * sqrt((double)P.dsc->sum_c2);
    const double lt = log(theta64);
    const double dlo = (c >= 1) ? (8.0 * (c - 1) + 1.0) * P.h : 0.0;
    // every node of the tile: phi <= K exp(-dlo/tau) < theta64 -> stays capped
    if (c >= 255 || P.logK - dlo / P.tau < lt) return;

    const int x = (D == 2) ? bx * 8 + (tid % (8 * TB)) : bx * 8 + (tid & 7);
    const int y = (D == 2) ? by * 8 + (tid / (8 * TB)) : by * 8 + ((tid >> 3) & 7);
    const int z = (D == 2) ? 0 : bz * 8 + (tid >> 6);
    const bool inb = x < P.N0 && y < P.N1 && (D == 2 || z < P.N2);
    const int64_t node = (int64_t)x + (int64_t)P.N0 * (y + (int64_t)P.N1 * z);
    const bool mine = inb && (P.flags[node] & SDF_FLAG_CAPPED) != 0;
    bool active = mine;      // still summing
    bool early_cap = false;  // shown below theta_64 before the sum finished
    const float h = (float)P.h, tau = (float)P.tau, itau = 1.f / tau, ih = 1.f / h;
    const float l2e_tau = 1.4426950408889634f / tau;
    // terms beyond m + ccut weigh < 1e-5 of the sum in total (K of them at most)
    const float lnK = (float)P.logK;
    const float ccut = tau * (lnK + 11.512925f);
    float m = INFINITY, sE = 0.f, sG[D], sH[NH];
#pragma unroll
    for (int a = 0; a < D; ++a) sG[a] = 0.f;
#pragma unroll
    for (int a = 0; a < NH; ++a) sH[a] = 0.f;
    unsigned long long nterm = 0;

    // ring k: bins at Chebyshev distance k from the tile's block of bins
    auto nring_of = [&](int k) {
        return (D == 2) ? 4 * (TB + 2 * k - 1)
                        : ((k == 0) ? 1 : (2 * k + 1) * (2 * k + 1) * (2 * k + 1) - (2 * k - 1) * (2 * k - 1) * (2 * k - 1));
    };
    // (m + ccut)^2 in grid units: terms beyond it are skipped before any MUFU work
    float rc2 = INFINITY;
    const int kmax = max(max(P.nb0, P.nb1), (D == 3) ? P.nb2 : 0);
    // rings are visited in batches {0,1,2}, {3,4}, then one at a time: most
    // tiles finish in the first batch, one staging round
    for (int k0 = 0; k0 <= kmax;) {
        if (!__syncthreads_or(active)) break;
        const int k1 = min(kmax, (k0 == 0) ? 2 : (k0 == 3 ? 4 : k0));
        int nring = 0;
        for (int k = k0; k <= k1; ++k) nring += nring_of(k);
        for (int i0 = 0; i0 < nring;) {
            // one candidate bin per thread
            const int i = i0 + tid;
            int nb = 0, gb = -1;
            if (i < nring) {
                int k = k0, ii = i;
                while (ii >= nring_of(k)) {
                    ii -= nring_of(k);
                    ++k;
                }
                int dx = 0, dy = 0, dz = 0;
                if (D == 2) {
                    square_border(TB + 2 * k, ii, dx, dy);
                    dx -= k;
                    dy -= k;
                } else if (k > 0) {
                    ring3(k, ii, dx, dy, dz);
                }
                const int qx = bx + dx, qy = by + dy, qz = bz + dz;
                if (qx >= 0 && qx < P.nb0 && qy >= 0 && qy < P.nb1 && (D == 2 || (qz >= 0 && qz < P.nb2))) {
                    gb = qx + P.nb0 * (qy + P.nb1 * qz);
                    nb = P.bin_nuniq[gb];
                }
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
            const bool take = (i < nring) && (off + nb <= kFixCap);
            const int taken = __syncthreads_count(take);  // taken bins form a prefix
            if (tid == taken - 1) soff[0] = off + nb;
            if (take && nb > 0) {
                const int s0 = P.bin_start[gb];
                const int qx = gb % P.nb0, qy = (gb / P.nb0) % P.nb1, qz = gb / (P.nb0 * P.nb1);
                for (int e = 0; e < nb; ++e) {
                    const int lc = P.ucell[s0 + e];
                    cell[off + e] = make_int4(qx * 8 + (lc & 7), qy * 8 + ((lc >> 3) & 7), qz * 8 + (lc >> 6),
                                              P.ucount[s0 + e]);
                }
            }
            __syncthreads();
            const int ncell = (taken > 0) ? soff[0] : 0;
            if (active) {
                for (int e = 0; e < ncell; ++e) {
                    const int4 q = cell[e];
                    const int ddx = x - q.x, ddy = y - q.y, ddz = (D == 3) ? z - q.z : 0;
                    const int r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                    if ((float)r2 > rc2) continue;
                    // r = h sqrt(r2) and 1/sqrt(r2) from one reciprocal square root
                    const float ir = r2 > 0 ? rsqrtf((float)r2) : 0.f;
                    const float r = (float)r2 * ir * h;
                    if (r - m > ccut) continue;
                    ++nterm;
                    if (r < m) {
                        const float sc = exp2f((r - m) * l2e_tau);
                        sE *= sc;
#pragma unroll
                        for (int a = 0; a < D; ++a) sG[a] *= sc;
#pragma unroll
                        for (int a = 0; a < NH; ++a) sH[a] *= sc;
                        m = r;
                        const float rc = (m + ccut) * ih * 1.0001f;
                        rc2 = rc * rc;
                    }
                    const float E = (float)q.w * exp2f((m - r) * l2e_tau);
                    sE += E;
                    if (r2 > 0) {
                        const float nn[3] = {ddx * ir, ddy * ir, ddz * ir};
                        const float irw = ir * ih;  // 1/r in world units
#pragma unroll
                        for (int a = 0; a < D; ++a) sG[a] += E * nn[a];
                        int qh = 0;
#pragma unroll
                        for (int a = 0; a < D; ++a, ++qh)
                            sH[qh] += E * ((1.f - nn[a] * nn[a]) * irw - nn[a] * nn[a] * itau);
#pragma unroll
                        for (int a = 0; a < D; ++a)
#pragma unroll
                            for (int bb = a + 1; bb < D; ++bb, ++qh) sH[qh] -= E * nn[a] * nn[bb] * (irw + itau);
                    }
                }
            }
            __syncthreads();
            i0 += max(taken, 1);
        }
        // after ring k1 every unvisited node lies at least lb from this tile
        if (active) {
            const float lb = (8.f * k1 + 1.f) * h;
            const float tailA = -lb * itau + lnK;                 // log of K exp(-lb/tau)
            if (m < INFINITY) {
                const float lsE = logf(sE);
                // the rest adds less than 1e-5 of the sum: final
                if ((lb - m) * itau >= lnK - lsE + 11.512925f) active = false;
                // phi < theta_64 whatever the rest adds: capped
                const float A = -m * itau + lsE;
                const float hi = fmaxf(A, tailA), lo = fminf(A, tailA);
                if (hi + log1pf(expf(lo - hi)) < (float)lt - 1e-4f) {
                    active = false;
                    early_cap = true;
                }
            } else if (tailA < (float)lt - 1e-4f) {
                active = false;
                early_cap = true;
            }
        }
        k0 = k1 + 1;
    }
    int fixed = 0, capped = 0;
    if (mine) {
        const double S = (double)m - P.tau * log((double)sE);
        const double scap = -P.tau * lt;
        TO *So = reinterpret_cast<TO *>(P.S);
        TO *dS = reinterpret_cast<TO *>(P.dS);
        TO *d2S = reinterpret_cast<TO *>(P.d2S);
        const double sg = (P.sign && P.sign[node] < 0) ? -1.0 : 1.0;
        if (early_cap || !(S <= scap)) {
            capped = 1;
            P.flags[node] = SDF_FLAG_CAPPED | SDF_FLAG_FIXUP;
        } else {
            fixed = 1;
            if (So) So[node] = (TO)(sg * S);
            const float inv = 1.f / sE;
            float g[D];
#pragma unroll
            for (int a = 0; a < D; ++a) {
                g[a] = sG[a] * inv;
                if (dS) dS[a * P.nnodes + node] = (TO)g[a];
            }
            if (d2S) {
                int q = 0;
#pragma unroll
                for (int a = 0; a < D; ++a, ++q) d2S[q * P.nnodes + node] = (TO)(sH[q] * inv + g[a] * g[a] * itau);
#pragma unroll
                for (int a = 0; a < D; ++a)
#pragma unroll
                    for (int bb = a + 1; bb < D; ++bb, ++q)
                        d2S[q * P.nnodes + node] = (TO)(sH[q] * inv + g[a] * g[bb] * itau);
            }
            P.flags[node] = SDF_FLAG_FIXUP;
        }
    }
    // statistics
    const unsigned fb = __ballot_sync(0xffffffffu, fixed), cb = __ballot_sync(0xffffffffu, capped);
    for (int o = 16; o > 0; o >>= 1) nterm += __shfl_down_sync(0xffffffffu, nterm, o);
    if ((tid & 31) == 0) {
        if (fb) atomicAdd(&P.dsc_w->n_fixup_nodes, (unsigned long long)__popc(fb));
        if (cb) atomicAdd(&P.dsc_w->n_capped, (unsigned long long)__popc(cb));
        if (nterm) atomicAdd(&P.dsc_w->n_fixup_terms, nterm);
    }
    if (tid == 0) atomicAdd(&P.dsc_w->n_fixup_tiles, 1ull);
}

cudaError_t launch_fixup(sdf_plan_impl *p, bool /*with_sign*/, void *S, void *dS, void *d2S, const int8_t *sign,
                         uint8_t *flags) {
    FixParams F;
    F.bin_start = p->bin_start;
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
    F.h = p->h;
    F.tau = p->tau;
    const int D = p->D;
    const double n = (double)p->M[0] * (double)p->M[1] * (D == 3 ? (double)p->M[2] : 1.0);
    F.coef64 = p->noise_c64 * ldexp(1.0, -53) * sqrt(log2(n)) / sqrt(n) * p->q_factor / kTrustEps;
    F.logK = log((double)p->last_K);
    F.fp64_out = 0;
    prof_begin(p, "fixup", p->stream);
    if (D == 2) {
        const int64_t nt = ((p->nb[0] + kTB2 - 1) / kTB2) * ((p->nb[1] + kTB2 - 1) / kTB2);
        k_fixup<2, float><<<(unsigned)nt, 64 * kTB2 * kTB2, 0, p->stream>>>(F);
    } else {
        k_fixup<3, float><<<(unsigned)p->nbins, 512, 0, p->stream>>>(F);
    }
    prof_end(p, p->stream);
    return cudaGetLastError();
}

}  // namespace sdf
