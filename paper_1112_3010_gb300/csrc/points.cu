// points.cu -- step A1: snap the points to their nearest nodes (Sec. 6,
// Examples 3-4 round the points to the grid) and form the
// scattered fields of eq. function_g (counts) and of Secs. 4.1-4.2
// (tangent- or normal-weighted sums), as a list of distinct occupied nodes
// grouped by 8^D-node bins.
//
// Determinism: every per-node sum is an integer sum (counts, and weights in
// 62-bit fixed point scaled to max|weight|), so the result does not depend on
// the order in which atomics land.
//
// Steps: k_snap (node, bin, count per bin, max|w|) -> k_scan (bin offsets) ->
// k_fill (bucket the points by bin) -> k_dedupe (per bin: per-node sums in
// shared memory, compaction in node order) -> k_cheb_* (Chebyshev distance in
// bins to the nearest occupied bin, used by the fix-up).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sdf_internal.cuh"

namespace sdf {

__device__ __forceinline__ void set_status(DevScalars *d, int code) { atomicCAS(&d->status, 0, code); }

__global__ void k_snap(int D, int64_t K, const double *__restrict__ P, const double *__restrict__ W, double h,
                       int N0, int N1, int N2, int nb0, int nb1, int *pt_bin, int *pt_lc, int *bin_count,
                       DevScalars *dsc) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = k < K;
    int j[3] = {0, 0, 0};
    const int Nn[3] = {N0, N1, N2};
    bool ok = live;
    for (int a = 0; live && a < D; ++a) {
        const double y = P[k * D + a];
        // nearest node, ties up: floor(y/h + 0.5)
        const double q = floor(y / h + 0.5);
        if (!(q >= 0.0 && q < (double)Nn[a])) {
            ok = false;
        } else {
            j[a] = (int)q;
        }
    }
    if (live && !ok) {
        pt_lc[k] = -1;
        set_status(dsc, SDF_ERR_POINT_OUT_OF_GRID);
    }
    if (ok) {
        const int b = (j[0] >> 3) + nb0 * ((j[1] >> 3) + nb1 * (j[2] >> 3));
        const int lc = (j[0] & 7) | ((j[1] & 7) << 3) | ((j[2] & 7) << 6);
        pt_bin[k] = b;
        pt_lc[k] = lc;
        atomicAdd(&bin_count[b], 1);
    }
    if (W) {
        // max |w| over the warp first: one atomic per warp, not per point
        // (non-negative doubles order like their bit patterns)
        double m = 0.0;
        for (int a = 0; ok && a < D; ++a) m = fmax(m, fabs(W[k * D + a]));
        unsigned long long bits = (isfinite(m) && m > 0.0) ? (unsigned long long)__double_as_longlong(m) : 0ull;
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long u = __shfl_xor_sync(0xffffffffu, bits, o);
            bits = u > bits ? u : bits;
        }
        if ((threadIdx.x & 31) == 0 && bits) atomicMax(&dsc->wmax, bits);
    }
}

__global__ void k_fill(int64_t K, const int *__restrict__ pt_bin, const int *__restrict__ pt_lc,
                       const int *__restrict__ bin_start, int *bin_fill, long long *entry) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int lc = pt_lc[k];
    if (lc < 0) return;
    const int b = pt_bin[k];
    const int slot = bin_start[b] + atomicAdd(&bin_fill[b], 1);
    entry[slot] = ((long long)lc << 40) | (long long)k;
}

// One CTA per bin: per-node counts and fixed-point weight sums in shared
// memory, then the occupied nodes in node order.
template <int NC>
__global__ void k_dedupe(int D, int64_t K, const double *__restrict__ W, const int *__restrict__ bin_start,
                         const long long *__restrict__ entry, int *bin_nuniq, int *ucell, int *ucount, double *uw,
                         DevScalars *dsc) {
    __shared__ int cnt[NC];
    __shared__ long long wf[3][NC];
    __shared__ int wsum[32];
    const int b = blockIdx.x;
    const int s = bin_start[b], e = bin_start[b + 1];
    const int tid = threadIdx.x, nt = blockDim.x;
    if (s == e) {
        if (tid == 0) bin_nuniq[b] = 0;
        return;
    }
    for (int i = tid; i < NC; i += nt) {
        cnt[i] = 0;
        wf[0][i] = wf[1][i] = wf[2][i] = 0;
    }
    // fixed-point scale: |w| * scale * K < 2^61 (one thread works it out)
    __shared__ double s_scale;
    if (tid == 0) {
        s_scale = 0.0;
        if (W) {
            const double wm = __longlong_as_double((long long)dsc->wmax);
            if (wm > 0.0) {
                const int ex = ilogb((double)K * wm) + 1;  // K*wm < 2^ex
                s_scale = ldexp(1.0, 61 - ex);
            }
        }
    }
    __syncthreads();
    const double scale = s_scale;
    for (int i = s + tid; i < e; i += nt) {
        const long long en = entry[i];
        const int lc = (int)(en >> 40);
        const int64_t k = en & ((1LL << 40) - 1);
        atomicAdd(&cnt[lc], 1);
        if (W) {
            for (int a = 0; a < D; ++a) {
                const long long q = llrint(W[k * D + a] * scale);
                atomicAdd(reinterpret_cast<unsigned long long *>(&wf[a][lc]), (unsigned long long)q);
            }
        }
    }
    __syncthreads();
    // compaction in node order: each thread owns a contiguous range of cells
    const int per = (NC + nt - 1) / nt;
    const int c0 = tid * per, c1 = min(NC, c0 + per);
    int mine = 0;
    unsigned long long c2 = 0;
    for (int c = c0; c < c1; ++c)
        if (cnt[c]) {
            ++mine;
            c2 += (unsigned long long)cnt[c] * (unsigned long long)cnt[c];
        }
    // block exclusive scan of `mine` (nt <= 1024)
    const int lane = tid & 31, wid = tid >> 5;
    int incl = mine;
    for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int v = (lane < (nt + 31) / 32) ? wsum[lane] : 0;
        int inc2 = v;
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, inc2, o);
            if (lane >= o) inc2 += u;
        }
        if (lane < 32) wsum[lane] = inc2 - v;  // exclusive warp offsets
    }
    __syncthreads();
    int pos = s + wsum[wid] + incl - mine;
    const double inv = (scale > 0.0) ? 1.0 / scale : 0.0;
    for (int c = c0; c < c1; ++c) {
        if (!cnt[c]) continue;
        ucell[pos] = c;
        ucount[pos] = cnt[c];
        uw[3 * (int64_t)pos + 0] = (double)wf[0][c] * inv;
        uw[3 * (int64_t)pos + 1] = (double)wf[1][c] * inv;
        uw[3 * (int64_t)pos + 2] = (double)wf[2][c] * inv;
        ++pos;
    }
    // totals
    for (int o = 16; o > 0; o >>= 1) c2 += __shfl_down_sync(0xffffffffu, c2, o);
    if (lane == 0 && c2) atomicAdd(&dsc->sum_c2, c2);
    if (tid == nt - 1) {
        const int total = wsum[wid] + incl;
        bin_nuniq[b] = total;
        atomicAdd(reinterpret_cast<unsigned long long *>(&dsc->n_unique), (unsigned long long)total);
    }
}

// 2D: one warp per bin (64 cells), BPC bins per CTA -- most bins are empty,
// and a CTA per bin would spend the pass launching CTAs.  Same results as
// k_dedupe: per-node counts and fixed-point weight sums, occupied nodes in
// node order.
template <int BPC>
__global__ void __launch_bounds__(32 * BPC) k_dedupe_w(int64_t K, int64_t nbins, const double *__restrict__ W,
                                                      const int *__restrict__ bin_start,
                                                      const long long *__restrict__ entry, int *bin_nuniq, int *ucell,
                                                      int *ucount, double *uw, DevScalars *dsc) {
    constexpr int NC = 64;
    __shared__ int cnt[BPC][NC];
    __shared__ long long wf[2][BPC][NC];
    __shared__ double s_scale;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        // fixed-point scale: |w| * scale * K < 2^61
        s_scale = 0.0;
        if (W) {
            const double wm = __longlong_as_double((long long)dsc->wmax);
            if (wm > 0.0) s_scale = ldexp(1.0, 61 - (ilogb((double)K * wm) + 1));
        }
    }
    __syncthreads();
    const double scale = s_scale;
    const int64_t b = (int64_t)blockIdx.x * BPC + w;
    if (b >= nbins) return;
    const int s = bin_start[b], e = bin_start[b + 1];
    if (s == e) {
        if (lane == 0) bin_nuniq[b] = 0;
        return;
    }
    for (int c = lane; c < NC; c += 32) {
        cnt[w][c] = 0;
        wf[0][w][c] = wf[1][w][c] = 0;
    }
    __syncwarp();
    for (int i = s + lane; i < e; i += 32) {
        const long long en = entry[i];
        const int lc = (int)(en >> 40);
        const int64_t k = en & ((1LL << 40) - 1);
        atomicAdd(&cnt[w][lc], 1);
        if (W) {
            for (int a = 0; a < 2; ++a) {
                const long long q = llrint(W[k * 2 + a] * scale);
                atomicAdd(reinterpret_cast<unsigned long long *>(&wf[a][w][lc]), (unsigned long long)q);
            }
        }
    }
    __syncwarp();
    // compaction in node order: lane owns cells 2 lane, 2 lane + 1
    const int n0 = cnt[w][2 * lane], n1 = cnt[w][2 * lane + 1];
    const int mine = (n0 > 0) + (n1 > 0);
    unsigned long long c2 = (unsigned long long)n0 * n0 + (unsigned long long)n1 * n1;
    int incl = mine;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    int pos = s + incl - mine;
    const double inv = (scale > 0.0) ? 1.0 / scale : 0.0;
    for (int q = 0; q < 2; ++q) {
        const int c = 2 * lane + q;
        const int n = q ? n1 : n0;
        if (!n) continue;
        ucell[pos] = c;
        ucount[pos] = n;
        uw[3 * (int64_t)pos + 0] = (double)wf[0][w][c] * inv;
        uw[3 * (int64_t)pos + 1] = (double)wf[1][w][c] * inv;
        uw[3 * (int64_t)pos + 2] = 0.0;
        ++pos;
    }
    for (int o = 16; o > 0; o >>= 1) c2 += __shfl_down_sync(0xffffffffu, c2, o);
    if (lane == 0) atomicAdd(&dsc->sum_c2, c2);
    if (lane == 31) {
        bin_nuniq[b] = incl;
        atomicAdd(reinterpret_cast<unsigned long long *>(&dsc->n_unique), (unsigned long long)incl);
    }
}

// Chebyshev distance (in bins) to the nearest occupied bin, separable, one
// axis at a time.  Only distances below `cap` matter to the fix-up (a tile at
// cap or beyond is provably below theta_64), so each search stops there and
// larger distances are stored as cap.
__device__ __forceinline__ int cheb_cap(const DevScalars *dsc, double coef64, double logK, double tau_over_h) {
    const double lt = log(coef64 * sqrt((double)dsc->sum_c2));
    const double c = floor(((logK - lt) * tau_over_h - 1.0) / 8.0) + 2.0;
    return (int)fmin(255.0, fmax(1.0, c));
}

__global__ void k_cheb_x(const int *__restrict__ nuniq, unsigned char *out, int nb0, int64_t nbins,
                         const DevScalars *dsc, double coef64, double logK, double tau_over_h) {
    // one thread works the cap out in double (the FP64 pipe is slow)
    __shared__ int s_cap;
    if (threadIdx.x == 0) s_cap = cheb_cap(dsc, coef64, logK, tau_over_h);
    __syncthreads();
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    const int cap = s_cap;
    const int x = (int)(b % nb0);
    const int64_t row = b - x;
    int best = cap;
    for (int d = 0; d < best; ++d) {
        if ((x - d >= 0 && nuniq[row + x - d] > 0) || (x + d < nb0 && nuniq[row + x + d] > 0)) {
            best = d;
            break;
        }
    }
    out[b] = (unsigned char)best;
}

// pass along an axis with stride `st` and length `n`: d(b) = min_j max(|i-j|, in(b_j))
__global__ void k_cheb_axis(const unsigned char *__restrict__ in, unsigned char *out, int64_t nbins, int64_t st, int n) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    const int i = (int)((b / st) % n);
    const int64_t b0 = b - (int64_t)i * st;
    int best = in[b];
    for (int dj = 1; dj < best && dj < n; ++dj) {
        if (i - dj >= 0) best = min(best, max(dj, (int)in[b0 + (int64_t)(i - dj) * st]));
        if (i + dj < n) best = min(best, max(dj, (int)in[b0 + (int64_t)(i + dj) * st]));
    }
    out[b] = (unsigned char)best;
}

// One warp per occupied bin (grid-stride over bins).
__global__ void k_source_flags(int64_t nb_total, const int *__restrict__ bin_start, const int *__restrict__ nuniq,
                               const int *__restrict__ ucell, int N0, int N1, int nb0, int nb1, uint8_t *flags) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = warp; b < nb_total; b += nwarp) {
        const int n = nuniq[b];
        if (n == 0) continue;
        const int s = bin_start[b];
        const int bx = (int)(b % nb0), by = (int)((b / nb0) % nb1), bz = (int)(b / ((int64_t)nb0 * nb1));
        for (int i = lane; i < n; i += 32) {
            const int lc = ucell[s + i];
            const int x = bx * 8 + (lc & 7), y = by * 8 + ((lc >> 3) & 7), z = bz * 8 + (lc >> 6);
            const int64_t node = x + (int64_t)N0 * (y + (int64_t)N1 * z);
            flags[node] |= SDF_FLAG_SOURCE;
        }
    }
}

// Exclusive scan of n counts in three phases: per 4096-element tile (local
// scan + tile total), tile totals (one block), tile offsets added.
constexpr int kScanTile = 4096;

__device__ __forceinline__ int block_excl_scan_1024(int v, int *wsum, int *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int w = wsum[lane];
        int i2 = w;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, i2, o);
            if (lane >= o) i2 += u;
        }
        wsum[lane] = i2 - w;
        if (lane == 31) *total = i2;
    }
    __syncthreads();
    return wsum[wid] + incl - v;
}

__global__ void __launch_bounds__(1024) k_scan_tiles(const int *__restrict__ count, int *start, int *tile_sum,
                                                     int64_t n) {
    __shared__ int wsum[32];
    __shared__ int total;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + 4 * threadIdx.x;
    int v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = (base + j < n) ? count[base + j] : 0;
    const int off = block_excl_scan_1024(v[0] + v[1] + v[2] + v[3], wsum, &total);
    int run = off;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (base + j < n) start[base + j] = run;
        run += v[j];
    }
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_sums(int *tile_sum, int ntiles, int *start, int64_t n) {
    __shared__ int wsum[32];
    __shared__ int total;
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int t0 = 0; t0 < ntiles; t0 += 1024) {
        const int i = t0 + threadIdx.x;
        const int v = i < ntiles ? tile_sum[i] : 0;
        const int off = block_excl_scan_1024(v, wsum, &total);
        if (i < ntiles) tile_sum[i] = carry + off;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) start[n] = carry;
}

__global__ void k_scan_add(int *start, const int *__restrict__ tile_sum, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && i >= kScanTile) start[i] += tile_sum[i / kScanTile];
}

cudaError_t launch_points(sdf_plan_impl *p, int64_t K, const double *points, const double *weights) {
    cudaStream_t st = p->stream;
    cudaError_t e;
    if ((e = cudaMemsetAsync(p->bin_count, 0, sizeof(int) * (p->nbins + 1), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(p->bin_fill, 0, sizeof(int) * p->nbins, st)) != cudaSuccess) return e;
    // clear the per-execute scalars but keep `status` (reported by sdf_sync)
    if ((e = cudaMemsetAsync(reinterpret_cast<char *>(p->dsc) + offsetof(DevScalars, wmax), 0,
                             sizeof(DevScalars) - offsetof(DevScalars, wmax), st)) != cudaSuccess)
        return e;
    const int tb = 256;
    const unsigned gk = (unsigned)((K + tb - 1) / tb);
    prof_begin(p, "snap", st);
    k_snap<<<gk, tb, 0, st>>>(p->D, K, points, weights, p->h, (int)p->N[0], (int)p->N[1], (int)p->N[2],
                              (int)p->nb[0], (int)p->nb[1], p->pt_key, p->pt_lc, p->bin_count, p->dsc);
    prof_end(p, st);
    // tile totals go to bin_nuniq, which k_dedupe overwrites for every bin
    const int64_t ntiles = (p->nbins + kScanTile - 1) / kScanTile;
    prof_begin(p, "scan", st);
    k_scan_tiles<<<(unsigned)ntiles, 1024, 0, st>>>(p->bin_count, p->bin_start, p->bin_nuniq, p->nbins);
    k_scan_sums<<<1, 1024, 0, st>>>(p->bin_nuniq, (int)ntiles, p->bin_start, p->nbins);
    if (ntiles > 1)
        k_scan_add<<<(unsigned)((p->nbins + 255) / 256), 256, 0, st>>>(p->bin_start, p->bin_nuniq, p->nbins);
    prof_end(p, st);
    prof_begin(p, "fill", st);
    k_fill<<<gk, tb, 0, st>>>(K, p->pt_key, p->pt_lc, p->bin_start, p->bin_fill, p->pt_entry);
    prof_end(p, st);
    prof_begin(p, "dedupe", st);
    if (p->D == 2)
        k_dedupe_w<8><<<(unsigned)((p->nbins + 7) / 8), 256, 0, st>>>(K, p->nbins, weights, p->bin_start, p->pt_entry,
                                                                      p->bin_nuniq, p->ucell, p->ucount, p->uw, p->dsc);
    else
        k_dedupe<512><<<(unsigned)p->nbins, 128, 0, st>>>(p->D, K, weights, p->bin_start, p->pt_entry,
                                                         p->bin_nuniq, p->ucell, p->ucount, p->uw, p->dsc);
    prof_end(p, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return debug_after_binning(p);
}

// Summed-area table of the points per bin, written over bin_count (free once
// bin_start, its prefix sum in bin order, exists): sat[b] = points in the
// bins (x' <= x, y' <= y, z' <= z).  One CTA per line scans along y (the
// values are row prefix counts from bin_start), then in 3D along z.
template <int PASS>
__global__ void __launch_bounds__(1024) k_sat_axis(const int *__restrict__ bin_start, int *__restrict__ sat, int nb0,
                                                   int nb1, int nb2) {
    __shared__ int wsum[32];
    const int64_t line = blockIdx.x;  // PASS 0: x + nb0 z; PASS 1: x + nb0 y
    const int x = (int)(line % nb0);
    const int64_t slab = (int64_t)nb0 * nb1;
    const int n = (PASS == 0) ? nb1 : nb2;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int carry = 0;
    for (int i0 = 0; i0 < n; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        int64_t at = 0;
        int v = 0;
        if (i < n) {
            if (PASS == 0) {
                const int64_t row = (int64_t)nb0 * i + slab * (line / nb0);
                at = row + x;
                v = bin_start[row + x + 1] - bin_start[row];
            } else {
                at = line + slab * i;
                v = sat[at];
            }
        }
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            const int w = (lane < nw) ? wsum[lane] : 0;
            int s = w;
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += u;
            }
            wsum[lane] = s - w;  // exclusive warp offsets
        }
        __syncthreads();
        const int out = carry + wsum[wid] + incl;
        if (i < n) sat[at] = out;
        // the chunk's total: the last thread's inclusive value
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) wsum[0] = out;
        __syncthreads();
        carry = wsum[0];
        __syncthreads();
    }
}

// The occupied bins of each bin row (row = by + nb1 bz), x ascending: one
// warp per row counts them (ballots over 32 bins at a time), the counts are
// scanned, and the same warps write the x indices.
template <bool FILL>
__global__ void k_occ_rows(const int *__restrict__ nuniq, int nb0, int64_t nrows, int *cnt_or_start, int *occ_x) {
    const int lane = threadIdx.x & 31;
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= nrows) return;
    const int *nu = nuniq + row * nb0;
    int at = FILL ? cnt_or_start[row] : 0;
    for (int x0 = 0; x0 < nb0; x0 += 32) {
        const int x = x0 + lane;
        const bool occ = x < nb0 && nu[x] > 0;
        const unsigned bal = __ballot_sync(0xffffffffu, occ);
        if (FILL && occ) occ_x[at + __popc(bal & ((1u << lane) - 1u))] = x;
        at += __popc(bal);
    }
    if (!FILL && lane == 0) cnt_or_start[row] = at;
}

cudaError_t launch_cheb(sdf_plan_impl *p, cudaStream_t on) {
    cudaStream_t st = on ? on : p->stream;
    const int64_t nb0 = p->nb[0], nb1 = p->nb[1], nb2 = p->nb[2];
    unsigned char *tmp = p->cheb + p->nbins;  // second half of the allocation
    const unsigned g = (unsigned)((p->nbins + 255) / 256);
    prof_begin(p, "cheb", st);
    k_cheb_x<<<g, 256, 0, st>>>(p->bin_nuniq, tmp, (int)nb0, p->nbins, p->dsc, theta_coef(p, SDF_FP64),
                                log((double)p->last_K), p->tau / p->h);
    if (p->D == 2) {
        k_cheb_axis<<<g, 256, 0, st>>>(tmp, p->cheb, p->nbins, nb0, (int)nb1);
    } else {
        k_cheb_axis<<<g, 256, 0, st>>>(tmp, p->cheb, p->nbins, nb0, (int)nb1);
        k_cheb_axis<<<g, 256, 0, st>>>(p->cheb, tmp, p->nbins, nb0 * nb1, (int)nb2);
        cudaError_t e = cudaMemcpyAsync(p->cheb, tmp, p->nbins, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    }
    const int nz = (p->D == 3) ? (int)nb2 : 1;
    auto threads = [](int64_t n) { return (unsigned)(n >= 1024 ? 1024 : ((n + 31) / 32) * 32); };
    k_sat_axis<0><<<(unsigned)(nb0 * nz), threads(nb1), 0, st>>>(p->bin_start, p->bin_count, (int)nb0, (int)nb1, nz);
    if (p->D == 3)
        k_sat_axis<1><<<(unsigned)(nb0 * nb1), threads(nz), 0, st>>>(p->bin_start, p->bin_count, (int)nb0, (int)nb1, nz);
    if (p->occ_start) {
        // occupied-bin lists per bin row (the fix-up enumerates its rings from them)
        const int64_t nrows = bin_rows(p);
        const unsigned gw = (unsigned)((nrows * 32 + 255) / 256);
        int *cnt = p->occ_tmp, *tsum = p->occ_tmp + nrows;
        k_occ_rows<false><<<gw, 256, 0, st>>>(p->bin_nuniq, (int)nb0, nrows, cnt, nullptr);
        const int64_t ntiles = (nrows + kScanTile - 1) / kScanTile;
        k_scan_tiles<<<(unsigned)ntiles, 1024, 0, st>>>(cnt, p->occ_start, tsum, nrows);
        k_scan_sums<<<1, 1024, 0, st>>>(tsum, (int)ntiles, p->occ_start, nrows);
        if (ntiles > 1)
            k_scan_add<<<(unsigned)((nrows + 255) / 256), 256, 0, st>>>(p->occ_start, tsum, nrows);
        k_occ_rows<true><<<gw, 256, 0, st>>>(p->bin_nuniq, (int)nb0, nrows, p->occ_start, p->occ_x);
    }
    prof_end(p, st);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return debug_after_cheb(p, st);
}

cudaError_t launch_source_flags(sdf_plan_impl *p, uint8_t *flags) {
    prof_begin(p, "source_flags", p->stream);
    k_source_flags<<<(unsigned)sm_count() * 8, 256, 0, p->stream>>>(p->nbins, p->bin_start, p->bin_nuniq, p->ucell, (int)p->N[0],
                                                  (int)p->N[1], (int)p->nb[0], (int)p->nb[1], flags);
    prof_end(p, p->stream);
    return cudaGetLastError();
}

}  // namespace sdf
