// debugcheck.cu -- optional device-side consistency checks
// (sdf_set_debug_checks, or SDF_DEBUG_CHECKS=1 in the environment) and the
// test hook that breaks one of the structures they check.  The paper has no
// counterpart: these guard this library's own data structures.
//
// The kernels after binning address memory through a few index structures:
// bin offsets (bin_start), unique-node counts (bin_nuniq), node codes within a
// bin (ucell, x fastest: lc = x + 8 y + 64 z) with their multiplicities
// (ucount), and for float plans the per-row lists of occupied bins (occ_start,
// occ_x).  When every check below holds, each of those kernels stays inside
// its buffers.  A check reads only; a failure records SDF_ERR_INTERNAL in the
// plan's status word (unless an earlier error is there) and, for the first
// failure, the check's number and the index where it failed.  Checks:
//   1  bin_start[0] == 0            2  bin offsets ascending, within the binned points (<= K)
//   3  0 <= nuniq <= the bin's points
//   4  node code within the bin     5  node inside the grid     6  multiplicity >= 1
//   7  occ_start[0] == 0, occ_start[rows] <= bins
//   8  row list offsets ascending   9  occupied bin x inside the row   10  row list ascending
//  11  S finite   12  dS finite   13  d2S finite
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>

#include "sdf_internal.cuh"

namespace sdf {

static std::atomic<int> g_debug{-1};  // -1: the environment not read yet

bool debug_checks() {
    int v = g_debug.load();
    if (v < 0) {
        const char *e = getenv("SDF_DEBUG_CHECKS");
        const int want = (e && *e && strcmp(e, "0") != 0) ? 1 : 0;
        int expect = -1;
        g_debug.compare_exchange_strong(expect, want);
        v = g_debug.load();
    }
    return v == 1;
}

void set_debug_checks(bool on) { g_debug.store(on ? 1 : 0); }

static std::atomic<long long> g_corrupt_bins{0};
void set_corrupt_bins(long long v) { g_corrupt_bins.store(v); }

__device__ __forceinline__ void dbg_fail(DevScalars *d, int check, long long where) {
    if (atomicCAS(&d->dbg_check, 0, check) == 0) d->dbg_where = where;
    atomicCAS(&d->status, 0, (int)SDF_ERR_INTERNAL);
}

__global__ void k_check_bins(int D, int64_t nbins, int nb0, int nb1, int N0, int N1, int N2, int64_t K,
                             const int *__restrict__ bin_start, const int *__restrict__ nuniq,
                             const int *__restrict__ ucell, const int *__restrict__ ucount, DevScalars *d) {
    const int tot = bin_start[nbins];
    if (tot < 0 || tot > K) {  // the node lists hold K entries
        if (blockIdx.x == 0 && threadIdx.x == 0) dbg_fail(d, 2, nbins);
        return;
    }
    const int ncode = (D == 3) ? 512 : 64;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nbins; b += stride) {
        const int s = bin_start[b], e = bin_start[b + 1];
        if (b == 0 && s != 0) dbg_fail(d, 1, 0);
        if (s < 0 || e < s || e > tot) {
            dbg_fail(d, 2, b);
            continue;
        }
        const int n = nuniq[b];
        if (n < 0 || n > e - s) {
            dbg_fail(d, 3, b);
            continue;
        }
        const int bx = (int)(b % nb0), by = (int)((b / nb0) % nb1), bz = (int)(b / ((int64_t)nb0 * nb1));
        for (int j = 0; j < n; ++j) {
            const int lc = ucell[s + j];
            if (lc < 0 || lc >= ncode) {
                dbg_fail(d, 4, s + j);
                continue;
            }
            const int x = bx * 8 + (lc & 7), y = by * 8 + ((lc >> 3) & 7), z = bz * 8 + (lc >> 6);
            if (x >= N0 || y >= N1 || (D == 3 && z >= N2)) dbg_fail(d, 5, s + j);
            if (ucount[s + j] < 1) dbg_fail(d, 6, s + j);
        }
    }
}

__global__ void k_check_occ(int64_t nrows, int nb0, int64_t cap, const int *__restrict__ occ_start,
                            const int *__restrict__ occ_x, DevScalars *d) {
    const int tot = occ_start[nrows];
    const bool head_ok = occ_start[0] == 0 && tot >= 0 && tot <= cap;
    if (blockIdx.x == 0 && threadIdx.x == 0 && !head_ok) dbg_fail(d, 7, 0);
    if (!head_ok) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += stride) {
        const int a = occ_start[r], b = occ_start[r + 1];
        if (a < 0 || b < a || b > tot) {
            dbg_fail(d, 8, r);
            continue;
        }
        for (int i = a; i < b; ++i) {
            const int x = occ_x[i];
            if (x < 0 || x >= nb0) dbg_fail(d, 9, i);
            if (i > a && x <= occ_x[i - 1]) dbg_fail(d, 10, i);
        }
    }
}

template <typename T>
__global__ void k_check_finite(int64_t n, const T *__restrict__ a, int check, DevScalars *d) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        if (!isfinite(a[i])) dbg_fail(d, check, i);
}

// The first bin (in bin order) wholly inside the grid whose points are all
// distinct nodes and that some later bin follows with points: its count grows
// by one, so its list takes in the next occupied bin's first node (a valid
// node code, whose node lies in this bin's box and so inside the grid).
__global__ void __launch_bounds__(1024) k_corrupt_bins(int D, int64_t nbins, int nb0, int nb1, int N0, int N1,
                                                       int N2, const int *__restrict__ bin_start, int *nuniq) {
    __shared__ long long s_first;
    if (threadIdx.x == 0) s_first = nbins;
    __syncthreads();
    const int tot = bin_start[nbins];
    for (int64_t b = threadIdx.x; b < nbins; b += blockDim.x) {
        const int bx = (int)(b % nb0), by = (int)((b / nb0) % nb1), bz = (int)(b / ((int64_t)nb0 * nb1));
        const bool inside = bx * 8 + 8 <= N0 && by * 8 + 8 <= N1 && (D == 2 || bz * 8 + 8 <= N2);
        const int s = bin_start[b], e = bin_start[b + 1];
        if (inside && e > s && nuniq[b] == e - s && e < tot) atomicMin(&s_first, (long long)b);
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_first < nbins) nuniq[s_first] += 1;
}

cudaError_t debug_after_binning(sdf_plan_impl *p) {
    cudaStream_t st = p->stream;
    if (g_corrupt_bins.load() != 0 && p->D >= 2) {
        k_corrupt_bins<<<1, 1024, 0, st>>>(p->D, p->nbins, (int)p->nb[0], (int)p->nb[1], (int)p->N[0],
                                           (int)p->N[1], (int)p->N[2], p->bin_start, p->bin_nuniq);
    }
    if (debug_checks() && p->D >= 2) {
        const unsigned g = (unsigned)std::min<int64_t>((p->nbins + 255) / 256, (int64_t)sm_count() * 8);
        k_check_bins<<<g, 256, 0, st>>>(p->D, p->nbins, (int)p->nb[0], (int)p->nb[1], (int)p->N[0], (int)p->N[1],
                                        (int)p->N[2], p->last_K, p->bin_start, p->bin_nuniq, p->ucell, p->ucount,
                                        p->dsc);
    }
    return cudaGetLastError();
}

cudaError_t debug_after_cheb(sdf_plan_impl *p, cudaStream_t st) {
    if (!debug_checks() || !p->occ_start) return cudaSuccess;
    const int64_t nrows = bin_rows(p);
    const unsigned g = (unsigned)std::min<int64_t>((nrows + 255) / 256, (int64_t)sm_count() * 8);
    k_check_occ<<<g, 256, 0, st>>>(nrows, (int)p->nb[0], p->nbins, p->occ_start, p->occ_x, p->dsc);
    return cudaGetLastError();
}

cudaError_t debug_scan_outputs(sdf_plan_impl *p, const void *S, const void *dS, const void *d2S) {
    if (!debug_checks()) return cudaSuccess;
    const int D = p->D;
    const int64_t nn = p->nnodes;
    const int64_t nd = (D == 1) ? 1 : D, nh = (D == 1) ? 1 : D * (D + 1) / 2;
    const void *arr[3] = {S, dS, d2S};
    const int64_t cnt[3] = {nn, nn * nd, nn * nh};
    for (int k = 0; k < 3; ++k) {
        if (!arr[k]) continue;
        const unsigned g = (unsigned)std::min<int64_t>((cnt[k] + 255) / 256, (int64_t)sm_count() * 8);
        if (p->prec == SDF_FP64)
            k_check_finite<double><<<g, 256, 0, p->stream>>>(cnt[k], (const double *)arr[k], 11 + k, p->dsc);
        else
            k_check_finite<float><<<g, 256, 0, p->stream>>>(cnt[k], (const float *)arr[k], 11 + k, p->dsc);
    }
    return cudaGetLastError();
}

}  // namespace sdf
