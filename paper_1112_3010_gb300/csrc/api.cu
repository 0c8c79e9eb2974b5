// api.cu -- the C ABI declared in include/sdf.h: plan creation (kernel set,
// transform programme, workspace), execute orchestration and status.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <stdio.h>
#include <stdlib.h>
#include <sys/stat.h>

#include <atomic>
#include <chrono>
#include <cmath>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "green.cuh"
#include "sdf_internal.cuh"

namespace sdf {
int kernel_parity(int id, int D);
cudaError_t build_kernel_list(sdf_plan_impl *p, const std::vector<int> &ids);
}  // namespace sdf

using namespace sdf;

static thread_local char g_last_error[256] = "";

static sdf_status cuda_fail(cudaError_t e) {
    if (e == cudaErrorMemoryAllocation) {
        snprintf(g_last_error, sizeof g_last_error, "%s", cudaGetErrorString(e));
        cudaGetLastError();
        return SDF_ERR_OOM;
    }
    snprintf(g_last_error, sizeof g_last_error, "%s", cudaGetErrorString(e));
    cudaGetLastError();  // a later call must not pick this error up again
    return SDF_ERR_CUDA;
}

#define CK(x)                                   \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

// Noise constants C_p of the transform error model: the largest
// |phi_computed - phi| over a grid stays below
// C_p u_p sqrt(log2 n) ||k||_1 ||g||_2 / sqrt(n), with ||k||_1 the larger
// stored l1 norm of the channel's packed pair.  Calibrated on GB300 against
// the FP64 oracle (largest ratios seen: 5.9 for double, 4.8 for float
// transforms, over 2D/3D point sets with tau/h from 0.5 to 1.5); 12 leaves a
// factor-two margin.
static const double kNoiseC32 = 12.0;
static const double kNoiseC64 = 12.0;

static int64_t next_pow2(int64_t v) {
    int64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

static double zeta_re(int nodd) { const int q = nodd & 3; return q == 0 ? 1.0 : (q == 2 ? -1.0 : 0.0); }
static double zeta_im(int nodd) { const int q = nodd & 3; return q == 1 ? -1.0 : (q == 3 ? 1.0 : 0.0); }

namespace sdf {
cudaError_t build_spectra(sdf_plan_impl *p);

double hessian_scale(const sdf_plan_impl *p) { return p->tau * p->h / (p->tau + p->h); }

void set_last_error(const char *msg) { snprintf(g_last_error, sizeof g_last_error, "%s", msg); }

// theta_p = theta_coef(p, precision) * ||g||_2 (see include/sdf.h, trust region)
double theta_coef(const sdf_plan_impl *p, int prec) {
    const double n = (double)p->M[0] * (double)p->M[1] * (p->D == 3 ? (double)p->M[2] : 1.0);
    const double base = sqrt(log2(n)) / sqrt(n) * p->q_factor / kTrustEps;
    return prec == SDF_FP64 ? p->noise_c64 * ldexp(1.0, -53) * base : p->noise_c32 * ldexp(1.0, -24) * base;
}

// ---- test hooks (sdf_debug_hook): a device allocation that fails on
// request, and the poll limit of the epilogue's TMA waits
static std::atomic<long long> g_fail_alloc{0};   // > 0: the count-down to the allocation that fails
static std::atomic<long long> g_tma_polls{0};    // > 0: non-blocking polls before a TMA wait expires

cudaError_t dev_alloc(void **ptr, size_t bytes) {
    long long c = g_fail_alloc.load();
    while (c > 0 && !g_fail_alloc.compare_exchange_weak(c, c - 1)) {
    }
    if (c == 1) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;  // as the runtime reports an exhausted device
    }
    return cudaMalloc(ptr, bytes);
}

unsigned tma_wait_polls() { return (unsigned)g_tma_polls.load(); }

// Multiprocessors of the current device (grid sizes of the grid-stride
// kernels), looked up once per device.
int sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 152;
    }
    if (!cache[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            n = 152;
        }
        cache[dev] = n;
    }
    return cache[dev];
}

ScopedRange::ScopedRange(const char *name) { nvtxRangePushA(name); }
ScopedRange::~ScopedRange() { nvtxRangePop(); }

void prof_begin(sdf_plan_impl *p, const char *name, cudaStream_t st) {
    ++p->nlaunch;
    nvtxRangePushA(name);  // one NVTX range per kernel launch (closed by prof_end)
    if (!p->prof_on) return;
    ProfRec r;
    r.name = name;
    for (cudaEvent_t *ev : {&r.a, &r.b}) {
        if (!p->prof_pool.empty()) {
            *ev = p->prof_pool.back();
            p->prof_pool.pop_back();
        } else if (cudaEventCreate(ev) != cudaSuccess) {
            *ev = nullptr;
        }
    }
    if (r.a) cudaEventRecord(r.a, st);
    p->prof_recs.push_back(r);
}

void prof_end(sdf_plan_impl *p, cudaStream_t st) {
    nvtxRangePop();
    if (!p->prof_on || p->prof_recs.empty()) return;
    ProfRec &r = p->prof_recs.back();
    if (r.b) cudaEventRecord(r.b, st);
}

// Add kernels (if absent) and build their spectra.
cudaError_t build_kernel_list(sdf_plan_impl *p, const std::vector<int> &ids) {
    std::vector<KernelSpec> keep = p->kernels;
    std::vector<KernelSpec> fresh;
    for (int id : ids) {
        if (p->kslot[id] >= 0) continue;
        KernelSpec k;
        k.id = id;
        k.parity = kernel_parity(id, p->D);
        k.l1 = 0;
        // The Hessian kernels are up to (1/tau + 1/h) times larger than f; they
        // are stored scaled to f's size so that a channel packed with one of
        // them in a complex inverse transform does not inherit its rounding
        // noise.  The epilogue undoes the scale.
        k.scale = (id >= KER_HXX && id <= KER_HYZ) ? hessian_scale(p) : 1.0;
        k.c = nullptr;
        fresh.push_back(k);
    }
    if (fresh.empty()) return cudaSuccess;
    p->kernels = fresh;
    cudaError_t e = build_spectra(p);
    fresh = p->kernels;
    p->kernels = keep;
    for (auto &k : fresh) {
        p->kslot[k.id] = (int)p->kernels.size();
        p->kernels.push_back(k);
    }
    return e;
}
}  // namespace sdf

static void add_pair(sdf_plan_impl *p, int kA, int chA, int kB, int chB) {
    Group &g = p->group[p->ngroup];
    g.nterm = 0;
    const int sa = p->kslot[kA];
    const int na = __builtin_popcount((unsigned)p->kernels[sa].parity);
    g.term[g.nterm++] = Term{sa, 0, zeta_re(na), zeta_im(na)};
    p->gch[p->ngroup][0] = chA;
    p->gch[p->ngroup][1] = CH_NONE;
    if (kB >= 0) {
        const int sb = p->kslot[kB];
        const int nb = __builtin_popcount((unsigned)p->kernels[sb].parity);
        // i * zeta
        g.term[g.nterm++] = Term{sb, 0, -zeta_im(nb), zeta_re(nb)};
        p->gch[p->ngroup][1] = chB;
    }
    ++p->ngroup;
}

static void add_mu(sdf_plan_impl *p) {
    Group &g = p->group[p->ngroup];
    g.nterm = 0;
    const double pi = 3.14159265358979323846;
    if (p->D == 2) {
        // mu = Re[(Khat_W1 + i Khat_W2) Fhat_1] / (2 pi)   (eq. kappadiscretefinal)
        const int s1 = p->kslot[KER_W1], s2 = p->kslot[KER_W2];
        const int n1 = __builtin_popcount((unsigned)p->kernels[s1].parity);
        const int n2 = __builtin_popcount((unsigned)p->kernels[s2].parity);
        const double c = 1.0 / (2.0 * pi);
        g.term[g.nterm++] = Term{s1, 1, c * zeta_re(n1), c * zeta_im(n1)};
        g.term[g.nterm++] = Term{s2, 1, -c * zeta_im(n2), c * zeta_re(n2)};
    } else {
        // mu = -Re[(Khat_W1 - i Khat_W2) Fhat_1 + Khat_W3 Fhat_2] / (4 pi)   (eq. mudef)
        const int s1 = p->kslot[KER_W1], s2 = p->kslot[KER_W2], s3 = p->kslot[KER_W3];
        const int n1 = __builtin_popcount((unsigned)p->kernels[s1].parity);
        const int n2 = __builtin_popcount((unsigned)p->kernels[s2].parity);
        const int n3 = __builtin_popcount((unsigned)p->kernels[s3].parity);
        const double c = -1.0 / (4.0 * pi);
        g.term[g.nterm++] = Term{s1, 1, c * zeta_re(n1), c * zeta_im(n1)};
        // -i * zeta2 * c
        g.term[g.nterm++] = Term{s2, 1, c * zeta_im(n2), -c * zeta_re(n2)};
        g.term[g.nterm++] = Term{s3, 2, c * zeta_re(n3), c * zeta_im(n3)};
    }
    p->gch[p->ngroup][0] = CH_MU;
    p->gch[p->ngroup][1] = CH_NONE;
    ++p->ngroup;
}

static size_t vbytes(const sdf_plan_impl *p) { return p->prec == SDF_FP64 ? sizeof(double2) : sizeof(float2); }

namespace sdf {

// Grid geometry of a plan: padded sizes, bins, node counts, defaults.
void plan_geometry(sdf_plan_impl *p, int D, const int64_t *dims, double h, double tau, int precision,
                   unsigned outputs, void *stream) {
    p->D = D;
    p->prec = precision;
    outputs |= SDF_OUT_S;
    if (outputs & SDF_OUT_D2S) outputs |= SDF_OUT_DS;
    p->outputs = outputs;
    p->h = h;
    p->tau = tau;
    p->stream = reinterpret_cast<cudaStream_t>(stream);
    p->nnodes = 1;
    p->nbins = 1;
    for (int a = 0; a < 3; ++a) {
        p->N[a] = (a < D) ? dims[a] : 1;
        p->M[a] = (a < D) ? std::max<int64_t>(16, next_pow2(2 * p->N[a] - 1)) : 1;
        p->logM[a] = line_code(p->M[a]);
        p->nb[a] = (p->N[a] + kBin - 1) / kBin;
        p->nnodes *= p->N[a];
        p->nbins *= p->nb[a];
    }
    for (int i = 0; i < KER_COUNT; ++i) p->kslot[i] = -1;
    p->noise_c32 = kNoiseC32;
    p->noise_c64 = kNoiseC64;
}

// Kernels the requested outputs need.
std::vector<int> plan_kernel_ids(const sdf_plan_impl *p) {
    const int D = p->D;
    const bool ds = p->outputs & SDF_OUT_DS, d2 = p->outputs & SDF_OUT_D2S, sg = p->outputs & SDF_OUT_SIGN;
    std::vector<int> ids = {KER_PHI};
    if (D == 1) {
        if (ds) ids.push_back(KER_GX);
        if (d2) ids.push_back(KER_HXX);
        return ids;
    }
    if (ds) {
        ids.push_back(KER_GX);
        ids.push_back(KER_GY);
        if (D == 3) ids.push_back(KER_GZ);
    }
    if (d2) {
        ids.push_back(KER_HXX);
        ids.push_back(KER_HYY);
        if (D == 3) ids.push_back(KER_HZZ);
        ids.push_back(KER_HXY);
        if (D == 3) {
            ids.push_back(KER_HXZ);
            ids.push_back(KER_HYZ);
        }
    }
    if (sg) {
        ids.push_back(KER_W1);
        ids.push_back(KER_W2);
        if (D == 3) ids.push_back(KER_W3);
    }
    return ids;
}

// Transform programme (input fields, packed output groups) and the noise-model
// factor Q; needs the kernel l1 norms.
void plan_programme(sdf_plan_impl *p) {
    const int D = p->D;
    const double tau = p->tau;
    const bool ds = p->outputs & SDF_OUT_DS, d2 = p->outputs & SDF_OUT_D2S, sg = p->outputs & SDF_OUT_SIGN;
    p->nfield = sg ? (D == 2 ? 2 : 3) : 1;
    p->ngroup = 0;
    if (D == 1) {
        // one line, one CTA (line1d.cu): phi and phi' share a transform, the
        // Hessian kernel has its own
        add_pair(p, KER_PHI, CH_PHI, ds ? KER_GX : -1, CH_GX);
        if (d2) add_pair(p, KER_HXX, CH_HXX, -1, CH_NONE);
    } else if (D == 2) {
        add_pair(p, KER_PHI, CH_PHI, ds ? KER_GX : -1, CH_GX);
        if (ds) add_pair(p, KER_GY, CH_GY, d2 ? KER_HXX : -1, CH_HXX);
        if (d2) add_pair(p, KER_HYY, CH_HYY, KER_HXY, CH_HXY);
    } else {
        add_pair(p, KER_PHI, CH_PHI, ds ? KER_GX : -1, CH_GX);
        if (ds) add_pair(p, KER_GY, CH_GY, KER_GZ, CH_GZ);
        if (d2) {
            add_pair(p, KER_HXX, CH_HXX, KER_HYY, CH_HYY);
            add_pair(p, KER_HZZ, CH_HZZ, KER_HXY, CH_HXY);
            add_pair(p, KER_HXZ, CH_HXZ, KER_HYZ, CH_HYZ);
        }
    }
    if (sg) add_mu(p);
    // noise-model factor Q (how phi's error enters each requested output).
    // Noise of a channel ~ the larger stored l1 norm of its packed pair,
    // times the channel's unscale factor.
    const Channel base_ch[] = {CH_PHI, CH_GX, CH_GY, CH_GZ, CH_HXX, CH_HYY, CH_HZZ, CH_HXY, CH_HXZ, CH_HYZ};
    const int base_k[] = {KER_PHI, KER_GX, KER_GY, KER_GZ, KER_HXX, KER_HYY, KER_HZZ, KER_HXY, KER_HXZ, KER_HYZ};
    auto kern_of = [&](int ch) {
        for (int i = 0; i < 10; ++i)
            if (base_ch[i] == ch) return base_k[i];
        return -1;
    };
    auto stored_l1 = [&](int ch) {
        const int id = kern_of(ch);
        if (id < 0 || p->kslot[id] < 0) return 0.0;
        const KernelSpec &k = p->kernels[p->kslot[id]];
        return k.l1 * k.scale;
    };
    double f = 0, gmax = 0, hmax = 0;
    for (int g = 0; g < p->ngroup; ++g) {
        const double pair = std::max(stored_l1(p->gch[g][0]), stored_l1(p->gch[g][1]));
        for (int hh = 0; hh < 2; ++hh) {
            const int ch = p->gch[g][hh];
            const int id = kern_of(ch);
            if (id < 0) continue;
            const double n = pair / p->kernels[p->kslot[id]].scale;
            if (ch == CH_PHI) f = n;
            else if (ch >= CH_GX && ch <= CH_GZ) gmax = std::max(gmax, n);
            else hmax = std::max(hmax, n);
        }
    }
    double q = f;
    if (ds) q = std::max(q, f + gmax);
    if (d2) q = std::max(q, tau * hmax + 2 * gmax + 2 * f);
    p->q_factor = q;
    p->q_f = f;
    p->q_g = gmax;
    p->q_h = hmax;
}

// Sizes of the two transform buffers (bytesA, bytesB).
void plan_buffer_sizes(sdf_plan_impl *p) {
    const int64_t N1 = p->N[1], N2 = p->N[2], M0 = p->M[0], M1 = p->M[1];
    const int64_t ng = std::max(p->ngroup, 2);
    const int64_t nf = p->nfield;
    int64_t a, b;
    if (p->D == 2) {
        a = nf * M0 * N1;
        b = ng * M0 * N1;
    } else {
        a = std::max(nf * M0 * N2 * N1, ng * M1 * M0 * N2);
        b = std::max(nf * M1 * M0 * N2, ng * M0 * N2 * N1);
    }
    p->bytesA = a * vbytes(p);
    p->bytesB = b * vbytes(p);
}

}  // namespace sdf

static cudaError_t alloc(void **ptr, size_t bytes, size_t *acc) {
    cudaError_t e = dev_alloc(ptr, bytes);
    if (e == cudaSuccess && acc) *acc += bytes;
    return e;
}

static void free_plan(sdf_plan_impl *p) {
    if (!p) return;
    if (p->stream) cudaStreamSynchronize(p->stream);
    if (!p->shares_spectra)
        for (auto &k : p->kernels) cudaFree(k.c);
    for (int a = 0; a < 3; ++a) cudaFree(p->tw[a]);
    cudaFree(p->bufA);
    cudaFree(p->bufB);
    cudaFree(p->pt_key);
    cudaFree(p->pt_lc);
    cudaFree(p->pt_entry);
    cudaFree(p->bin_count);
    cudaFree(p->bin_start);
    cudaFree(p->bin_fill);
    cudaFree(p->bin_nuniq);
    cudaFree(p->ucell);
    cudaFree(p->ucount);
    cudaFree(p->uw);
    cudaFree(p->cheb);
    cudaFree(p->occ_start);
    cudaFree(p->occ_x);
    cudaFree(p->occ_tmp);
    cudaFree(p->tile_flag);
    cudaFree(p->flags_int);
    cudaFree(p->sign_int);
    cudaFree(p->dsc);
    cudaFree(p->staging);
    cudaFree(p->adj_planes);
    cudaFree(p->adj_part);
    if (p->hsc) cudaFreeHost(p->hsc);
    for (auto &r : p->prof_recs) {
        if (r.a) cudaEventDestroy(r.a);
        if (r.b) cudaEventDestroy(r.b);
    }
    for (auto ev : p->prof_pool) cudaEventDestroy(ev);
}

template <typename T>
static cudaError_t upload_twiddles(void **dst, int64_t L, size_t *acc) {
    using V = typename cplx_t<T>::type;
    std::vector<V> h(L);
    fill_twiddle_table(line_code(L), h.data());
    cudaError_t e = alloc(dst, sizeof(V) * L, acc);
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, h.data(), sizeof(V) * L, cudaMemcpyHostToDevice);
}

// Largest padded line the transforms take per dimension (the FFT core runs
// up to 8192-point lines; 3D buffers are kept to 1024^3).
static int64_t max_padded(int D) { return D == 3 ? 1024 : 8192; }

// Smallest 3 * 2^k >= v (k >= 4), or 0 when it is not below the power of two.
static int64_t r3_padding(int64_t v) {
    int64_t m = 48;
    while (m < v) m *= 2;
    return m < next_pow2(v) ? m : 0;
}

namespace sdf {
// Rebuild what depends on the padded sizes (twiddles, kernel spectra,
// transform buffers, the adjoint's programme) for padded sizes M; with
// share_from, take that plan's spectra (same geometry and M).  On error the
// plan is left without buffers and must be destroyed.
sdf_status plan_repad(sdf_plan_impl *p, const int64_t *M, const sdf_plan_impl *share_from) {
    CK(cudaStreamSynchronize(p->stream));
    const size_t vb = vbytes(p);
    const int64_t esz = (p->prec == SDF_FP64) ? 8 : 4;
    for (int a = 0; a < p->D; ++a) {
        cudaFree(p->tw[a]);
        p->tw[a] = nullptr;
        p->workspace_bytes -= vb * p->M[a];
    }
    if (!p->shares_spectra) {
        for (auto &k : p->kernels) {
            cudaFree(k.c);
            p->workspace_bytes -= esz * spec_rows(p) * spec_row_len(p);
        }
    }
    p->kernels.clear();
    for (int i = 0; i < KER_COUNT; ++i) p->kslot[i] = -1;
    if (p->adj_ngroup > 0) {
        cudaFree(p->adj_planes);
        cudaFree(p->adj_part);
        p->adj_planes = nullptr;
        p->adj_part = nullptr;
        p->workspace_bytes -= esz * (p->D + 1) * p->nnodes + sizeof(double) * 2 * kAdjParts;
        p->adj_ngroup = 0;
    }
    cudaFree(p->bufA);
    cudaFree(p->bufB);
    p->bufA = p->bufB = nullptr;
    p->workspace_bytes -= p->bytesA + p->bytesB;
    for (int a = 0; a < p->D; ++a) {
        p->M[a] = M[a];
        p->logM[a] = line_code(M[a]);
    }
    for (int a = 0; a < p->D; ++a) {
        if (p->prec == SDF_FP64) CK(upload_twiddles<double>(&p->tw[a], p->M[a], &p->workspace_bytes));
        else CK(upload_twiddles<float>(&p->tw[a], p->M[a], &p->workspace_bytes));
    }
    if (share_from) {
        p->kernels = share_from->kernels;
        for (int i = 0; i < KER_COUNT; ++i) p->kslot[i] = share_from->kslot[i];
        p->shares_spectra = true;
    } else {
        p->shares_spectra = false;
        CK(build_kernel_list(p, plan_kernel_ids(p)));
    }
    plan_programme(p);
    plan_buffer_sizes(p);
    CK(alloc(&p->bufA, p->bytesA, &p->workspace_bytes));
    CK(alloc(&p->bufB, p->bytesB, &p->workspace_bytes));
    CK(cudaDeviceSynchronize());
    return SDF_OK;
}

// Padded-size choices of a plan (sdf_plan_set_padding rules).
bool padding_ok(const sdf_plan_impl *p, const int64_t *M) {
    for (int a = 0; a < p->D; ++a) {
        const int64_t need = std::max<int64_t>(16, 2 * p->N[a] - 1);
        if (M[a] < need || M[a] > max_padded(p->D) || line_code(M[a]) < 0) return false;
        if (line_r3(line_code(M[a])) && M[a] < 48) return false;
    }
    return true;
}
}  // namespace sdf

extern "C" {

const char *sdf_status_string(sdf_status s) {
    switch (s) {
        case SDF_OK: return "ok";
        case SDF_ERR_INVALID_ARG: return "invalid argument";
        case SDF_ERR_UNSUPPORTED: return "unsupported configuration";
        case SDF_ERR_POINT_OUT_OF_GRID: return "a point snapped outside the grid";
        case SDF_ERR_OOM: return "device out of memory";
        case SDF_ERR_CUDA: return "CUDA runtime error";
        case SDF_ERR_TIMEOUT: return "a bounded device wait expired";
        case SDF_ERR_CAPACITY: return "input exceeds a fixed-size buffer";
        case SDF_ERR_INTERNAL: return "a device-side consistency check failed";
        default: return "unknown status";
    }
}

const char *sdf_last_error(void) { return g_last_error; }

sdf_status sdf_plan_create(sdf_plan *out, int D, const int64_t *dims, double h, double tau, int precision,
                           unsigned outputs, void *stream) {
    return sdf::plan_create_shared(out, D, dims, h, tau, precision, outputs, stream, nullptr);
}

}  // extern "C"

// A plan; with share_from, the kernel spectra of that plan (same D, dims, h,
// tau, precision and outputs) are used instead of building new ones.
sdf_status sdf::plan_create_shared(sdf_plan *out, int D, const int64_t *dims, double h, double tau, int precision,
                                   unsigned outputs, void *stream, const sdf_plan_impl *share_from) {
    if (!out) return SDF_ERR_INVALID_ARG;
    *out = nullptr;
    if (D < 1 || D > 3) return SDF_ERR_UNSUPPORTED;
    if (!dims || !(h > 0.0) || !(tau > 0.0) || !std::isfinite(h) || !std::isfinite(tau)) return SDF_ERR_INVALID_ARG;
    if (precision != SDF_FP64 && precision != SDF_FP32) return SDF_ERR_INVALID_ARG;
    if (outputs & ~15u) return SDF_ERR_INVALID_ARG;
    if (D == 1 && (outputs & SDF_OUT_SIGN)) {
        set_last_error("sdf_plan_create: no sign in 1D (the paper defines winding numbers in 2D, degrees in 3D)");
        return SDF_ERR_UNSUPPORTED;
    }
    const int64_t nmax = (D == 1) ? 2048 : ((D == 2) ? 4096 : 512);
    for (int a = 0; a < D; ++a)
        if (dims[a] < 2 || dims[a] > nmax) return SDF_ERR_UNSUPPORTED;
    auto t0 = std::chrono::steady_clock::now();
    sdf_plan_s *p = new (std::nothrow) sdf_plan_s();
    if (!p) return SDF_ERR_OOM;
    plan_geometry(p, D, dims, h, tau, precision, outputs, stream);
    outputs = p->outputs;
    const std::vector<int> ids = plan_kernel_ids(p);
    cudaError_t e;
#define PCK(x)                          \
    do {                                \
        e = (x);                        \
        if (e != cudaSuccess) {         \
            sdf_status s_ = cuda_fail(e); \
            free_plan(p);               \
            delete p;                   \
            return s_;                  \
        }                               \
    } while (0)
    // twiddles in the plan precision
    for (int a = 0; a < D; ++a) {
        if (precision == SDF_FP64) PCK(upload_twiddles<double>(&p->tw[a], p->M[a], &p->workspace_bytes));
        else PCK(upload_twiddles<float>(&p->tw[a], p->M[a], &p->workspace_bytes));
    }
    if (share_from) {
        p->kernels = share_from->kernels;
        for (int i = 0; i < KER_COUNT; ++i) p->kslot[i] = share_from->kslot[i];
        p->shares_spectra = true;
    } else {
        PCK(build_kernel_list(p, ids));
    }
    plan_programme(p);
    // workspace
    {
        plan_buffer_sizes(p);
        PCK(alloc(&p->bufA, p->bytesA, &p->workspace_bytes));
        PCK(alloc(&p->bufB, p->bytesB, &p->workspace_bytes));
        const int64_t nb = p->nbins;
        PCK(alloc((void **)&p->bin_count, sizeof(int) * (nb + 1), &p->workspace_bytes));
        PCK(alloc((void **)&p->bin_start, sizeof(int) * (nb + 1), &p->workspace_bytes));
        PCK(alloc((void **)&p->bin_fill, sizeof(int) * nb, &p->workspace_bytes));
        PCK(alloc((void **)&p->bin_nuniq, sizeof(int) * nb, &p->workspace_bytes));
        PCK(alloc((void **)&p->cheb, 2 * nb, &p->workspace_bytes));
        PCK(alloc((void **)&p->tile_flag, nb, &p->workspace_bytes));
        PCK(alloc((void **)&p->dsc, sizeof(DevScalars), &p->workspace_bytes));
        PCK(cudaMemset(p->dsc, 0, sizeof(DevScalars)));
        PCK(cudaMallocHost((void **)&p->hsc, sizeof(DevScalars)));
        if (precision == SDF_FP32) {
            PCK(alloc((void **)&p->flags_int, p->nnodes, &p->workspace_bytes));
            PCK(alloc((void **)&p->sign_int, p->nnodes, &p->workspace_bytes));
            PCK(alloc((void **)&p->occ_start, sizeof(int) * (bin_rows(p) + 1), &p->workspace_bytes));
            PCK(alloc((void **)&p->occ_x, sizeof(int) * nb, &p->workspace_bytes));
            PCK(alloc((void **)&p->occ_tmp, sizeof(int) * occ_tmp_len(p), &p->workspace_bytes));
        }
    }
    PCK(cudaDeviceSynchronize());
#undef PCK
    p->plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = p;
    return SDF_OK;
}

extern "C" {

static cudaError_t ensure_points(sdf_plan_impl *p, int64_t K) {
    if (K <= p->Kcap) return cudaSuccess;
    cudaStreamSynchronize(p->stream);
    cudaFree(p->pt_key);
    cudaFree(p->pt_lc);
    cudaFree(p->pt_entry);
    cudaFree(p->ucell);
    cudaFree(p->ucount);
    cudaFree(p->uw);
    p->pt_key = p->pt_lc = p->ucell = p->ucount = nullptr;
    p->pt_entry = nullptr;
    p->uw = nullptr;
    p->Kcap = 0;
    const int64_t cap = std::max<int64_t>(K, 1024);
    cudaError_t e;
    if ((e = dev_alloc((void **)&p->pt_key, sizeof(int) * cap)) != cudaSuccess) return e;
    if ((e = dev_alloc((void **)&p->pt_lc, sizeof(int) * cap)) != cudaSuccess) return e;
    if ((e = dev_alloc((void **)&p->pt_entry, sizeof(long long) * cap)) != cudaSuccess) return e;
    if ((e = dev_alloc((void **)&p->ucell, sizeof(int) * cap)) != cudaSuccess) return e;
    if ((e = dev_alloc((void **)&p->ucount, sizeof(int) * cap)) != cudaSuccess) return e;
    if ((e = dev_alloc((void **)&p->uw, sizeof(double) * 3 * cap)) != cudaSuccess) return e;
    p->Kcap = cap;
    return cudaSuccess;
}

static sdf_status check_execute_args(sdf_plan p, int64_t K, const double *points, const double *weights,
                                     const void *dS, const void *d2S, const int8_t *sign) {
    if (!p || !points) return SDF_ERR_INVALID_ARG;
    if (K < 1 || K >= (int64_t(1) << 31) - 1) return SDF_ERR_INVALID_ARG;
    if (dS && !(p->outputs & SDF_OUT_DS)) return SDF_ERR_INVALID_ARG;
    if (d2S && !(p->outputs & SDF_OUT_D2S)) return SDF_ERR_INVALID_ARG;
    if (sign && !((p->outputs & SDF_OUT_SIGN) && weights)) return SDF_ERR_INVALID_ARG;
    if (weights && !(p->outputs & SDF_OUT_SIGN)) return SDF_ERR_INVALID_ARG;
    return SDF_OK;
}

sdf_status sdf_execute(sdf_plan p, int64_t K, const double *points, const double *weights, void *S, void *dS,
                       void *d2S, int8_t *sign, uint8_t *flags) {
    ScopedRange range_("sdf_execute");
    sdf_status s = check_execute_args(p, K, points, weights, dS, d2S, sign);
    if (s != SDF_OK) return s;
    CK(ensure_points(p, K));
    p->last_K = K;
    p->nlaunch = 0;
    const bool ww = weights != nullptr;
    if (p->D == 1) {
        CK(launch_line1d(p, K, points, S, dS, d2S, flags));
        CK(debug_scan_outputs(p, S, dS, d2S));
        return SDF_OK;
    }
    CK(launch_points(p, K, points, weights));
    uint8_t *fl = flags;
    int8_t *sg = sign;
    if (p->prec == SDF_FP32) {
        if (!fl) fl = p->flags_int;
        if (ww && !sg) sg = p->sign_int;
        CK(cudaMemsetAsync(p->tile_flag, 0, p->nbins, p->stream));
        CK(launch_cheb(p));
    }
    CK(launch_forward(p, ww, nullptr, 0, nullptr));
    CK(launch_inverse_epilogue(p, ww, S, dS, d2S, sg, fl));
    if (p->prec == SDF_FP32) CK(launch_fixup(p, ww, S, dS, d2S, ww ? sg : nullptr, fl));
    if (flags) CK(launch_source_flags(p, flags));
    CK(debug_scan_outputs(p, S, dS, d2S));
    return SDF_OK;
}

// Host destinations of one plan's outputs in sdf_execute_multi_host (the
// device outputs given to multi_core are then the plan's staging buffers).
// early: S, dS and d2S are copied to the host as soon as the epilogue has
// written them, and the fix-up, which runs after that copy, writes its nodes
// straight into the host buffers (mS, mdS, md2: their device-mapped
// addresses); otherwise every output is copied after the plan's fix-up.
struct HostCopy {
    void *S, *dS, *d2S;
    int8_t *sign;
    uint8_t *flags;
    void *mS, *mdS, *md2;
    bool early;
};

static sdf_status multi_core(int n, const sdf_plan *plans, int64_t K, const double *points, const double *weights,
                             void *const *S, void *const *dS, void *const *d2S, int8_t *const *sign,
                             uint8_t *const *flags, const HostCopy *hc);

sdf_status sdf_execute_multi(int n, const sdf_plan *plans, int64_t K, const double *points, const double *weights,
                             void *const *S, void *const *dS, void *const *d2S, int8_t *const *sign,
                             uint8_t *const *flags) {
    ScopedRange range_("sdf_execute_multi");
    return multi_core(n, plans, K, points, weights, S, dS, d2S, sign, flags, nullptr);
}

static sdf_status multi_core(int n, const sdf_plan *plans, int64_t K, const double *points, const double *weights,
                             void *const *S, void *const *dS, void *const *d2S, int8_t *const *sign,
                             uint8_t *const *flags, const HostCopy *hc) {
    if (n < 1 || !plans || !plans[0] || !points) return SDF_ERR_INVALID_ARG;
    sdf_plan p0 = plans[0];
    auto at = [](auto *const *arr, int i) { return arr ? arr[i] : nullptr; };
    for (int i = 0; i < n; ++i) {
        sdf_plan p = plans[i];
        if (!p) return SDF_ERR_INVALID_ARG;
        for (int j = 0; j < i; ++j)
            if (plans[j] == p) return SDF_ERR_INVALID_ARG;
        bool same = p->D == p0->D && p->prec == p0->prec && p->outputs == p0->outputs && p->h == p0->h;
        for (int a = 0; a < 3; ++a) same = same && p->N[a] == p0->N[a] && p->M[a] == p0->M[a];
        if (!same) {
            set_last_error("sdf_execute_multi: the plans differ in D, dims, padded sizes, h, precision or outputs");
            return SDF_ERR_INVALID_ARG;
        }
        sdf_status s = check_execute_args(p, K, points, weights, at(dS, i), at(d2S, i), at(sign, i));
        if (s != SDF_OK) return s;
    }
    if (p0->D == 1) {
        // one CTA per line: nothing worth sharing
        for (int i = 0; i < n; ++i) {
            sdf_plan p = plans[i];
            sdf_status s = sdf_execute(p, K, points, weights, at(S, i), at(dS, i), at(d2S, i), at(sign, i),
                                       at(flags, i));
            if (s != SDF_OK) return s;
            if (!hc) continue;
            const size_t esz = (p->prec == SDF_FP64) ? sizeof(double) : sizeof(float);
            const int64_t nn = p->nnodes;
            const HostCopy &h = hc[i];
            if (h.S) CK(cudaMemcpyAsync(h.S, at(S, i), esz * nn, cudaMemcpyDeviceToHost, p->stream));
            if (h.dS) CK(cudaMemcpyAsync(h.dS, at(dS, i), esz * nn, cudaMemcpyDeviceToHost, p->stream));
            if (h.d2S) CK(cudaMemcpyAsync(h.d2S, at(d2S, i), esz * nn, cudaMemcpyDeviceToHost, p->stream));
            if (h.sign) CK(cudaMemcpyAsync(h.sign, at(sign, i), nn, cudaMemcpyDeviceToHost, p->stream));
            if (h.flags) CK(cudaMemcpyAsync(h.flags, at(flags, i), nn, cudaMemcpyDeviceToHost, p->stream));
        }
        return SDF_OK;
    }
    const bool ww = weights != nullptr;
    for (int i = 0; i < n; ++i) {
        CK(ensure_points(plans[i], K));
        plans[i]->last_K = K;
        plans[i]->nlaunch = 0;
    }
    cudaStream_t st0 = p0->stream;
    // events: entry (one per plan), after each fused pass, after each plan's
    // work, after the shared part, after plans[0]'s sign, after plans[0]'s
    // Chebyshev map
    std::vector<cudaEvent_t> ev(3 * n + 3, nullptr);
    auto cleanup = [&]() {
        for (auto &x : ev)
            if (x) cudaEventDestroy(x);
    };
#define MCK(x)                       \
    do {                             \
        cudaError_t e_ = (x);        \
        if (e_ != cudaSuccess) {     \
            cleanup();               \
            return cuda_fail(e_);    \
        }                            \
    } while (0)
    for (auto &x : ev) MCK(cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
    cudaEvent_t *ev_entry = ev.data() + 2 * n + 2;
    // st0 writes into the other plans' buffers (binned points, fused outputs):
    // it first waits for whatever their own streams already hold
    for (int i = 1; i < n; ++i) {
        MCK(cudaEventRecord(ev_entry[i], plans[i]->stream));
        MCK(cudaStreamWaitEvent(st0, ev_entry[i], 0));
    }
    // the points and the tau-independent forward transforms, once, on p0's stream
    MCK(launch_points(p0, K, points, weights));
    MCK(launch_forward_shared_part(p0, ww));
    // the others' fix-up, Chebyshev map and source flags read the binned points:
    // copied here, before p0's own later kernels update its scalars
    for (int i = 1; i < n; ++i) {
        sdf_plan p = plans[i];
        MCK(cudaMemcpyAsync(p->bin_start, p0->bin_start, sizeof(int) * (p0->nbins + 1), cudaMemcpyDeviceToDevice, st0));
        MCK(cudaMemcpyAsync(p->bin_nuniq, p0->bin_nuniq, sizeof(int) * p0->nbins, cudaMemcpyDeviceToDevice, st0));
        MCK(cudaMemcpyAsync(p->ucell, p0->ucell, sizeof(int) * K, cudaMemcpyDeviceToDevice, st0));
        MCK(cudaMemcpyAsync(p->ucount, p0->ucount, sizeof(int) * K, cudaMemcpyDeviceToDevice, st0));
        const size_t o = offsetof(DevScalars, wmax);
        MCK(cudaMemcpyAsync(reinterpret_cast<char *>(p->dsc) + o, reinterpret_cast<const char *>(p0->dsc) + o,
                            sizeof(DevScalars) - o, cudaMemcpyDeviceToDevice, st0));
    }
    // the sign does not depend on tau or the kernel set: plans[0] computes it,
    // the others read it (their fused pass and epilogue skip the mu group)
    const bool share_sign = ww && n > 1 && (p0->outputs & SDF_OUT_SIGN);
    int8_t *sign0 = at(sign, 0);
    if (share_sign && !sign0) {
        if (!p0->sign_int) MCK(alloc((void **)&p0->sign_int, p0->nnodes, &p0->workspace_bytes));
        sign0 = p0->sign_int;
    }
    MCK(cudaEventRecord(ev[2 * n], st0));
    // two plans: one fused launch does both (the second plan's products and
    // inverses reuse the forward transform of field 0)
    const bool pair = n == 2;
    // per plan: Chebyshev map, the fused pass on p0's transforms
    for (int i = 0; i < n; ++i) {
        sdf_plan p = plans[i];
        if (i > 0) MCK(cudaStreamWaitEvent(p->stream, ev[2 * n], 0));
        if (p->prec == SDF_FP32) {
            // with two plans, plans[0]'s map goes on the second stream, beside
            // the fused launch that occupies its own
            cudaStream_t sc = (pair && i == 0) ? plans[1]->stream : p->stream;
            if (sc != p->stream) MCK(cudaStreamWaitEvent(sc, ev[2 * n], 0));
            MCK(cudaMemsetAsync(p->tile_flag, 0, p->nbins, sc));
            MCK(launch_cheb(p, sc));
            if (sc != p->stream) MCK(cudaEventRecord(ev[3 * n + 2], sc));
        }
        if (!(pair && i == 1)) MCK(launch_forward_from(p, p0, share_sign && i > 0, (pair && i == 0) ? plans[1] : nullptr));
        MCK(cudaEventRecord(ev[i], p->stream));
    }
    // 3D: p0's inverse y-pass overwrites the buffer the others' fused passes read
    if (p0->D == 3)
        for (int i = 1; i < n; ++i) MCK(cudaStreamWaitEvent(st0, ev[i], 0));
    for (int i = 0; i < n; ++i) {
        sdf_plan p = plans[i];
        uint8_t *fl = at(flags, i);
        int8_t *sg = at(sign, i);
        if (p->prec == SDF_FP32 && !fl) fl = p->flags_int;
        const int8_t *sin = nullptr;
        if (share_sign && i == 0) {
            sg = sign0;
        } else if (share_sign) {
            MCK(cudaStreamWaitEvent(p->stream, ev[2 * n + 1], 0));  // plans[0]'s sign is written
            sin = sign0;
        } else if (p->prec == SDF_FP32 && ww && !sg) {
            sg = p->sign_int;
        }
        if (pair && i == 1) MCK(cudaStreamWaitEvent(p->stream, ev[0], 0));  // its fused pass ran on st0
        if (pair && i == 0 && p->prec == SDF_FP32 && plans[1]->stream != p->stream)
            MCK(cudaStreamWaitEvent(p->stream, ev[3 * n + 2], 0));  // its map and cleared tile flags
        MCK(launch_inverse_epilogue(p, ww, at(S, i), at(dS, i), at(d2S, i), sg, fl, sin));
        if (share_sign && i == 0) MCK(cudaEventRecord(ev[2 * n + 1], p->stream));
        const int8_t *sfix = ww ? (sg ? sg : sin) : nullptr;
        void *fS = at(S, i), *fdS = at(dS, i), *fd2 = at(d2S, i);
        const size_t esz = (p->prec == SDF_FP64) ? sizeof(double) : sizeof(float);
        const int64_t nn = p->nnodes;
        const int nh = p->D * (p->D + 1) / 2;
        // outputs bound for the host: S, dS, d2S (before the fix-up when
        // early: it then writes its nodes into the host buffers directly),
        // or everything after the fix-up
        auto copy_fields = [&]() -> cudaError_t {
            const HostCopy &h = hc[i];
            cudaError_t e = cudaSuccess;
            if (h.S && e == cudaSuccess) e = cudaMemcpyAsync(h.S, at(S, i), esz * nn, cudaMemcpyDeviceToHost, p->stream);
            if (h.dS && e == cudaSuccess)
                e = cudaMemcpyAsync(h.dS, at(dS, i), esz * nn * p->D, cudaMemcpyDeviceToHost, p->stream);
            if (h.d2S && e == cudaSuccess)
                e = cudaMemcpyAsync(h.d2S, at(d2S, i), esz * nn * nh, cudaMemcpyDeviceToHost, p->stream);
            return e;
        };
        if (hc && hc[i].early) {
            MCK(copy_fields());
            fS = hc[i].mS;
            fdS = hc[i].mdS;
            fd2 = hc[i].md2;
        }
        if (p->prec == SDF_FP32) MCK(launch_fixup(p, ww, fS, fdS, fd2, sfix, fl));
        if (at(flags, i)) MCK(launch_source_flags(p, at(flags, i)));
        MCK(debug_scan_outputs(p, at(S, i), at(dS, i), at(d2S, i)));
        if (hc) {
            if (!hc[i].early) MCK(copy_fields());
            if (hc[i].sign) MCK(cudaMemcpyAsync(hc[i].sign, at(sign, i), nn, cudaMemcpyDeviceToHost, p->stream));
            if (hc[i].flags) MCK(cudaMemcpyAsync(hc[i].flags, at(flags, i), nn, cudaMemcpyDeviceToHost, p->stream));
        }
        MCK(cudaEventRecord(ev[n + i], p->stream));
    }
    // join: p0's next x-pass must not overwrite what the others still read
    for (int i = 1; i < n; ++i) MCK(cudaStreamWaitEvent(st0, ev[n + i], 0));
#undef MCK
    cleanup();
    return SDF_OK;
}

// Device address of a pinned, mapped host buffer (kernels can store there
// directly over the CPU-GPU link), else nullptr.
static void *mapped_host(void *ptr) {
    if (!ptr) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (a.type == cudaMemoryTypeHost && a.devicePointer) ? a.devicePointer : nullptr;
}

sdf_status sdf_execute_host(sdf_plan p, int64_t K, const double *points, const double *weights, void *S, void *dS,
                            void *d2S, int8_t *sign, uint8_t *flags) {
    sdf_status s = check_execute_args(p, K, points, weights, dS, d2S, sign);
    if (s != SDF_OK) return s;
    const int D = p->D;
    const size_t esz = (p->prec == SDF_FP64) ? sizeof(double) : sizeof(float);
    const int64_t nn = p->nnodes;
    const int nh = D * (D + 1) / 2;
    // S and its derivatives go straight to pinned host buffers (the kernels
    // write them over the link while the rest computes); other outputs and
    // unpinned buffers go through device staging and a copy at the end
    void *mS = mapped_host(S), *mdS = mapped_host(dS), *md2 = mapped_host(d2S);
    size_t need = sizeof(double) * K * D * (weights ? 2 : 1);
    size_t oS = need, odS = oS + ((S && !mS) ? esz * nn : 0), od2 = odS + ((dS && !mdS) ? esz * nn * D : 0),
           osg = od2 + ((d2S && !md2) ? esz * nn * nh : 0), ofl = osg + (sign ? nn : 0), tot = ofl + (flags ? nn : 0);
    if (tot > p->staging_bytes) {
        cudaStreamSynchronize(p->stream);
        cudaFree(p->staging);
        p->staging = nullptr;
        p->staging_bytes = 0;
        CK(dev_alloc((void **)&p->staging, tot));
        p->staging_bytes = tot;
    }
    char *base = reinterpret_cast<char *>(p->staging);
    double *dpts = reinterpret_cast<double *>(base);
    double *dw = weights ? dpts + K * D : nullptr;
    CK(cudaMemcpyAsync(dpts, points, sizeof(double) * K * D, cudaMemcpyHostToDevice, p->stream));
    if (weights) CK(cudaMemcpyAsync(dw, weights, sizeof(double) * K * D, cudaMemcpyHostToDevice, p->stream));
    void *dS_ = S ? (mS ? mS : base + oS) : nullptr;
    void *ddS = dS ? (mdS ? mdS : base + odS) : nullptr;
    void *dd2 = d2S ? (md2 ? md2 : base + od2) : nullptr;
    int8_t *dsg = sign ? reinterpret_cast<int8_t *>(base + osg) : nullptr;
    uint8_t *dfl = flags ? reinterpret_cast<uint8_t *>(base + ofl) : nullptr;
    s = sdf_execute(p, K, dpts, dw, dS_, ddS, dd2, dsg, dfl);
    if (s != SDF_OK) return s;
    if (S && !mS) CK(cudaMemcpyAsync(S, dS_, esz * nn, cudaMemcpyDeviceToHost, p->stream));
    if (dS && !mdS) CK(cudaMemcpyAsync(dS, ddS, esz * nn * D, cudaMemcpyDeviceToHost, p->stream));
    if (d2S && !md2) CK(cudaMemcpyAsync(d2S, dd2, esz * nn * nh, cudaMemcpyDeviceToHost, p->stream));
    if (sign) CK(cudaMemcpyAsync(sign, dsg, nn, cudaMemcpyDeviceToHost, p->stream));
    if (flags) CK(cudaMemcpyAsync(flags, dfl, nn, cudaMemcpyDeviceToHost, p->stream));
    return sdf_sync(p);
}

sdf_status sdf_execute_multi_host(int n, const sdf_plan *plans, int64_t K, const double *points,
                                  const double *weights, void *const *S, void *const *dS, void *const *d2S,
                                  int8_t *const *sign, uint8_t *const *flags) {
    ScopedRange range_("sdf_execute_multi_host");
    if (n < 1 || !plans || !points || K < 1) return SDF_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (!plans[i]) return SDF_ERR_INVALID_ARG;
    auto at = [](auto *const *arr, int i) { return arr ? arr[i] : nullptr; };
    sdf_plan p0 = plans[0];
    const int D = p0->D;
    const int nh = D * (D + 1) / 2;
    // every output is computed into the plan's staging buffer and copied
    // by the copy engine; plans[0]'s S, dS and d2S go as soon as its
    // epilogue has written them, beside the other plans' work, and its
    // fix-up then stores its nodes straight into the host buffers (which
    // needs them pinned, device-mapped).  With several plans this kept the
    // CPU-GPU link busiest: on two 2048^2 plans 2.19 ms per call, against
    // 2.44 ms with every output stored by the kernels into host memory and
    // 2.78 ms with every copy after the fix-ups
    std::vector<void *> dev_S(n), dev_dS(n), dev_d2(n);
    std::vector<int8_t *> dev_sg(n);
    std::vector<uint8_t *> dev_fl(n);
    std::vector<HostCopy> hc(n);
    double *dpts = nullptr, *dw = nullptr;
    for (int i = 0; i < n; ++i) {
        sdf_plan p = plans[i];
        const size_t esz = (p->prec == SDF_FP64) ? sizeof(double) : sizeof(float);
        const int64_t nn = p->nnodes;
        const int nd = (p->D == 1) ? 1 : p->D, nhh = (p->D == 1) ? 1 : nh;
        const size_t need = (i == 0) ? sizeof(double) * K * D * (weights ? 2 : 1) : 0;
        const size_t oS = need, odS = oS + (at(S, i) ? esz * nn : 0), od2 = odS + (at(dS, i) ? esz * nn * nd : 0),
                     osg = od2 + (at(d2S, i) ? esz * nn * nhh : 0), ofl = osg + (at(sign, i) ? nn : 0),
                     tot = ofl + (at(flags, i) ? nn : 0);
        if (tot > p->staging_bytes) {
            cudaStreamSynchronize(p->stream);
            cudaFree(p->staging);
            p->staging = nullptr;
            p->staging_bytes = 0;
            CK(dev_alloc((void **)&p->staging, tot));
            p->staging_bytes = tot;
        }
        char *base = reinterpret_cast<char *>(p->staging);
        if (i == 0) {
            dpts = reinterpret_cast<double *>(base);
            dw = weights ? dpts + K * D : nullptr;
        }
        dev_S[i] = at(S, i) ? base + oS : nullptr;
        dev_dS[i] = at(dS, i) ? base + odS : nullptr;
        dev_d2[i] = at(d2S, i) ? base + od2 : nullptr;
        dev_sg[i] = at(sign, i) ? reinterpret_cast<int8_t *>(base + osg) : nullptr;
        dev_fl[i] = at(flags, i) ? reinterpret_cast<uint8_t *>(base + ofl) : nullptr;
        HostCopy &h = hc[i];
        h.S = at(S, i);
        h.dS = at(dS, i);
        h.d2S = at(d2S, i);
        h.sign = at(sign, i);
        h.flags = at(flags, i);
        h.mS = mapped_host(h.S);
        h.mdS = mapped_host(h.dS);
        h.md2 = mapped_host(h.d2S);
        h.early = i == 0 && n > 1 && p->D >= 2 && p->prec == SDF_FP32 && (!h.S || h.mS) && (!h.dS || h.mdS) &&
                  (!h.d2S || h.md2);
    }
    CK(cudaMemcpyAsync(dpts, points, sizeof(double) * K * D, cudaMemcpyHostToDevice, p0->stream));
    if (weights) CK(cudaMemcpyAsync(dw, weights, sizeof(double) * K * D, cudaMemcpyHostToDevice, p0->stream));
    sdf_status s = multi_core(n, plans, K, dpts, dw, dev_S.data(), dev_dS.data(), dev_d2.data(), dev_sg.data(),
                              dev_fl.data(), hc.data());
    if (s != SDF_OK) {
        for (int i = 0; i < n; ++i) cudaStreamSynchronize(plans[i]->stream);
        return s;
    }
    sdf_status first = SDF_OK;
    for (int i = 0; i < n; ++i) {
        const sdf_status si = sdf_sync(plans[i]);
        if (first == SDF_OK) first = si;
    }
    return first;
}

sdf_status sdf_sync(sdf_plan p) {
    if (!p) return SDF_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(p->stream));
    CK(cudaMemcpy(p->hsc, p->dsc, sizeof(DevScalars), cudaMemcpyDeviceToHost));
    const int st = p->hsc->status;
    if (st == SDF_ERR_INTERNAL) {
        char msg[160];
        snprintf(msg, sizeof msg, "sdf_sync: device consistency check %d failed at index %lld", p->hsc->dbg_check,
                 (long long)p->hsc->dbg_where);
        set_last_error(msg);
    }
    if (st != 0) CK(cudaMemset(p->dsc, 0, sizeof(int)));
    return (sdf_status)st;
}

sdf_status sdf_plan_get_info(sdf_plan p, sdf_plan_info *info) {
    if (!p || !info) return SDF_ERR_INVALID_ARG;
    memset(info, 0, sizeof(*info));
    info->D = p->D;
    info->precision = p->prec;
    info->outputs = p->outputs;
    for (int a = 0; a < 3; ++a) {
        info->dims[a] = p->N[a];
        info->padded[a] = p->M[a];
    }
    info->h = p->h;
    info->tau = p->tau;
    info->n_kernels = (int)p->kernels.size();
    for (size_t i = 0; i < p->kernels.size() && i < 16; ++i) info->kernel_l1[i] = p->kernels[i].l1;
    info->noise_const_fp32 = p->noise_c32;
    info->noise_const_fp64 = p->noise_c64;
    info->plan_ms = p->plan_ms;
    info->workspace_bytes = p->workspace_bytes;
    return SDF_OK;
}

// A-priori bounds on the error of the last execute over the nodes not
// flagged CAPPED, against the exact S (eq. STilde via eq. Bound1), grad S and
// Hessian of the snapped points, from three sources:
//  * Transform noise.  Under the error model behind the trust threshold
//    (include/sdf.h, "Trust region"), the computed phi_p of precision p errs by
//    at most F = C_p u_p sqrt(log2 n) ||g||_2/sqrt(n) times the channel's l1
//    norm, and theta_p = F_phi Q/(eps f) (eps = kTrustEps, f the phi channel's
//    norm).  A node the transform keeps has phi_p >= theta_p, so the relative
//    error of phi there is at most d = (eps f/Q)/(1 - eps f/Q): S = -tau log phi
//    errs by tau d; grad S = num/phi by (F_grad + F_phi)/phi, i.e.
//    eps (f + g)/Q/(1 - ...) since |grad S| <= 1; the Hessian, in units of
//    1/tau, by eps (tau h + 2 g + 2 f)/Q (g, h: the gradient and Hessian
//    channels' norms) -- the same combination Q weighs.
//  * The fix-up's direct sum (SDF_FP32 plans), relative error of the sum:
//    the tail left out when a node stops (below 1e-5 of its sum by the stop
//    test; in 3D plus 1e-6 per ring batch for the bins a warp skips), each
//    term's error (1/r and 2^x by rsqrt.approx / ex2.approx, both within
//    2^-21 relative; the exponent's absolute error is (r/tau) log2(e) times
//    that, and the terms that matter have r/tau log2(e) <= L + 64 with
//    L = log2(e) R_max/tau, R_max the largest distance to the nearest point
//    of an uncapped node: S_cap + tau log K, or the grid diagonal in full-range
//    mode), and float summation of at most n_max positive terms (n_max u).
//    S errs by tau times that relative error, grad S by twice it, and the
//    Hessian -- a weighted mean of (delta - n n)/r - n n/tau, each term at
//    most 1/r_min + 1/tau, plus g g/tau -- by (2 tau/r_min + 6) times it in
//    units of 1/tau, with r_min >= h the smallest distance from a written
//    node to its nearest point (recorded by the fix-up kernel).
//  * Rounding of the outputs (float: 2^-24 relative to S <= R_max).
// The noise part rests on the calibrated constants C_p: a bound under the
// model, as the trust region itself is.
static void error_bounds(const sdf_plan_impl *p, const DevScalars &d, sdf_exec_stats *st) {
    const double eps = kTrustEps, tau = p->tau, h = p->h;
    const double Q = p->q_factor > 0 ? p->q_factor : 1.0;
    const double f = p->q_f, g = p->q_g, hh = p->q_h;
    const double den = 1.0 - eps * f / Q;
    const double dS_rel = eps * f / Q / den;
    const double dG = eps * (f + g) / Q / den;
    const double dH_tau = eps * (tau * hh + 2 * g + 2 * f) / Q / den;
    const double logK = log((double)std::max<int64_t>(1, p->last_K));
    double diag = 0;
    for (int a = 0; a < p->D; ++a) diag += (double)p->N[a] * (double)p->N[a];
    diag = h * sqrt(diag);
    const double rmax = (p->prec == SDF_FP32 && p->full_range) ? diag : std::min(diag, st->s_cap + tau * logK);
    const double u = (p->prec == SDF_FP64) ? ldexp(1.0, -53) : ldexp(1.0, -24);
    const bool ds = p->outputs & SDF_OUT_DS, d2 = p->outputs & SDF_OUT_D2S;
    // transform part (the FP64 path, and the nodes an FP32 plan keeps)
    double bS = tau * dS_rel + 2 * u * rmax;
    double bG = ds ? dG + 2 * u : 0.0;
    double bH = d2 ? (dH_tau + 4 * u * (tau / h + 2)) / tau : 0.0;
    if (p->prec == SDF_FP32 && (d.n_fixup_nodes > 0 || p->D == 1)) {
        const double L = 1.4426950408889634 * rmax / tau;
        const double e_term = log(2.0) * (L + 64.0 + 1.0) * ldexp(1.0, -21) + ldexp(1.0, -23);
        const double e_sum = (double)(d.fix_nmax + d.fix_rounds + 1) * ldexp(1.0, -24);
        const double e_tail = 1e-5 + (p->D == 3 ? 1e-6 * (double)d.fix_rounds : 0.0);
        const double e = e_term + e_sum + e_tail;
        bS = std::max(bS, tau * e + 2 * u * rmax);
        if (ds) bG = std::max(bG, 2 * e + 2 * u);
        float rinv_f;  // the largest h/r_min over written nodes (at most 1)
        memcpy(&rinv_f, &d.fix_rinv_bits, sizeof rinv_f);
        const double rinv = std::min(1.0, (double)rinv_f);
        if (d2) bH = std::max(bH, ((2 * tau * rinv / h + 6) * e + 4 * u * (tau / h + 2)) / tau);
    }
    st->err_bound_S = bS;
    st->err_bound_dS = bG;
    st->err_bound_d2S = bH;
}

sdf_status sdf_get_stats(sdf_plan p, sdf_exec_stats *st) {
    if (!p || !st) return SDF_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(p->stream));
    CK(cudaMemcpy(p->hsc, p->dsc, sizeof(DevScalars), cudaMemcpyDeviceToHost));
    const DevScalars &d = *p->hsc;
    const int D = p->D;
    const double n = (double)p->M[0] * (double)p->M[1] * (D == 3 ? (double)p->M[2] : 1.0);
    const double base = sqrt(log2(n)) / sqrt(n) * p->q_factor / kTrustEps;
    const double gn = sqrt((double)d.sum_c2);
    memset(st, 0, sizeof(*st));
    st->g_norm2 = gn;
    st->theta64 = p->noise_c64 * ldexp(1.0, -53) * base * gn;
    st->theta32 = p->noise_c32 * ldexp(1.0, -24) * base * gn;
    st->s_cap = -p->tau * log(st->theta64);
    st->n_unique = d.n_unique;
    st->n_fixup_tiles = (int64_t)d.n_fixup_tiles;
    st->n_fixup_nodes = (int64_t)d.n_fixup_nodes;
    st->n_capped = (int64_t)d.n_capped;
    st->n_launches = p->nlaunch;
    st->n_fixup_terms = (int64_t)d.n_fixup_terms;
    st->trusted_frac = 1.0 - (double)(int64_t)d.n_capped / (double)p->nnodes;
    error_bounds(p, d, st);
    return SDF_OK;
}

sdf_status sdf_plan_set_noise_constants(sdf_plan p, double c32, double c64) {
    if (!p) return SDF_ERR_INVALID_ARG;
    if (c32 > 0) p->noise_c32 = c32;
    if (c64 > 0) p->noise_c64 = c64;
    return SDF_OK;
}

sdf_status sdf_plan_set_tuning(sdf_plan p, int lines_T, int lines_F, int fused_variant) {
    if (!p) return SDF_ERR_INVALID_ARG;
    p->tune_RT = lines_T > 0 ? lines_T : 0;
    p->tune_RF = lines_F > 0 ? lines_F : 0;
    p->tune_FV = (fused_variant >= 1 && fused_variant <= 3) ? fused_variant : 0;
    return SDF_OK;
}

sdf_status sdf_debug_hook(int hook, int64_t value) {
    if (value < 0) return SDF_ERR_INVALID_ARG;
    switch (hook) {
        case SDF_HOOK_FAIL_ALLOC: g_fail_alloc.store(value); return SDF_OK;
        case SDF_HOOK_TMA_WAIT_POLLS: g_tma_polls.store(value); return SDF_OK;
        case SDF_HOOK_CORRUPT_BINS: set_corrupt_bins(value); return SDF_OK;
        default: return SDF_ERR_INVALID_ARG;
    }
}

sdf_status sdf_set_debug_checks(int on) {
    set_debug_checks(on != 0);
    return SDF_OK;
}

int sdf_get_debug_checks(void) { return debug_checks() ? 1 : 0; }

sdf_status sdf_plan_set_epilogue_loads(sdf_plan p, int mode) {
    if (!p || (mode != 0 && mode != 1)) return SDF_ERR_INVALID_ARG;
    p->tune_EV = mode;
    return SDF_OK;
}

sdf_status sdf_plan_set_full_range(sdf_plan p, int enable) {
    if (!p) return SDF_ERR_INVALID_ARG;
    if (p->prec != SDF_FP32) {
        set_last_error("sdf_plan_set_full_range: SDF_FP32 plans only (the fix-up supplies the range)");
        return SDF_ERR_UNSUPPORTED;
    }
    p->full_range = enable != 0;
    return SDF_OK;
}

sdf_status sdf_plan_set_padding(sdf_plan p, const int64_t *padded) {
    if (!p || !padded) return SDF_ERR_INVALID_ARG;
    if (p->D == 1) {
        set_last_error("sdf_plan_set_padding: 1D plans keep their power-of-two line");
        return SDF_ERR_UNSUPPORTED;
    }
    if (p->shares_spectra) {
        set_last_error("sdf_plan_set_padding: the plan uses spectra owned by another plan of its batch");
        return SDF_ERR_UNSUPPORTED;
    }
    if (!padding_ok(p, padded)) {
        set_last_error("sdf_plan_set_padding: each M_a must be 2^k or 3*2^k (>= 48), >= max(2 N_a - 1, 16), "
                       "and within the transform limit");
        return SDF_ERR_INVALID_ARG;
    }
    bool same = true;
    for (int a = 0; a < p->D; ++a) same = same && padded[a] == p->M[a];
    if (same) return SDF_OK;
    return plan_repad(p, padded, nullptr);
}

sdf_status sdf_plan_set_kernel(sdf_plan p, int kernel_set) {
    if (!p || (kernel_set != SDF_KERNEL_EXP && kernel_set != SDF_KERNEL_GREEN)) return SDF_ERR_INVALID_ARG;
    if (kernel_set == p->kernel_set) return SDF_OK;
    if (kernel_set == SDF_KERNEL_GREEN && p->prec != SDF_FP64) {
        set_last_error("sdf_plan_set_kernel: the Green's function set needs an SDF_FP64 plan");
        return SDF_ERR_UNSUPPORTED;
    }
    if (p->shares_spectra) {
        set_last_error("sdf_plan_set_kernel: the plan uses spectra owned by another plan of its batch");
        return SDF_ERR_UNSUPPORTED;
    }
    CK(cudaStreamSynchronize(p->stream));
    // drop every spectrum (forward and adjoint) and the adjoint programme
    for (auto &k : p->kernels) {
        cudaFree(k.c);
        const int64_t esz = (p->prec == SDF_FP64) ? 8 : 4;
        p->workspace_bytes -= esz * spec_rows(p) * spec_row_len(p);
    }
    p->kernels.clear();
    for (int i = 0; i < KER_COUNT; ++i) p->kslot[i] = -1;
    if (p->adj_ngroup > 0) {
        const size_t esz = (p->prec == SDF_FP64) ? sizeof(double) : sizeof(float);
        cudaFree(p->adj_planes);
        cudaFree(p->adj_part);
        p->adj_planes = nullptr;
        p->adj_part = nullptr;
        p->workspace_bytes -= esz * (p->D + 1) * p->nnodes + sizeof(double) * 2 * kAdjParts;
        p->adj_ngroup = 0;
    }
    p->kernel_set = kernel_set;
    CK(build_kernel_list(p, plan_kernel_ids(p)));
    plan_programme(p);
    return SDF_OK;
}

sdf_status sdf_green_profile(int D, int64_t n, const double *z, double *g, double *g1, double *g2) {
    if (D < 1 || D > 3 || n < 0 || (n > 0 && (!z || !g || !g1 || !g2))) return SDF_ERR_INVALID_ARG;
    for (int64_t i = 0; i < n; ++i) {
        if (!(z[i] >= 0.0) || !std::isfinite(z[i])) return SDF_ERR_INVALID_ARG;
        if (z[i] == 0.0) {
            g[i] = green_origin_integral(D);
            g1[i] = g2[i] = 0.0;
        } else {
            green_profile(D, z[i], &g[i], &g1[i], &g2[i]);
        }
    }
    return SDF_OK;
}

// Device time of the named kernels (every kernel when nnames = 0) over `reps`
// executes (after one warm-up).
static sdf_status time_kernels(sdf_plan p, int64_t K, const double *points, const double *weights, int reps,
                               const char *const *names, int nnames, double *ms) {
    sdf_status s = sdf_execute(p, K, points, weights, nullptr, nullptr, nullptr, nullptr, nullptr);
    if (s != SDF_OK) return s;
    const bool was = p->prof_on;
    p->prof_on = true;
    sdf_kernel_time kt[32];
    sdf_profile_read(p, kt, 32);  // drop older records
    for (int r = 0; r < reps; ++r) {
        s = sdf_execute(p, K, points, weights, nullptr, nullptr, nullptr, nullptr, nullptr);
        if (s != SDF_OK) break;
    }
    const int n = sdf_profile_read(p, kt, 32);
    p->prof_on = was;
    if (s != SDF_OK) return s;
    if (n < 0) return SDF_ERR_CUDA;
    *ms = 0;
    for (int i = 0; i < n; ++i) {
        if (nnames == 0) *ms += kt[i].total_ms;
        for (int j = 0; j < nnames; ++j)
            if (strcmp(kt[i].name, names[j]) == 0) *ms += kt[i].total_ms;
    }
    return SDF_OK;
}

// ---- the autotuner's cache: one line per tuned problem,
// "<key>\t<M0> <M1> <M2> <lines_T> <lines_F> <fused_variant> <epilogue_loads>", the last line
// of a key wins.  Path: $SDF_AUTOTUNE_CACHE (empty: no cache), else
// $XDG_CACHE_HOME/sdf_gb300/autotune.tsv, else $HOME/.cache/sdf_gb300/autotune.tsv.
static std::mutex g_tune_mutex;

static std::string tune_cache_path() {
    const char *e = getenv("SDF_AUTOTUNE_CACHE");
    if (e) return std::string(e);
    std::string base;
    const char *x = getenv("XDG_CACHE_HOME");
    if (x && *x) {
        base = x;
    } else {
        const char *h = getenv("HOME");
        if (!h || !*h) return std::string();
        base = std::string(h) + "/.cache";
    }
    return base + "/sdf_gb300/autotune.tsv";
}

// GPU name and architecture, D, node counts, precision, outputs, kernel set.
static std::string tune_key(const sdf_plan_impl *p) {
    int dev = 0;
    cudaDeviceProp prop;
    std::string gpu = "unknown";
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
        gpu = prop.name;
        gpu += " sm_" + std::to_string(prop.major) + std::to_string(prop.minor);
    }
    cudaGetLastError();
    for (auto &c : gpu)
        if (c == '\t' || c == '\n' || c == '|') c = ' ';
    char buf[256];
    snprintf(buf, sizeof buf, "|D%d|%lldx%lldx%lld|%s|out%u|kernel%d", p->D, (long long)p->N[0], (long long)p->N[1],
             (long long)p->N[2], p->prec == SDF_FP64 ? "fp64" : "fp32", p->outputs, p->kernel_set);
    return gpu + buf;
}

struct TuneRec {
    int64_t M[3];
    int RT, RF, FV, EV;
};

static bool tune_lookup(const std::string &key, TuneRec *out) {
    const std::string path = tune_cache_path();
    if (path.empty()) return false;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    FILE *f = fopen(path.c_str(), "r");
    if (!f) return false;
    bool found = false;
    char line[1024];
    while (fgets(line, sizeof line, f)) {
        char *tab = strchr(line, '\t');
        if (!tab) continue;
        *tab = 0;
        if (key != line) continue;
        long long m0, m1, m2;
        int rt, rf, fv, ev = 0;
        if (sscanf(tab + 1, "%lld %lld %lld %d %d %d %d", &m0, &m1, &m2, &rt, &rf, &fv, &ev) >= 6) {
            out->M[0] = m0;
            out->M[1] = m1;
            out->M[2] = m2;
            out->RT = rt;
            out->RF = rf;
            out->FV = fv;
            out->EV = ev;
            found = true;
        }
    }
    fclose(f);
    return found;
}

static void tune_store(const std::string &key, const TuneRec &r) {
    const std::string path = tune_cache_path();
    if (path.empty()) return;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    // create the directories on the way (ignore failures: the cache is optional)
    for (size_t i = 1; i < path.size(); ++i)
        if (path[i] == '/') mkdir(path.substr(0, i).c_str(), 0755);
    FILE *f = fopen(path.c_str(), "a");
    if (!f) return;
    fprintf(f, "%s\t%lld %lld %lld %d %d %d %d\n", key.c_str(), (long long)r.M[0], (long long)r.M[1],
            (long long)r.M[2], r.RT, r.RF, r.FV, r.EV);
    fclose(f);
}

sdf_status sdf_plan_autotune(sdf_plan p, int64_t K, const double *points, const double *weights, int reps,
                             int *lines_T, int *lines_F, int *fused_variant) {
    if (!p || !points || reps < 1) return SDF_ERR_INVALID_ARG;
    if (p->D == 1) {
        set_last_error("sdf_plan_autotune: a 1D plan has no tile schedule");
        return SDF_ERR_UNSUPPORTED;
    }
    auto report = [&]() {
        if (lines_T) *lines_T = p->tune_RT;
        if (lines_F) *lines_F = p->tune_RF;
        if (fused_variant) *fused_variant = p->tune_FV;
    };
    const std::string key = tune_key(p);
    TuneRec rec;
    if (tune_lookup(key, &rec)) {
        bool sameM = true;
        for (int a = 0; a < p->D; ++a) sameM = sameM && rec.M[a] == p->M[a];
        if (!sameM && !p->shares_spectra && padding_ok(p, rec.M)) {
            sdf_status s = plan_repad(p, rec.M, nullptr);
            if (s != SDF_OK) return s;
        }
        p->tune_RT = rec.RT;
        p->tune_RF = rec.RF;
        p->tune_FV = rec.FV;
        p->tune_EV = rec.EV;
        report();
        return SDF_OK;
    }
    // 1. padded sizes: per axis the power of two, or 3 * 2^k where that is
    // smaller; every combination timed over the whole execute (default tile
    // schedule).  A plan of a batch that borrows its spectra keeps its sizes.
    p->tune_RT = p->tune_RF = p->tune_FV = p->tune_EV = 0;
    if (!p->shares_spectra) {
        std::vector<std::vector<int64_t>> opts(p->D);
        size_t ncomb = 1;
        for (int a = 0; a < p->D; ++a) {
            const int64_t need = std::max<int64_t>(16, 2 * p->N[a] - 1);
            opts[a].push_back(std::max<int64_t>(16, next_pow2(need)));
            const int64_t r3 = r3_padding(need);
            if (r3 && r3 <= max_padded(p->D)) opts[a].push_back(r3);
            ncomb *= opts[a].size();
        }
        if (ncomb > 1) {
            double best = 1e300;
            int64_t bestM[3] = {p->M[0], p->M[1], p->M[2]};
            for (size_t c = 0; c < ncomb; ++c) {
                int64_t M[3] = {1, 1, 1};
                size_t r = c;
                for (int a = 0; a < p->D; ++a) {
                    M[a] = opts[a][r % opts[a].size()];
                    r /= opts[a].size();
                }
                sdf_status s = sdf_plan_set_padding(p, M);
                if (s != SDF_OK) return s;
                double ms;
                s = time_kernels(p, K, points, weights, reps, nullptr, 0, &ms);
                if (s != SDF_OK) return s;
                if (ms < best) {
                    best = ms;
                    for (int a = 0; a < 3; ++a) bestM[a] = M[a];
                }
            }
            sdf_status s = sdf_plan_set_padding(p, bestM);
            if (s != SDF_OK) return s;
        }
    }
    // 2. the tile schedule on those sizes
    const char *tnames[] = {"xpass", "fwd_y", "inv_y", "epilogue"};
    const char *fnames[] = {"fused"};
    double best = 1e300;
    int bestT = 0, bestF = 0, bestV = 0, bestE = 0;
    for (int EV : {0, 1}) {
        for (int RT : {0, 1, 2, 4, 8, 16}) {
            p->tune_RT = RT;
            p->tune_EV = EV;
            double ms;
            sdf_status s = time_kernels(p, K, points, weights, reps, tnames, 4, &ms);
            if (s != SDF_OK) return s;
            if (ms < best) {
                best = ms;
                bestT = RT;
                bestE = EV;
            }
        }
    }
    p->tune_RT = bestT;
    p->tune_EV = bestE;
    best = 1e300;
    for (int RF : {0, 1, 2, 4}) {
        for (int FV : {1, 2, 3}) {
            p->tune_RF = RF;
            p->tune_FV = FV;
            double ms;
            sdf_status s = time_kernels(p, K, points, weights, reps, fnames, 1, &ms);
            if (s != SDF_OK) return s;
            if (ms < best) {
                best = ms;
                bestF = RF;
                bestV = FV;
            }
        }
    }
    p->tune_RF = bestF;
    p->tune_FV = bestV;
    for (int a = 0; a < 3; ++a) rec.M[a] = p->M[a];
    rec.RT = bestT;
    rec.RF = bestF;
    rec.FV = bestV;
    rec.EV = bestE;
    tune_store(key, rec);
    report();
    return SDF_OK;
}

sdf_status sdf_profile_enable(sdf_plan p, int enable) {
    if (!p) return SDF_ERR_INVALID_ARG;
    p->prof_on = enable != 0;
    return SDF_OK;
}

int sdf_profile_read(sdf_plan p, sdf_kernel_time *out, int max) {
    if (!p || (max > 0 && !out)) return -1;
    if (cudaStreamSynchronize(p->stream) != cudaSuccess) return -1;
    std::vector<sdf_kernel_time> agg;
    for (auto &r : p->prof_recs) {
        float ms = 0.f;
        if (r.a && r.b) cudaEventElapsedTime(&ms, r.a, r.b);
        size_t i = 0;
        for (; i < agg.size(); ++i)
            if (strncmp(agg[i].name, r.name, sizeof(agg[i].name)) == 0) break;
        if (i == agg.size()) {
            sdf_kernel_time k;
            memset(&k, 0, sizeof k);
            snprintf(k.name, sizeof k.name, "%s", r.name);
            agg.push_back(k);
        }
        agg[i].launches += 1;
        agg[i].total_ms += ms;
        if (r.a) p->prof_pool.push_back(r.a);
        if (r.b) p->prof_pool.push_back(r.b);
    }
    p->prof_recs.clear();
    int n = 0;
    for (; n < (int)agg.size() && n < max; ++n) out[n] = agg[n];
    return n;
}

void sdf_plan_destroy(sdf_plan p) {
    if (!p) return;
    free_plan(p);
    delete p;
}

sdf_status sdf_backward(sdf_plan p, int64_t K, const double *points, const void *w, const void *S_saved,
                        const uint8_t *flags, double *dL_dY, double *dL_dtau) {
    if (!p || !points || !w || !S_saved || !dL_dY || !dL_dtau) return SDF_ERR_INVALID_ARG;
    if (p->kernel_set != SDF_KERNEL_EXP) {
        set_last_error("sdf_backward: the adjoint is derived for the exp(-r/tau) kernel set only");
        return SDF_ERR_UNSUPPORTED;
    }
    if (p->D == 1) {
        set_last_error("sdf_backward: 2D and 3D plans only");
        return SDF_ERR_UNSUPPORTED;
    }
    if (!(p->outputs & SDF_OUT_DS)) return SDF_ERR_INVALID_ARG;
    if (K < 1 || K >= (int64_t(1) << 31) - 1) return SDF_ERR_INVALID_ARG;
    CK(ensure_points(p, K));
    p->last_K = K;
    p->nlaunch = 0;
    CK(launch_adjoint(p, K, points, w, S_saved, flags, dL_dY, dL_dtau));
    return SDF_OK;
}

}  // extern "C"
