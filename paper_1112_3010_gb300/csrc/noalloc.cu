// noalloc.cu -- sdf_execute_noalloc: the whole path for one small problem
// without any device allocation.
//
// Some callers cannot call cudaMalloc: a process whose device memory is
// owned by another allocator (a framework's caching pool that must see every
// byte), a plugin whose host application forbids device allocation after
// start-up, or a service that must stay inside a memory budget fixed in
// advance.  For them every scratch buffer of this entry point -- kernel
// spectra, transform buffers, point bins, flags and device status -- is
// carved out of one file-scope static __device__ array of kScratchBytes.
// Every GPU that loads the library holds that array until the process exits.
//
// In host code the array's name is only a host-side stand-in for the device
// symbol, so the set-up below asks the runtime for its device address
// (cudaGetSymbolAddress) once per device, with that device current, and
// passes the address on.  The first call on each device does this set-up.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <cmath>
#include <memory>
#include <mutex>
#include <vector>

#include "sdf_internal.cuh"

namespace sdf {
cudaError_t launch_points(sdf_plan_impl *p, int64_t K, const double *points, const double *weights);
}

using namespace sdf;

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;  // 32 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mutex;                      // serialises calls from this process
unsigned char *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device (set-up on first use).
cudaError_t scratch_address(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = reinterpret_cast<unsigned char *>(ptr);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// Bump allocator over the static array (256-byte aligned pieces).
struct Carver {
    unsigned char *base;
    size_t off = 0;
    template <typename P> void take(P **ptr, size_t bytes) {
        off = (off + 255) & ~size_t(255);
        *ptr = reinterpret_cast<P *>(base ? base + off : nullptr);
        off += bytes;
    }
};

// The twiddle table goes to the scratch with a copy ordered on the caller's
// stream (not the legacy default stream, which would serialise with every
// other stream of the device).  The source is pageable: the copy has been
// staged by the time cudaMemcpyAsync returns, so h may go out of scope.
template <typename T>
cudaError_t fill_twiddles(void *dst, int64_t L, cudaStream_t st) {
    using V = typename cplx_t<T>::type;
    std::vector<V> h(L);
    fill_twiddle_table(line_code(L), h.data());
    return cudaMemcpyAsync(dst, h.data(), sizeof(V) * L, cudaMemcpyHostToDevice, st);
}

// Lay out every buffer of plan p in the scratch; returns the bytes needed.
size_t layout(sdf_plan_impl *p, int64_t K, unsigned char *base, double2 **tw64, double **part, double2 **bufX,
              double2 **bufY) {
    Carver c{base};
    const int D = p->D;
    const size_t vb = (p->prec == SDF_FP64) ? sizeof(double2) : sizeof(float2);
    const size_t esz = (p->prec == SDF_FP64) ? sizeof(double) : sizeof(float);
    c.take(&p->dsc, sizeof(DevScalars));
    for (int a = 0; a < D; ++a) {
        c.take(&p->tw[a], vb * p->M[a]);
        c.take(&tw64[a], sizeof(double2) * p->M[a]);
    }
    c.take(part, sizeof(double) * kSpectraParts);
    const int64_t H = spec_rows(p) * spec_row_len(p);
    for (auto &k : p->kernels) c.take(&k.c, esz * H);
    const int64_t nb = p->nbins;
    c.take(&p->bin_count, sizeof(int) * (nb + 1));
    c.take(&p->bin_start, sizeof(int) * (nb + 1));
    c.take(&p->bin_fill, sizeof(int) * nb);
    c.take(&p->bin_nuniq, sizeof(int) * nb);
    c.take(&p->cheb, 2 * nb);
    c.take(&p->tile_flag, nb);
    if (p->prec == SDF_FP32) {
        c.take(&p->flags_int, p->nnodes);
        c.take(&p->sign_int, p->nnodes);
        c.take(&p->occ_start, sizeof(int) * (bin_rows(p) + 1));
        c.take(&p->occ_x, sizeof(int) * nb);
        c.take(&p->occ_tmp, sizeof(int) * occ_tmp_len(p));
    }
    c.take(&p->pt_key, sizeof(int) * K);
    c.take(&p->pt_lc, sizeof(int) * K);
    c.take(&p->ucell, sizeof(int) * K);
    c.take(&p->ucount, sizeof(int) * K);
    c.take(&p->pt_entry, sizeof(long long) * K);
    c.take(&p->uw, sizeof(double) * 3 * K);
    p->Kcap = K;
    // the plan-time transform buffers and the execute-time ones share one region
    int64_t total = 1;
    for (int a = 0; a < D; ++a) total *= p->M[a];
    const size_t plan_time = 2 * sizeof(double2) * total;
    const size_t run_time = ((p->bytesA + 255) & ~size_t(255)) + p->bytesB;
    unsigned char *region = nullptr;
    c.take(&region, std::max(plan_time, run_time));
    *bufX = reinterpret_cast<double2 *>(region);
    *bufY = region ? reinterpret_cast<double2 *>(region + sizeof(double2) * total) : nullptr;
    p->bufA = region;
    p->bufB = region ? region + ((p->bytesA + 255) & ~size_t(255)) : nullptr;
    return c.off;
}

// An error return: first wait for whatever this call already queued on the
// stream, so that no kernel of a failed call still reads or writes the
// scratch when the lock is released and the next call rewrites it.
sdf_status fail(cudaError_t e, cudaStream_t st) {
    set_last_error(cudaGetErrorString(e));
    cudaStreamSynchronize(st);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? SDF_ERR_OOM : SDF_ERR_CUDA;
}

}  // namespace

#define NCK(x)                                           \
    do {                                                 \
        cudaError_t e_ = (x);                            \
        if (e_ != cudaSuccess) return fail(e_, p->stream); \
    } while (0)

extern "C" sdf_status sdf_execute_noalloc(int D, const int64_t *dims, double h, double tau, int precision,
                                          unsigned outputs, int64_t K, const double *points, const double *weights,
                                          void *S, void *dS, void *d2S, int8_t *sign, uint8_t *flags,
                                          void *stream) {
    if (D != 2 && D != 3) return SDF_ERR_UNSUPPORTED;
    if (!dims || !points || !(h > 0.0) || !(tau > 0.0) || !std::isfinite(h) || !std::isfinite(tau))
        return SDF_ERR_INVALID_ARG;
    if (precision != SDF_FP64 && precision != SDF_FP32) return SDF_ERR_INVALID_ARG;
    if (outputs & ~15u) return SDF_ERR_INVALID_ARG;
    if (K < 1 || K >= (int64_t(1) << 31) - 1) return SDF_ERR_INVALID_ARG;
    for (int a = 0; a < D; ++a)
        if (dims[a] < 2 || dims[a] > 4096) return SDF_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mutex);
    std::unique_ptr<sdf_plan_s> P(new (std::nothrow) sdf_plan_s());
    if (!P) return SDF_ERR_OOM;
    sdf_plan_impl *p = P.get();
    plan_geometry(p, D, dims, h, tau, precision, outputs, stream);
    if (dS && !(p->outputs & SDF_OUT_DS)) return SDF_ERR_INVALID_ARG;
    if (d2S && !(p->outputs & SDF_OUT_D2S)) return SDF_ERR_INVALID_ARG;
    if (sign && !((p->outputs & SDF_OUT_SIGN) && weights)) return SDF_ERR_INVALID_ARG;
    if (weights && !(p->outputs & SDF_OUT_SIGN)) return SDF_ERR_INVALID_ARG;
    for (int id : plan_kernel_ids(p)) {
        KernelSpec k;
        k.id = id;
        k.parity = kernel_parity(id, D);
        k.l1 = 0;
        k.scale = (id >= KER_HXX && id <= KER_HYZ) ? hessian_scale(p) : 1.0;
        k.c = nullptr;
        p->kslot[id] = (int)p->kernels.size();
        p->kernels.push_back(k);
    }
    plan_programme(p);  // groups (the noise factor is redone once the l1 norms exist)
    plan_buffer_sizes(p);
    double2 *tw64[3] = {nullptr, nullptr, nullptr};
    double *part = nullptr;
    double2 *bufX = nullptr, *bufY = nullptr;
    const size_t need = layout(p, K, nullptr, tw64, &part, &bufX, &bufY);
    if (need > kScratchBytes) {
        char msg[160];
        snprintf(msg, sizeof msg, "problem needs %zu bytes of scratch; the static array holds %zu", need,
                 kScratchBytes);
        set_last_error(msg);
        return SDF_ERR_CAPACITY;
    }
    // the scratch address belongs to the current device: the stream must be
    // one of that device's (else the kernels would address another GPU's
    // copy of the array, or fail to launch)
    {
        int dev = 0, sdev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaStreamGetDevice(p->stream, &sdev);
        if (e != cudaSuccess) {
            set_last_error(cudaGetErrorString(e));
            cudaGetLastError();
            return SDF_ERR_INVALID_ARG;
        }
        if (sdev != dev) {
            set_last_error("sdf_execute_noalloc: the stream belongs to another device than the current one");
            return SDF_ERR_INVALID_ARG;
        }
    }
    unsigned char *base = nullptr;
    NCK(scratch_address(&base));
    layout(p, K, base, tw64, &part, &bufX, &bufY);
    for (int a = 0; a < D; ++a) {
        if (precision == SDF_FP64) NCK(fill_twiddles<double>(p->tw[a], p->M[a], p->stream));
        else NCK(fill_twiddles<float>(p->tw[a], p->M[a], p->stream));
        NCK(fill_twiddles<double>(tw64[a], p->M[a], p->stream));
    }
    std::vector<double> host_part(kSpectraParts);
    NCK(build_spectra_into(p, bufX, bufY, part, host_part.data(), tw64));
    plan_programme(p);
    // the array keeps the previous call's contents: clear the device status
    NCK(cudaMemsetAsync(p->dsc, 0, sizeof(DevScalars), p->stream));
    p->last_K = K;
    const bool ww = weights != nullptr;
    NCK(launch_points(p, K, points, weights));
    uint8_t *fl = flags;
    int8_t *sg = sign;
    if (p->prec == SDF_FP32) {
        if (!fl) fl = p->flags_int;
        if (ww && !sg) sg = p->sign_int;
        NCK(cudaMemsetAsync(p->tile_flag, 0, p->nbins, p->stream));
        NCK(launch_cheb(p));
    }
    NCK(launch_forward(p, ww, nullptr, 0, nullptr));
    NCK(launch_inverse_epilogue(p, ww, S, dS, d2S, sg, fl));
    if (p->prec == SDF_FP32) NCK(launch_fixup(p, ww, S, dS, d2S, ww ? sg : nullptr, fl));
    if (flags) NCK(launch_source_flags(p, flags));
    NCK(debug_scan_outputs(p, S, dS, d2S));
    DevScalars hs;
    NCK(cudaMemcpyAsync(&hs, p->dsc, sizeof(DevScalars), cudaMemcpyDeviceToHost, p->stream));
    NCK(cudaStreamSynchronize(p->stream));
    return (sdf_status)hs.status;
}

