// sdf_internal.cuh -- plan layout and kernel launchers shared by the .cu files
// of the library.  Nothing here is part of the C ABI (include/sdf.h).
#pragma once
#include <cuda.h>  // CUtensorMap (the type only: tensor maps are encoded through the runtime's driver entry point)
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sdf.h"
#include "fft_core.cuh"

namespace sdf {

constexpr int kBin = 8;          // bin edge in nodes (8x8 in 2D, 8x8x8 in 3D)
constexpr int kMaxKernels = 16;  // kernel spectra per plan
constexpr int kMaxGroups = 8;    // complex inverse transforms per execute

// Kernels sampled on the padded grid (Table 1 step 1, Secs. 4-5).  Offsets o
// are in world units (node offset times h), r = ||o||, n = o/r, E = exp(-r/tau).
enum KernelId {
    KER_PHI = 0,  // E                                   (eq. function_f)
    KER_GX, KER_GY, KER_GZ,  // n_j E                    (eq. SxSyconv)
    KER_HXX, KER_HYY, KER_HZZ, KER_HXY, KER_HXZ, KER_HYZ,  // [(d_ij - n_i n_j)/r - n_i n_j/tau] E
    KER_W1, KER_W2, KER_W3,  // 2D: o_2/r^2, o_1/r^2 (eq. fcfsfr products); 3D: o_j/r^3 (eq. mudef)
    KER_RF,                  // r E (derivative in tau, adjoint only)
    KER_COUNT
};

struct KernelSpec {
    int id;
    int parity;     // bit a set: kernel odd along axis a
    double l1;      // sum over the padded grid of |k| (unscaled)
    double scale;   // stored spectrum = scale * spectrum of k (keeps packed pairs balanced)
    void *c;        // device, compressed real spectrum (plan precision)
};

// One complex inverse transform: out = sum_t beta_t * Khat_{kernel_t} * Fhat_{field_t}.
// Terms 0..n-1; the real and imaginary parts of the inverse are two real channels.
struct Term {
    int kslot;      // index into plan->kernels
    int field;      // input field 0..2
    double br, bi;  // complex coefficient beta (includes the kernel's i^odd factor)
};
struct Group {
    int nterm;
    Term term[3];
};

// Epilogue channel layout of each group (what the real / imaginary parts hold).
enum Channel { CH_NONE = 0, CH_PHI, CH_GX, CH_GY, CH_GZ, CH_HXX, CH_HYY, CH_HZZ, CH_HXY, CH_HXZ, CH_HYZ, CH_MU,
               CH_AGX, CH_AGY, CH_AGZ, CH_ARF };

// Device-side scalars of one plan.
struct DevScalars {
    int status;                 // sdf_status recorded on the device
    int pad0;
    unsigned long long wmax;    // bits of max |weight| (positive doubles order as integers)
    unsigned long long sum_c2;  // sum over nodes of count^2
    unsigned long long n_fixup_tiles, n_fixup_nodes, n_capped, n_fixup_terms;
    int64_t n_unique;
    double dl_dtau_acc;         // adjoint partial sum (deterministic order not required)
    // fix-up facts behind the error report (sdf_get_stats): the most terms any
    // written node summed, the most ring batches any tile took, and the bits
    // of the largest 1/max(m, 1) over written nodes (m: distance to the
    // nearest point in nodes; positive floats order as their bits)
    unsigned long long fix_nmax, fix_rounds;
    unsigned fix_rinv_bits, pad1;
    // debug checks (sdf_set_debug_checks): the first failed check and where
    int dbg_check, pad2;
    long long dbg_where;
};

// Kernel-level event timing (sdf_profile_enable) and the launch counter.
struct ProfRec {
    const char *name;
    cudaEvent_t a, b;
};

struct sdf_plan_impl {
    int D = 0;
    int prec = SDF_FP32;
    unsigned outputs = 0;
    int64_t N[3] = {1, 1, 1}, M[3] = {1, 1, 1};
    int logM[3] = {0, 0, 0};
    int64_t nb[3] = {1, 1, 1};  // bins per axis
    int64_t nbins = 0, nnodes = 0;
    double h = 0, tau = 0;
    cudaStream_t stream = nullptr;
    double plan_ms = 0;
    double noise_c32 = 0, noise_c64 = 0;
    double q_factor = 0;     // combination of kernel l1 norms entering theta
    double q_f = 0, q_g = 0, q_h = 0;  // its parts: l1 noise norms of the phi, gradient, Hessian channels
    double q_factor_adj = 0;

    void *tw[3] = {nullptr, nullptr, nullptr};  // per-axis twiddle tables (plan precision)
    std::vector<KernelSpec> kernels;
    int kslot[KER_COUNT];

    // fixed transform programme (forward fields, output groups)
    int nfield = 0;
    int ngroup = 0;
    Group group[kMaxGroups];
    int gch[kMaxGroups][2];  // channel of real / imaginary part

    // workspace
    void *bufA = nullptr, *bufB = nullptr;
    size_t bytesA = 0, bytesB = 0;
    int64_t Kcap = 0;
    int *pt_key = nullptr;    // per point: bin
    int *pt_lc = nullptr;     // per point: local cell (or -1 when out of grid)
    long long *pt_entry = nullptr;  // per bin slot: (local cell << 40) | point
    int *bin_count = nullptr, *bin_start = nullptr, *bin_fill = nullptr, *bin_nuniq = nullptr;
    int *ucell = nullptr, *ucount = nullptr;
    double *uw = nullptr;
    unsigned char *cheb = nullptr;   // Chebyshev bin distance to an occupied bin (capped)
    // FP32 plans: the occupied bins of each bin row (row = by + nb1 bz), x
    // ascending: occ_x[occ_start[row] .. occ_start[row + 1]); occ_tmp holds
    // the per-row counts and scan partials while the lists are built
    int *occ_start = nullptr, *occ_x = nullptr, *occ_tmp = nullptr;
    unsigned char *tile_flag = nullptr;
    uint8_t *flags_int = nullptr;    // FP32 plans: flags when the caller passes none
    int8_t *sign_int = nullptr;      // FP32 plans: sign when the caller passes none
    int64_t last_K = 0;
    DevScalars *dsc = nullptr;
    DevScalars *hsc = nullptr;       // pinned mirror
    double *staging = nullptr;       // device copies for sdf_execute_host
    size_t staging_bytes = 0;
    size_t workspace_bytes = 0;
    double last_theta64 = 0, last_theta32 = 0, last_scap = 0;
    // adjoint programme (built at the first sdf_backward) and its buffers
    int adj_ngroup = 0;
    Group adj_group[2];
    int adj_gch[2][2];
    void *adj_planes = nullptr;      // D+1 dense planes (plan precision)
    double *adj_part = nullptr;      // reduction partials
    // kernel spectra owned by another plan of the same shape (batches)
    bool shares_spectra = false;
    // tile schedule (0: built-in rule): lines per CTA of the transposed passes
    // and of the fused pass, and the fused pass's register variant
    int tune_RT = 0, tune_RF = 0, tune_FV = 0;
    int tune_EV = 0;  // epilogue loads: 0 = TMA staging where it applies, 1 = per-thread loads
    bool full_range = false;  // fix-up without the theta_64 cap (sdf_plan_set_full_range)
    // the epilogue's TMA tensor map over its input (encoded for the buffer,
    // sizes and lines per CTA in epi_tmap_key; rebuilt when they change)
    CUtensorMap epi_tmap;
    int64_t epi_tmap_key[5] = {0, 0, 0, 0, 0};
    int kernel_set = SDF_KERNEL_EXP;  // sdf_plan_set_kernel
    // profiling
    bool prof_on = false;
    int64_t nlaunch = 0;      // kernels launched by the current/last execute
    std::vector<ProfRec> prof_recs;
    std::vector<cudaEvent_t> prof_pool;
};

// An NVTX range for the lifetime of the object (public calls); kernel
// launches get theirs from prof_begin / prof_end.
struct ScopedRange {
    explicit ScopedRange(const char *name);
    ~ScopedRange();
};

// Multiprocessors of the current device.
int sm_count();

// cudaMalloc through the allocation-failure test hook (sdf_debug_hook); the
// poll limit the hook sets for the epilogue's TMA waits (0: the default).
cudaError_t dev_alloc(void **ptr, size_t bytes);
unsigned tma_wait_polls();

// Bracket one kernel launch: prof_begin before, prof_end after (also an NVTX
// range named after the kernel).
void prof_begin(sdf_plan_impl *p, const char *name, cudaStream_t st);
void prof_end(sdf_plan_impl *p, cudaStream_t st);

// ---- launchers (defined in the .cu files) ----
cudaError_t launch_points(sdf_plan_impl *p, int64_t K, const double *points, const double *weights);
cudaError_t launch_cheb(sdf_plan_impl *p, cudaStream_t on = nullptr);  // on: another stream than p's
cudaError_t launch_forward(sdf_plan_impl *p, bool with_weights, const void *dense_in, int dense_mode,
                           const uint8_t *flags_in);
cudaError_t launch_forward_shared_part(sdf_plan_impl *p, bool with_weights);
cudaError_t launch_forward_from(sdf_plan_impl *p, const sdf_plan_impl *shared, bool skip_mu = false,
                                const sdf_plan_impl *pair = nullptr);
cudaError_t launch_inverse_epilogue(sdf_plan_impl *p, bool with_weights, void *S, void *dS, void *d2S,
                                    int8_t *sign, uint8_t *flags, const int8_t *sign_in = nullptr);
cudaError_t launch_fixup(sdf_plan_impl *p, bool with_sign, void *S, void *dS, void *d2S, const int8_t *sign,
                         uint8_t *flags);
cudaError_t launch_source_flags(sdf_plan_impl *p, uint8_t *flags);
// Debug checks (debugcheck.cu): the switch, the bin-corruption test hook, and
// the check launches after binning, after the Chebyshev map and on outputs.
bool debug_checks();
void set_debug_checks(bool on);
void set_corrupt_bins(long long v);
cudaError_t debug_after_binning(sdf_plan_impl *p);
cudaError_t debug_after_cheb(sdf_plan_impl *p, cudaStream_t st);
cudaError_t debug_scan_outputs(sdf_plan_impl *p, const void *S, const void *dS, const void *d2S);
cudaError_t build_spectra(sdf_plan_impl *p);
cudaError_t launch_line1d(sdf_plan_impl *p, int64_t K, const double *points, void *S, void *dS, void *d2S,
                          uint8_t *flags);
cudaError_t launch_adjoint(sdf_plan_impl *p, int64_t K, const double *points, const void *w, const void *S_saved,
                           const uint8_t *flags, double *dL_dY, double *dL_dtau);

double hessian_scale(const sdf_plan_impl *p);
double green_origin_integral(int D);  // A_D of the exact Green's function set (spectra.cu)

// Compressed spectrum of one kernel: one row per folded line-axis frequency
// (2D: f0; 3D: (f1, f0)), each row the folded last-axis frequencies padded to
// a multiple of 4 values (16-byte aligned rows).
// Rows of bins (x fixed to the row) and the scratch the occupied-bin lists need.
inline int64_t bin_rows(const sdf_plan_impl *p) { return p->nb[1] * p->nb[2]; }
inline int64_t occ_tmp_len(const sdf_plan_impl *p) { return bin_rows(p) + (bin_rows(p) + 4095) / 4096 + 1; }

inline int64_t spec_row_len(const sdf_plan_impl *p) { return ((p->M[p->D - 1] / 2 + 1) + 3) & ~int64_t(3); }
inline int64_t spec_rows(const sdf_plan_impl *p) {
    return p->D == 1 ? 1 : (p->D == 2 ? p->M[0] / 2 + 1 : (p->M[0] / 2 + 1) * (p->M[1] / 2 + 1));
}

sdf_status plan_create_shared(sdf_plan *out, int D, const int64_t *dims, double h, double tau, int precision,
                              unsigned outputs, void *stream, const sdf_plan_impl *share_from);
// New padded sizes (twiddles, spectra, buffers rebuilt; share_from: borrow
// its spectra), and whether sizes M are allowed for plan p.
sdf_status plan_repad(sdf_plan_impl *p, const int64_t *M, const sdf_plan_impl *share_from);
bool padding_ok(const sdf_plan_impl *p, const int64_t *M);

// plan set-up steps shared by sdf_plan_create and sdf_execute_noalloc
void plan_geometry(sdf_plan_impl *p, int D, const int64_t *dims, double h, double tau, int precision,
                   unsigned outputs, void *stream);
std::vector<int> plan_kernel_ids(const sdf_plan_impl *p);
void plan_programme(sdf_plan_impl *p);
void plan_buffer_sizes(sdf_plan_impl *p);
int kernel_parity(int id, int D);
void set_last_error(const char *msg);  // text returned by sdf_last_error()
double theta_coef(const sdf_plan_impl *p, int prec);
constexpr int kSpectraParts = 1024;
constexpr int kAdjParts = 1024;  // blocks of each adjoint reduction (fixed: deterministic sums)
cudaError_t build_spectra_into(sdf_plan_impl *p, double2 *bufX, double2 *bufY, double *part, double *host_part,
                               double2 *const *tw64);

// noise model: floor_p = C_p u_p sqrt(log2 n) ||k||_1 ||g||_2 / sqrt(n), theta = floor/eps
constexpr double kTrustEps = 2.5e-4;

}  // namespace sdf

struct sdf_plan_s : public sdf::sdf_plan_impl {};
