/*
 * sdf.h -- C ABI of the GB300 (sm_103a) implementation of the convolution-based
 * signed distance method of Gurumoorthy & Rangarajan, "Fast convolution based
 * method for computing the signed distance function and its derivatives".
 *
 * What one execute computes (all on the GPU, on the plan's CUDA stream):
 *   1. Snap each point Y_k to its nearest grid node (Sec. 6, Examples 3-4) and
 *      scatter it onto a zero-padded M^D grid: g(X) = sum_k delta(X - Y_k)
 *      (eq. function_g, Table 1 step 2), and the tangent- or normal-weighted
 *      fields g_j = sum_k Z_k^j delta(X - Y_k) (Sec. 4.1) / P_k^j (Sec. 4.2).
 *   2. Convolve g by FFT with f(X) = exp(-||X||/tau) (eq. function_f, Table 1
 *      steps 1, 3-5), with f*X_j/||X|| (eq. SxSyconv) and with the Hessian
 *      kernels (eqs. Sxx, Syy, Sxy; the same differentiation in 3D), and the
 *      g_j with the winding-number kernels X_j/||X||^2 (eq.
 *      kappadiscretefinal, 2D) or degree kernels X_j/||X||^3 (eq. mudef, 3D).
 *   3. S = -tau log(phi) (eq. STilde, Table 1 step 6), grad S = (f_j f * g)/phi
 *      (eq. SxSyconv), the Hessian (eqs. Sxx, Syy, Sxy), and the sign: +1
 *      (inside) where |mu| >= 1/2, -1 outside (Sec. 4; positive inside, Sec. 1).
 *
 * Grids.  dims[a] = N_a nodes on axis a (x first); node i sits at i*h (origin
 * 0).  Every grid array is C-order with x fastest: element (x, y[, z]) at
 * x + N_0*(y + N_1*z).  The padded FFT size per axis is the smallest power of
 * two M_a >= max(2*N_a - 1, 16) (sdf_plan_set_padding may choose 3 * 2^k
 * instead), so the circular convolution equals the linear one on the N^D
 * output nodes.
 *
 * Precision.  SDF_FP64: every FFT pass, product and epilogue in double; grid
 * outputs are double.  SDF_FP32 (the mixed path): FFT passes and products in
 * float, outputs float; nodes where phi falls below the FP32 transform's noise
 * bound but inside the FP64 trust region are recomputed by a shifted direct
 * sum (flag SDF_FLAG_FIXUP), so S matches the FP64 path there.
 *
 * Trust region.  The FFT returns phi with an absolute error near u*|f|_1*|g|_2
 * (u the unit roundoff), so -tau log(phi) is noise where phi is tiny (the
 * paper's Sec. 3.3).  Both paths use the same FP64 trust threshold theta_64;
 * at nodes with phi < theta_64 they return S_cap = -tau log(theta_64) (a lower
 * bound on S), zero derivatives, and set SDF_FLAG_CAPPED (an SDF_FP32 plan in
 * full-range mode, sdf_plan_set_full_range, recomputes those nodes too and
 * caps nothing).  The sign is valid everywhere.
 *
 * Ownership and errors.  The caller owns every points/weights/output buffer;
 * the plan owns its workspace and kernel spectra.  All calls are asynchronous
 * on the plan's stream unless stated.  Errors detected on the device (a point
 * outside the grid, a bounded wait that expired) are recorded in the plan and
 * returned by sdf_sync().  No exception or longjmp crosses this ABI.  A plan is
 * not thread-safe: one host thread at a time per plan.
 */
#ifndef SDF_GB300_H
#define SDF_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sdf_plan_s *sdf_plan;

typedef enum {
    SDF_OK = 0,
    SDF_ERR_INVALID_ARG = 1,       /* bad argument; nothing was enqueued        */
    SDF_ERR_UNSUPPORTED = 2,       /* D not 1..3, a grid too large, or a        */
                                   /* combination the plan does not support    */
    SDF_ERR_POINT_OUT_OF_GRID = 3, /* some point snapped outside [0, N_a)       */
    SDF_ERR_OOM = 4,               /* device allocation failed                  */
    SDF_ERR_CUDA = 5,              /* a CUDA runtime call failed                */
    SDF_ERR_TIMEOUT = 6,           /* a bounded device-side wait expired        */
    SDF_ERR_CAPACITY = 7,          /* input larger than a fixed-size buffer     */
    SDF_ERR_INTERNAL = 8           /* a device-side consistency check failed    */
                                   /* (sdf_set_debug_checks)                    */
} sdf_status;

typedef enum { SDF_FP64 = 0, SDF_FP32 = 1 } sdf_precision;

/* Kernel sets (sdf_plan_set_kernel). */
typedef enum { SDF_KERNEL_EXP = 0, SDF_KERNEL_GREEN = 1 } sdf_kernel_set;

/* Output fields a plan prepares kernel spectra for (bit mask). */
enum {
    SDF_OUT_S = 1,    /* S (always computed)                               */
    SDF_OUT_DS = 2,   /* grad S, D planes                                  */
    SDF_OUT_D2S = 4,  /* Hessian, D(D+1)/2 planes: xx,yy[,zz],xy[,xz,yz]   */
    SDF_OUT_SIGN = 8  /* winding number (2D) / topological degree (3D)     */
};

/* Per-node flag bits written to the optional flags output. */
enum {
    SDF_FLAG_CAPPED = 1, /* phi below the FP64 trust threshold: S = S_cap       */
    SDF_FLAG_FIXUP = 2,  /* value from the shifted direct sum (SDF_FP32 plans)  */
    SDF_FLAG_SOURCE = 4  /* a point snapped onto this node (mu is meaningless) */
};

/* Plan facts, filled by sdf_plan_get_info(). */
typedef struct {
    int D;
    int precision;
    unsigned outputs;
    int64_t dims[3];          /* N_a                                       */
    int64_t padded[3];        /* M_a                                       */
    double h, tau;
    double kernel_l1[16];     /* l1 norm of each sampled kernel on the     */
                              /* padded grid, in plan order (unscaled)     */
    int n_kernels;
    double noise_const_fp32;  /* C in the noise model, float transforms    */
    double noise_const_fp64;  /* C in the noise model, double transforms   */
    double plan_ms;           /* wall time of sdf_plan_create              */
    size_t workspace_bytes;   /* device bytes owned by the plan            */
} sdf_plan_info;

/* Results of the last execute, filled by sdf_get_stats() (synchronises). */
typedef struct {
    double theta64;      /* FP64 trust threshold on phi                        */
    double theta32;      /* FP32 trust threshold on phi (SDF_FP32 plans)       */
    double s_cap;        /* -tau log(theta64)                                  */
    double g_norm2;      /* ||g||_2 = sqrt(sum over nodes of count^2)          */
    int64_t n_unique;    /* distinct occupied nodes                            */
    int64_t n_fixup_tiles;  /* tiles the direct-sum fix-up visited             */
    int64_t n_fixup_nodes;  /* nodes whose values it wrote (flag FIXUP only)   */
    int64_t n_capped;    /* nodes returned as S_cap (flag CAPPED)              */
    int64_t n_launches;  /* kernels the last execute launched                  */
    int64_t n_fixup_terms;  /* (node, occupied node) terms the fix-up summed   */
    /* Error report of the last execute, over the nodes NOT flagged CAPPED: a
     * priori bounds on |S - S_exact|, on each component of |grad S - exact|
     * and of |Hessian - exact| (0 when not requested), S_exact being the
     * paper's S (eq. STilde, in the shifted form of eq. Bound1) of the snapped
     * points in exact arithmetic.  They combine the transform error model of
     * the trust region (relative error of phi at most
     * (eps f/Q)/(1 - eps f/Q) where phi >= theta, eps = 2.5e-4, f and Q the
     * l1-norm terms of the model), the fix-up's tail, term and summation
     * errors (SDF_FP32 plans), and the rounding of the outputs.  For an
     * SDF_FP32 plan and an SDF_FP64 plan of the same problem,
     * |S_32 - S_64| <= err_bound_S(32) + err_bound_S(64) wherever neither is
     * capped.  Like the trust region, the transform part is a bound under the
     * calibrated noise model, not a proof. */
    double err_bound_S;
    double err_bound_dS;
    double err_bound_d2S;
    double trusted_frac; /* fraction of the N^D nodes not flagged CAPPED        */
} sdf_exec_stats;

/* Per-kernel device time, filled by sdf_profile_read(). */
typedef struct {
    char name[32];
    int64_t launches;
    double total_ms;     /* sum of CUDA-event durations on the plan's stream  */
} sdf_kernel_time;

/*
 * sdf_plan_create -- build a plan for a D-dimensional grid.
 *   out        receives the plan (NULL on failure).
 *   D          1, 2 or 3 (else SDF_ERR_UNSUPPORTED).  D = 1 (Sec. 2.1 treats
 *              1D alongside 2D and 3D) runs the whole path in one CTA per
 *              execute: no sign output (SDF_OUT_SIGN gives
 *              SDF_ERR_UNSUPPORTED), no sdf_backward, sdf_curvature,
 *              batches or autotuning.
 *   dims       host array of D node counts, x first, each in [2, 2048] (1D),
 *              [2, 4096] (2D) or [2, 512] (3D); M_a (above) must fit the
 *              device (else SDF_ERR_UNSUPPORTED).  sdf_plan_set_padding and
 *              sdf_plan_autotune may change M_a to 3 * 2^k.
 *   h          grid spacing (> 0).  tau: the paper's tau (> 0).
 *   precision  SDF_FP64 or SDF_FP32.
 *   outputs    mask of SDF_OUT_* bits.  SDF_OUT_S is implied.
 *   stream     cudaStream_t (as void*) on which every call enqueues; NULL is
 *              the legacy default stream.
 * Samples every kernel on the padded grid and transforms it in FP64 (Table 1
 * step 1 and the kernels of Secs. 4-5), storing 1/2^D of each spectrum in the
 * plan's precision.  Synchronous; allocates device memory.
 */
sdf_status sdf_plan_create(sdf_plan *out, int D, const int64_t *dims, double h,
                           double tau, int precision, unsigned outputs,
                           void *stream);

/*
 * sdf_execute -- one pass of the whole path (steps 1-3 above), enqueued on the
 * plan's stream.
 *   K          number of points (>= 1).
 *   points     device, K x D doubles, row-major, world coordinates.
 *   weights    device, K x D doubles: 2D tangents Z_k (eq. tangentVec;
 *              chord- or arc-length-weighted), 3D outward normals P_k times
 *              area (eq. normflux).  NULL: no sign is computed and S is
 *              unsigned.  Component sums per node are formed in 62-bit fixed
 *              point scaled to max|weight| (order-independent, deterministic).
 *   S          device, N^D values (double for SDF_FP64, float for SDF_FP32):
 *              signed S (sign * S) when the sign is computed, else S.
 *   dS         device, D planes of N^D (same type), grad S; NULL to skip.
 *   d2S        device, D(D+1)/2 planes, the Hessian; NULL to skip.
 *   sign       device, N^D int8 (+1 inside, -1 outside); NULL to skip.
 *   flags      device, N^D uint8 of SDF_FLAG_* bits; NULL to skip.
 * Requesting a field the plan was not created for returns SDF_ERR_INVALID_ARG.
 * The first call with a larger K than any before allocates point buffers.
 * Points that snap outside the grid are dropped and reported by sdf_sync().
 */
sdf_status sdf_execute(sdf_plan plan, int64_t K, const double *points,
                       const double *weights, void *S, void *dS, void *d2S,
                       int8_t *sign, uint8_t *flags);

/*
 * sdf_execute_multi -- sdf_execute of n plans on the same points: a sweep of
 * tau (the experiments of Sec. 6 vary tau on one point set), or the two
 * kernel sets side by side.  The plans must agree in D, dims, h, precision
 * and outputs (else SDF_ERR_INVALID_ARG) and be distinct; tau, the kernel set,
 * noise constants, tuning and full-range mode may differ.
 *   plans      host array of n plans.
 *   K, points, weights   as sdf_execute, shared by all plans.
 *   S, dS, d2S, sign, flags   host arrays of n device pointers (plan i's
 *              outputs, as sdf_execute); a NULL array skips that output for
 *              every plan, a NULL entry for that plan.
 * The snapping, binning and the tau-independent forward transforms (the
 * x-pass, and the y-pass in 3D: Table 1 step 3 up to the last axis) run once,
 * on plans[0]'s stream.  Each plan then runs its spectrum multiply, inverse
 * transforms, epilogue and fix-up on its own stream.  The sign (winding
 * number or degree, eqs. kappdiscreteZ, normflux) depends on neither tau nor
 * the kernel set: with weights, plans[0] computes it and the others copy it,
 * skipping its transforms.  With two plans, one fused launch on plans[0]'s
 * stream does both plans' products and inverse transforms on a single
 * forward transform of the counts.  plans[0]'s stream waits for all of them before
 * the call returns, so later work on plans[0]'s stream is ordered after the
 * whole call.  For plans with the same tile schedule, the results equal
 * those of n separate sdf_execute calls bit for bit.  1D plans run one
 * sdf_execute each.
 * Errors as sdf_execute; device errors are reported by sdf_sync() of the plan
 * that met them.
 */
sdf_status sdf_execute_multi(int n, const sdf_plan *plans, int64_t K,
                             const double *points, const double *weights,
                             void *const *S, void *const *dS, void *const *d2S,
                             int8_t *const *sign, uint8_t *const *flags);

/*
 * sdf_execute_multi_host -- sdf_execute_multi with HOST buffers, as
 * sdf_execute_host is to sdf_execute: the points and weights are copied once
 * (to plans[0]'s staging buffer); every output is computed into the plan's
 * device staging buffer and copied back by the copy engine, each plan's as
 * soon as its fix-up is done.  With two or more FP32 plans whose S, dS and
 * d2S buffers (those requested) of plans[0] are page-locked (pinned,
 * device-mapped), plans[0]'s S, dS and d2S are copied as soon as its
 * epilogue has written them, while the other plans compute, and its fix-up
 * then writes the nodes it recomputes straight into those host buffers.
 * The staging buffers grow to the outputs' size on first use (an
 * allocation, SDF_ERR_OOM if it fails).  Waits for every plan's stream and
 * returns the first non-OK status of sdf_sync() over the plans.  Errors as
 * sdf_execute_multi.
 */
sdf_status sdf_execute_multi_host(int n, const sdf_plan *plans, int64_t K,
                                  const double *points, const double *weights,
                                  void *const *S, void *const *dS,
                                  void *const *d2S, int8_t *const *sign,
                                  uint8_t *const *flags);

/*
 * sdf_execute_host -- sdf_execute with HOST buffers (same shapes and types):
 * copies points/weights to plan-owned device buffers, executes, brings the
 * requested outputs back, and waits for the stream.  S, dS and d2S in
 * page-locked (pinned, device-mapped) host memory are written by the kernels
 * directly, over the CPU-GPU link while the rest of the execute runs; other
 * outputs, and outputs in pageable memory, are staged on the device and
 * copied at the end.  Returns the device status as sdf_sync().
 */
sdf_status sdf_execute_host(sdf_plan plan, int64_t K, const double *points,
                            const double *weights, void *S, void *dS, void *d2S,
                            int8_t *sign, uint8_t *flags);

/*
 * sdf_backward -- adjoint of L = sum_X w(X) S(X) for UNSIGNED S (the chain
 * rule applied to eq. STilde):
 *   dL/dY_k = (a * k_grad)(Y^_k), a = w/phi, k_grad(X) = f(X) X/||X||
 *   dL/dtau = ( sum_X w S - sum_k (a * (||X|| f))(Y^_k) ) / tau
 * evaluated at the snapped points Y^_k (snapping is piecewise constant; this
 * is the gradient of the continuous definition at Y = Y^).
 *   K, points  as in sdf_execute (the same points as the forward).
 *   w          device, N^D loss weights dL/dS (plan type).
 *   S_saved    device, N^D unsigned S from the forward (plan type); phi is
 *              recovered as exp(-S/tau).
 *   flags      device, N^D flags from the forward or NULL; nodes with
 *              SDF_FLAG_CAPPED are skipped (their S does not depend on Y).
 *   dL_dY      device, K x D doubles (written for every point).
 *   dL_dtau    device, one double.
 * The plan must have SDF_OUT_DS.  Recomputes spectra; keeps no forward state.
 */
sdf_status sdf_backward(sdf_plan plan, int64_t K, const double *points,
                        const void *w, const void *S_saved,
                        const uint8_t *flags, double *dL_dY, double *dL_dtau);

/*
 * sdf_mesh_sources -- point sources of an oriented triangle mesh for the 3D
 * degree (Sec. 4.2, Example 5): triangle k becomes the point Y_k = its
 * incentre (vertices weighted by the opposite side lengths) with the weight
 * P_k = (B - A) x (C - A) / 2, the edge cross product scaled to the
 * triangle's area (area-weighted outward normal, so mu ~ 1 inside).
 *   nf, nv     triangles and vertices.
 *   V          device, nv x 3 doubles (world coordinates, as points).
 *   F          device, nf x 3 int64 vertex indices (A, B, C).
 *   center     host, 3 doubles, or NULL.  NULL: the faces' vertex order
 *              orients P_k (counter-clockwise seen from outside = outward).
 *              Given: P_k is negated where <Y_k - center, P_k> < 0 (the rule
 *              of Example 5, for objects star-shaped about center).
 *   points, weights  device, nf x 3 doubles each (caller-owned): pass them
 *              to sdf_execute as points and weights.
 * 3D plans only (SDF_ERR_UNSUPPORTED otherwise); a face index outside
 * [0, nv) sets SDF_ERR_INVALID_ARG, reported by sdf_sync.  Enqueued on the
 * plan's stream.
 */
sdf_status sdf_mesh_sources(sdf_plan plan, int64_t nf, int64_t nv, const double *V,
                            const int64_t *F, const double *center, double *points,
                            double *weights);

/*
 * sdf_curvature -- curvature fields from the grad S and Hessian planes an
 * sdf_execute wrote (Sec. 5 names the Gaussian, mean and principal
 * curvatures of S among the uses of its derivatives, without formulas).
 *   2D: the graph z = S(x, y) as a Monge patch, W = 1 + S_x^2 + S_y^2:
 *       K = (S_xx S_yy - S_xy^2)/W^2,
 *       H = ((1 + S_y^2) S_xx - 2 S_x S_y S_xy + (1 + S_x^2) S_yy)/(2 W^{3/2}).
 *   3D: the paper is silent; the level surfaces of S, g = |grad S|:
 *       H = (g^2 tr(Hess) - grad S^T Hess grad S)/(2 g^3),
 *       K = grad S^T adj(Hess) grad S / g^4 (0 where g = 0).
 *   Principal curvatures k1 >= k2 = H +- sqrt(max(H^2 - K, 0)).
 *   dS, d2S  device, the D and D(D+1)/2 planes of one execute (plan type).
 *   flags    device N^D flags of the same execute, or NULL; nodes with
 *            SDF_FLAG_CAPPED get 0.
 *   curv     device, 4 planes of N^D (plan type): K, H, k1, k2.
 * Caller-owned buffers; enqueued on the plan's stream (asynchronous, errors
 * as for sdf_execute).  SDF_ERR_INVALID_ARG for a NULL plan or plane;
 * SDF_ERR_UNSUPPORTED for a 1D plan.
 */
sdf_status sdf_curvature(sdf_plan plan, const void *dS, const void *d2S,
                         const uint8_t *flags, void *curv);

/* Wait for the plan's stream; return (and clear) any error recorded on the
 * device since the last sdf_sync, or SDF_ERR_CUDA for an asynchronous fault. */
sdf_status sdf_sync(sdf_plan plan);

/* Plan facts (host-side, no synchronisation). */
sdf_status sdf_plan_get_info(sdf_plan plan, sdf_plan_info *info);

/* Statistics of the last execute (synchronises the stream). */
sdf_status sdf_get_stats(sdf_plan plan, sdf_exec_stats *stats);

/*
 * sdf_plan_set_noise_constants -- replace the constants C_32 and C_64 of the
 * transform error model (include/sdf.h, "Trust region"): the trust threshold
 * is theta_p = C_p u_p sqrt(log2 n) Q ||g||_2 / (sqrt(n) * 2.5e-4), with
 * n = prod(M_a), u_p the unit roundoff and Q a combination of kernel l1 norms.
 * Values <= 0 keep the current constant.  Used to calibrate the model
 * against the oracle; the built-in constants come from that calibration.
 */
sdf_status sdf_plan_set_noise_constants(sdf_plan plan, double c_fp32, double c_fp64);

/*
 * Tile schedule.  lines_T: lines of the transforms each CTA of the transposed
 * passes (x-pass, 3D y-passes, epilogue) handles; lines_F: lines per CTA of the
 * fused pass; fused_variant: 1 = at most 256 threads and two CTAs per SM,
 * 2 = up to 128 registers per thread, 3 = 2D float plans: one CTA per pair of
 * mirror columns with the spectrum rows staged in shared memory (falls back to
 * 2 when it does not fit).  0 (or an invalid value, rounded down to a valid
 * one) keeps the built-in rule (2).  Results agree across schedules to the
 * rounding of the transforms (the order of a few float operations differs).
 */
sdf_status sdf_plan_set_tuning(sdf_plan plan, int lines_T, int lines_F, int fused_variant);

/*
 * sdf_plan_set_epilogue_loads -- how the epilogue (the last inverse
 * transform and Table 1 step 6) reads its transposed input.  mode 0 (the
 * default): SDF_FP32 plans whose last-axis lines have a compiled length
 * that is a multiple of 256 (256 ... 4096, 768, 1536, 3072) with at least
 * two lines per CTA and an even line count stage each group's lines in
 * shared memory by TMA tensor copies (cp.async.bulk.tensor, mbarrier
 * completion), the next group's copy overlapping the current group's
 * transform; other plans load per thread.  mode 1: per-thread loads always.
 * Results are identical either way.  A TMA wait that does not complete
 * within a bounded number of polls makes the execute report
 * SDF_ERR_TIMEOUT (sdf_sync).  SDF_ERR_INVALID_ARG for another mode or a
 * NULL plan.  sdf_plan_autotune times both.
 */
sdf_status sdf_plan_set_epilogue_loads(sdf_plan plan, int mode);

/*
 * sdf_plan_autotune -- choose the padded sizes and the tile schedule by
 * timing them on the plan's stream with the given inputs (as sdf_execute;
 * outputs are not written), keep the fastest, and report the schedule in
 * *lines_T, *lines_F, *fused_variant (host, may be NULL; the sizes are in
 * sdf_plan_get_info's `padded`).
 *   1. Padded sizes: per axis the power of two of sdf_plan_create and, where
 *      it is smaller, the least 3 * 2^k >= 2 N_a - 1 (sdf_plan_set_padding);
 *      every combination is timed over the whole execute.  A plan of a batch
 *      that borrows another plan's spectra keeps its sizes.
 *   2. The tile schedule (sdf_plan_set_tuning) and the epilogue's loads
 *      (sdf_plan_set_epilogue_loads) on those sizes: the passes each knob
 *      affects are timed.
 * Each candidate runs `reps` executes after one warm-up, timed with CUDA
 * events.  The choice is kept in a cache keyed by the GPU's name and
 * architecture, D, dims, precision, outputs and kernel set: a later call on
 * a problem of the same key applies the cached choice without timing.  The
 * cache is the text file $SDF_AUTOTUNE_CACHE (an empty value disables it),
 * else $XDG_CACHE_HOME/sdf_gb300/autotune.tsv, else
 * $HOME/.cache/sdf_gb300/autotune.tsv; it is optional (unreadable or
 * unwritable: no cache).  Synchronous; may rebuild the plan's spectra.
 * The paper chooses no transform sizes or schedules; this is the library's.
 */
sdf_status sdf_plan_autotune(sdf_plan plan, int64_t K, const double *points,
                             const double *weights, int reps, int *lines_T,
                             int *lines_F, int *fused_variant);

/*
 * sdf_plan_set_padding -- set the padded transform size of each axis:
 * padded[a] (host, D values) must be a power of two or 3 * 2^k (>= 48), at
 * least max(2 N_a - 1, 16) so that the circular convolution still equals
 * the linear one on the N^D nodes, and at most 8192 (2D) or 1024 (3D); else
 * SDF_ERR_INVALID_ARG.  Lines of 3 * 2^k points are transformed with a
 * radix-3 stage ahead of the radix-16 ones.  Rebuilds the plan's twiddles,
 * kernel spectra and transform buffers (synchronous, allocates); on a CUDA
 * error the plan must be destroyed.  SDF_ERR_UNSUPPORTED for 1D plans and
 * for a plan of a batch that borrows another plan's spectra.  Results agree
 * with the power-of-two padding to the rounding of the transforms (the trust
 * threshold follows n = prod M_a).
 */
sdf_status sdf_plan_set_padding(sdf_plan plan, const int64_t *padded);

/*
 * sdf_plan_set_full_range -- SDF_FP32 plans: when enable != 0, the fix-up
 * computes every node whose phi is below theta_32, with no cap at theta_64:
 * S, grad S and the Hessian come from the shifted direct sum of Sec. 2.4
 * (eq. Bound1) however small phi is, so nothing is flagged SDF_FLAG_CAPPED.
 * This is the range the paper reaches only with multiple-precision FFTs
 * (Secs. 3.3-3.4, Example 1 at tau/h ~ 0.03).  Costs fix-up time in
 * proportion to the untrusted nodes.  SDF_ERR_UNSUPPORTED for SDF_FP64 plans
 * (they have no fix-up); SDF_ERR_INVALID_ARG for a NULL plan.
 */
sdf_status sdf_plan_set_full_range(sdf_plan plan, int enable);

/*
 * sdf_plan_set_kernel -- choose the kernel phi is convolved from.
 *   SDF_KERNEL_EXP    exp(-||o||/tau): the paper's G~ (eq. GTildeDefinition)
 *                     with its constants dropped (eq. wavefunc).  The default.
 *   SDF_KERNEL_GREEN  the exact Green's function of -tau^2 lap phi + phi =
 *                     psi (Sec. 2.1: K_0(r/tau)/(2 pi tau^2) in 2D, eq.
 *                     GreensFunction2D; exp(-r/tau)/(4 pi tau^2 r) in 3D, eq.
 *                     GreensFunction3D), scaled as in eq. phiapproxSol with
 *                     gamma = D/2 (psi_k = tau^-D/2 on a box of side tau,
 *                     Sec. 2.2): g(o) = tau^-D/2 c_D Gamma_D(||o||/tau), see
 *                     sdf_green_profile.  At o = 0, where the mid-point value
 *                     is infinite, g is the integral of tau^-D/2 G over the
 *                     source's box, tau^-D/2 c_D A_D.  S = -tau log phi keeps
 *                     the constants, so S tends to R only as tau -> 0
 *                     (App. A); grad S, the Hessian and the sign are computed
 *                     as for SDF_KERNEL_EXP from the matching derivative
 *                     kernels.
 * Rebuilds the plan's kernel spectra (synchronous, allocates).  Errors:
 * SDF_ERR_INVALID_ARG for a NULL plan or an unknown set; SDF_ERR_UNSUPPORTED
 * for SDF_KERNEL_GREEN on an SDF_FP32 plan (its fix-up sums exp(-r/tau)
 * terms) or on a plan of a batch.  sdf_backward on a plan with
 * SDF_KERNEL_GREEN returns SDF_ERR_UNSUPPORTED (the adjoint is derived for
 * exp(-r/tau)).  Call between executes, not while one is in flight.
 */
sdf_status sdf_plan_set_kernel(sdf_plan plan, int kernel_set);

/*
 * sdf_green_profile -- host only, no device work: the radial profile of the
 * exact Green's function set in the unit z = r/tau, G = tau^-D c_D Gamma_D(z)
 * (c_1 = 1/2, c_2 = 1/(2 pi), c_3 = 1/(4 pi); Gamma_1 = exp(-z),
 * Gamma_2 = K_0(z), Gamma_3 = exp(-z)/z; Sec. 2.1).
 *   D         1, 2 or 3.
 *   n, z      n host values z >= 0.
 *   g, g1, g2 host arrays of n: Gamma_D(z), Gamma_D'(z), Gamma_D''(z).  For
 *             z = 0: g = A_D (the integral of Gamma_D over [-1/2, 1/2]^D,
 *             from the divergence theorem; 1 for D = 1) and g1 = g2 = 0.
 * SDF_ERR_INVALID_ARG for D outside 1..3, NULL arrays with n > 0, or a z that
 * is negative or not finite (the arrays are then partly written).
 */
sdf_status sdf_green_profile(int D, int64_t n, const double *z, double *g,
                             double *g1, double *g2);

/*
 * sdf_profile_enable -- when enable != 0, every kernel the plan launches is
 * bracketed by a pair of CUDA events recorded on the plan's stream (the
 * stream the kernel runs on), so the durations are device times of that
 * kernel.  Costs two event records per launch; off by default.
 */
sdf_status sdf_profile_enable(sdf_plan plan, int enable);

/*
 * sdf_profile_read -- synchronise the stream and return, per kernel name, the
 * launches and summed event durations recorded since the last read (at most
 * max entries written to out, host memory).  Returns the number of entries
 * written (>= 0) or -1 on error.  Resets the counters.
 */
int sdf_profile_read(sdf_plan plan, sdf_kernel_time *out, int max);

/*
 * Batches: many independent problems (uneven grid sizes and point counts)
 * executed together.  Problems with identical (D, dims, h, tau, precision,
 * outputs) share one set of kernel spectra.  Problems are spread over
 * `n_streams` worker streams; the first sdf_batch_execute (and any call whose
 * K or buffer pointers differ from the previous call's) runs every problem
 * once, then captures the whole batch -- all problems, all passes, forked
 * across the worker streams and joined back -- into one CUDA graph; every
 * later call with the same arguments is one cudaGraphLaunch on `stream`.
 * This is the paper's method applied per problem (Table 1, Secs. 4-5); the
 * batching itself has no counterpart in the paper.
 */
typedef struct sdf_batch_s *sdf_batch;

/*
 * sdf_batch_create -- n problems of dimension D.
 *   dims       host, n x D node counts (x first per problem).
 *   h, tau     host, n values each.
 *   precision, outputs   as sdf_plan_create, common to all problems.
 *   n_streams  worker streams (1..32) the problems are spread over.
 *   stream     cudaStream_t (as void*) the graph is launched on.
 * Synchronous; allocates device memory.
 */
sdf_status sdf_batch_create(sdf_batch *out, int n, int D, const int64_t *dims,
                            const double *h, const double *tau, int precision,
                            unsigned outputs, int n_streams, void *stream);

/*
 * sdf_batch_execute -- every problem of the batch, as sdf_execute per problem.
 * All arrays are host arrays of n entries; each pointer entry is a device
 * buffer as in sdf_execute (NULL where sdf_execute allows NULL; the whole
 * array may be NULL to mean all NULL).  Asynchronous on `stream`.
 */
sdf_status sdf_batch_execute(sdf_batch batch, const int64_t *K,
                             const double *const *points,
                             const double *const *weights, void *const *S,
                             void *const *dS, void *const *d2S,
                             int8_t *const *sign, uint8_t *const *flags);

/*
 * sdf_batch_autotune -- sdf_plan_autotune for a batch: each problem that owns
 * a set of kernel spectra (the first of its geometry) is tuned on its own
 * inputs (K, points, weights: host arrays of n entries, as
 * sdf_batch_execute), and the problems sharing its spectra take its padded
 * sizes, spectra and tile schedule.  The next sdf_batch_execute captures a
 * new graph.  Synchronous.
 */
sdf_status sdf_batch_autotune(sdf_batch batch, const int64_t *K,
                              const double *const *points,
                              const double *const *weights, int reps);

/* Wait for the batch; return the first device-side error of any problem. */
sdf_status sdf_batch_sync(sdf_batch batch);

/* Plan of problem i (owned by the batch), for sdf_get_stats and the like. */
sdf_plan sdf_batch_plan(sdf_batch batch, int i);

/* Free the batch, its plans, streams and graph. */
void sdf_batch_destroy(sdf_batch batch);

/*
 * sdf_execute_noalloc -- the whole path (plan set-up and one execute) for a
 * small problem, with no device allocation at all.  The paper has no
 * counterpart; this entry point exists for callers that cannot call
 * cudaMalloc: a process whose device memory belongs to another allocator
 * (a framework's caching pool), a plugin whose host forbids device
 * allocation after start-up, or a service held to a memory budget fixed in
 * advance.  Every scratch buffer (kernel spectra, transform buffers, point
 * bins, flags, device status) lives in one static 32 MiB device array
 * inside this library; every GPU that loads the library holds it until the
 * process exits.  The caller still owns points, weights and outputs.
 *
 *   D, dims, h, tau, precision, outputs   as sdf_plan_create (D = 2 or 3)
 *   K, points, weights, S, dS, d2S, sign, flags   as sdf_execute (K >= 1)
 *   stream     cudaStream_t (as void*) for the work; it must belong to the
 *              current device (else SDF_ERR_INVALID_ARG, nothing enqueued)
 *
 * Limits: problems whose scratch exceeds 32 MiB are rejected with
 * SDF_ERR_CAPACITY before any device work (sdf_last_error() gives the size
 * needed).  That admits 2D grids up to 256 x 256 in either precision with
 * K <= 65536 points, and 3D grids up to 32^3.
 *
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.  The call
 * is synchronous (it waits for its stream and returns the device status, as
 * sdf_sync), on success and on every error return after work was enqueued,
 * so no kernel of a finished call still uses the array.  Host-to-device
 * copies (twiddle tables) are ordered on `stream`, not the legacy default
 * stream.  All calls share the one array, which keeps the last call's
 * contents; every counter that must start at zero is cleared by each call.
 * Calls from this process are serialised by a lock; calls that overlap on the
 * GPU from elsewhere (another process using the same library image cannot)
 * would race on the array.
 */
sdf_status sdf_execute_noalloc(int D, const int64_t *dims, double h, double tau,
                               int precision, unsigned outputs, int64_t K,
                               const double *points, const double *weights,
                               void *S, void *dS, void *d2S, int8_t *sign,
                               uint8_t *flags, void *stream);

/*
 * sdf_debug_hook -- test hooks for the failure paths (process-wide; the
 * paper has no counterpart).  value >= 0, else SDF_ERR_INVALID_ARG; an
 * unknown hook gives SDF_ERR_INVALID_ARG.
 *   SDF_HOOK_FAIL_ALLOC      the value-th device allocation the library
 *                            makes from now on (1 = the next) fails as if the
 *                            device were out of memory: the call reports
 *                            SDF_ERR_OOM and releases what it had allocated.
 *                            0 disables.
 *   SDF_HOOK_TMA_WAIT_POLLS  value > 0: the epilogue's TMA waits poll, `value`
 *                            times, a barrier that nothing completes, so every
 *                            execute through the TMA epilogue meets the expiry
 *                            path on its first group: the copy in flight still
 *                            lands (the kernel waits for it, bounded) and
 *                            sdf_sync reports SDF_ERR_TIMEOUT; the plan stays
 *                            usable.  0: the normal waits.
 */
enum { SDF_HOOK_FAIL_ALLOC = 1, SDF_HOOK_TMA_WAIT_POLLS = 2, SDF_HOOK_CORRUPT_BINS = 3 };
sdf_status sdf_debug_hook(int hook, int64_t value);
/*   SDF_HOOK_CORRUPT_BINS    value != 0: after binning, every execute adds
 *                            one to the unique-node count of the first bin
 *                            that lies wholly inside the grid and holds no
 *                            repeated node, so that its node list takes in
 *                            the next occupied bin's first node.  Every
 *                            kernel still reads and writes inside its
 *                            buffers (the borrowed node is a valid node of
 *                            the bin's box); the results are wrong, and with
 *                            the debug checks on the execute reports
 *                            SDF_ERR_INTERNAL.  0 disables. */

/*
 * sdf_set_debug_checks -- device-side consistency checks (process-wide; the
 * paper has no counterpart).  Off unless the environment variable
 * SDF_DEBUG_CHECKS is set to a non-zero value when the library is first
 * used, or this call turns them on (on != 0).  With them on, every execute
 * also checks on the device, after binning, the structures the later
 * kernels address memory through: bin offsets ascending and within the
 * binned points, each bin's unique-node count within its points, node codes
 * inside the bin and the grid, multiplicities positive; for float plans,
 * after the Chebyshev map, the per-row lists of occupied bins (ascending,
 * within the row); and at the end, that S, dS and d2S are finite.  A failed
 * check records SDF_ERR_INTERNAL (reported by sdf_sync, unless an earlier
 * error was recorded) and sdf_last_error() names the check and the index
 * where it failed.  The checks read only: results are bitwise those of an
 * execute without them.  Cost: a few extra launches per execute.
 */
sdf_status sdf_set_debug_checks(int on);
int sdf_get_debug_checks(void);

/* Free the plan and everything it owns (synchronises its stream). */
void sdf_plan_destroy(sdf_plan plan);

/* Static description of a status code. */
const char *sdf_status_string(sdf_status status);

/* Last CUDA error text recorded by the library (thread-local; static storage). */
const char *sdf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SDF_GB300_H */
