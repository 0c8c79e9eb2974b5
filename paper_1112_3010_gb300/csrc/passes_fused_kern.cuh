// passes_fused_kern.cuh -- definitions of the fused pass's launch helpers
// (run_fused, run_fused2p), included by the translation units that
// instantiate them (passes_fused_f2.cu, passes_fused_f3.cu,
// passes_fused_d.cu), so the many line-length variants compile in parallel.
#pragma once
#include "passes.cuh"

namespace sdf {

template <typename T, int DD, int FVV, int LG>
cudaError_t run_fused(unsigned grid, int nthr, size_t smem, cudaStream_t st, const cx<T> *fin, cx<T> *fout, int logL,
                      int n_in, int n_out, int R, int64_t n_lines, int64_t in_fs, int64_t out_fs, const FusedParams &F,
                      const cx<T> *twl, const FusedParams &F1, cx<T> *fout1) {
    cudaError_t e = set_smem<T>((const void *)k_fused<T, DD, FVV, LG>, smem);
    if (e != cudaSuccess) return e;
    k_fused<T, DD, FVV, LG><<<grid, nthr, smem, st>>>(fin, fout, logL, n_in, n_out, R, n_lines, in_fs, out_fs, F, twl,
                                                      F1, fout1);
    return cudaSuccess;
}

template <typename T, int LG>
cudaError_t run_fused2p(unsigned grid, int nthr, size_t smem, cudaStream_t st, const cx<T> *fin, cx<T> *fout,
                        int logL, int n_in, int n_out, int64_t in_fs, int64_t out_fs, const FusedParams &F, int nker,
                        const cx<T> *twl) {
    cudaError_t e = set_smem<T>((const void *)k_fused2p<T, LG>, smem);
    if (e != cudaSuccess) return e;
    k_fused2p<T, LG><<<grid, nthr, smem, st>>>(fin, fout, logL, n_in, n_out, in_fs, out_fs, F, nker, twl);
    return cudaSuccess;
}

// Explicit instantiations of run_fused<T, DD, FVV, LG> for every float line
// length SDF_BY_LOGL dispatches on.
#define SDF_INST_FUSED(T, DD, FVV, LG)                                                                          \
    template cudaError_t run_fused<T, DD, FVV, LG>(unsigned, int, size_t, cudaStream_t, const cx<T> *, cx<T> *, \
                                                   int, int, int, int, int64_t, int64_t, int64_t,               \
                                                   const FusedParams &, const cx<T> *, const FusedParams &, cx<T> *);
#define SDF_INST_FUSED2P(T, LG)                                                                                  \
    template cudaError_t run_fused2p<T, LG>(unsigned, int, size_t, cudaStream_t, const cx<T> *, cx<T> *, int, int, \
                                            int, int64_t, int64_t, const FusedParams &, int, const cx<T> *);
#define SDF_FOR_FLOAT_LOGL(M, ...)                                                                               \
    M(__VA_ARGS__, 0) M(__VA_ARGS__, 8) M(__VA_ARGS__, 9) M(__VA_ARGS__, 10) M(__VA_ARGS__, 11) M(__VA_ARGS__, 12) \
    M(__VA_ARGS__, 8 | kLineR3) M(__VA_ARGS__, 9 | kLineR3) M(__VA_ARGS__, 10 | kLineR3)

}  // namespace sdf
