// passes_fused_f2.cu -- the 2D float variants of the fused pass (per-line and
// paired-column kernels, every compiled line length).
#include "passes_fused_kern.cuh"

namespace sdf {
SDF_FOR_FLOAT_LOGL(SDF_INST_FUSED, float, 2, 0)
SDF_INST_FUSED(float, 2, 1, 0)
SDF_FOR_FLOAT_LOGL(SDF_INST_FUSED2P, float)
}  // namespace sdf
