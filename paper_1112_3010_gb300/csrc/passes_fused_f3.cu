// passes_fused_f3.cu -- the 3D float variants of the fused pass (every
// compiled line length).
#include "passes_fused_kern.cuh"

namespace sdf {
SDF_FOR_FLOAT_LOGL(SDF_INST_FUSED, float, 3, 0)
SDF_INST_FUSED(float, 3, 1, 0)
}  // namespace sdf
