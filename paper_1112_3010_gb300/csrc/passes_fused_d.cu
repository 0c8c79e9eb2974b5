// passes_fused_d.cu -- the double variants of the fused pass (run-time line
// length).
#include "passes_fused_kern.cuh"

namespace sdf {
SDF_INST_FUSED(double, 2, 0, 0)
SDF_INST_FUSED(double, 2, 1, 0)
SDF_INST_FUSED(double, 3, 0, 0)
SDF_INST_FUSED(double, 3, 1, 0)
}  // namespace sdf
