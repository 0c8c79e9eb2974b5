// adjoint.cu -- placeholder translation unit (filled in with the adjoint).
#include "sdf_internal.cuh"
