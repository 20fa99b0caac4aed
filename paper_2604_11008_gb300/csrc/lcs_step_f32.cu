// Step-kernel instantiations for FP32 field storage.
#include "lcs_step_kernel.cuh"

namespace lcs {
LCS_STEP_KIND_INSTANTIATE(FK_F32)
}  // namespace lcs
