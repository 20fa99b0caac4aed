// Step-kernel instantiations for the all-FP64 kernel.
#include "lcs_step_kernel.cuh"

namespace lcs {
LCS_STEP_KIND_INSTANTIATE(FK_F64)
}  // namespace lcs
