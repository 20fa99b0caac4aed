// Step-kernel instantiations for FP64 field stored as float pairs (float-float kernel).
#include "lcs_step_kernel.cuh"

namespace lcs {
LCS_STEP_KIND_INSTANTIATE(FK_DF)
}  // namespace lcs
