// Step-kernel instantiations for BF16 field storage.
#include "lcs_step_kernel.cuh"

namespace lcs {
LCS_STEP_KIND_INSTANTIATE(FK_BF16)
}  // namespace lcs
