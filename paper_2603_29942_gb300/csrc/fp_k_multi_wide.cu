// fp_k_multi_wide.cu -- the batched kernel for codes with p in {3, 5, 7} and
// any n - k <= 128, dispatching the variant per task.
#include "fp_kernel.cuh"
#include "fp_kernels.h"

namespace fpk {
const void *kernel_multi357_wide() { return (const void *)bz_kernel<Multi357<4>>; }
}  // namespace fpk
