// fp_k_multi.cu -- the batched kernel: one persistent launch over codes
// with p in {3, 5, 7}, dispatching the variant per task.
#include "fp_kernel.cuh"
#include "fp_kernels.h"

namespace fpk {
const void *kernel_multi357() { return (const void *)bz_kernel<Multi357>; }
}  // namespace fpk
