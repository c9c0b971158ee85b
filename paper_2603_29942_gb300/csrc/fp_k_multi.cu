// fp_k_multi.cu -- the batched kernel for codes with p in {3, 5, 7} and
// n - k <= 64 (one or two words per slice), dispatching the variant per task.
#include "fp_kernel.cuh"
#include "fp_kernels.h"

namespace fpk {
const void *kernel_multi357_narrow() { return (const void *)bz_kernel<Multi357<2>>; }
}  // namespace fpk
