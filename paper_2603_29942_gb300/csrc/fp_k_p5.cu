// fp_k_p5.cu -- enumeration kernels for p = 5 (one per word count W).
#include "fp_kernel.cuh"
#include "fp_kernels.h"

namespace fpk {
const void *kernel_p5(int W) {
  switch (W) {
    case 1: return (const void *)bz_kernel<Fixed<5, 3, 1>>;
    case 2: return (const void *)bz_kernel<Fixed<5, 3, 2>>;
    case 3: return (const void *)bz_kernel<Fixed<5, 3, 3>>;
    case 4: return (const void *)bz_kernel<Fixed<5, 3, 4>>;
    default: return nullptr;
  }
}
}  // namespace fpk
