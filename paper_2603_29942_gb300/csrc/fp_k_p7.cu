// fp_k_p7.cu -- enumeration kernels for p = 7 (one per word count W), with
// pair-leaf passes.
#include "fp_kernel.cuh"
#include "fp_kernels.h"

namespace fpk {
const void *kernel_p7(int W) {
  switch (W) {
    case 1: return (const void *)bz_kernel<Fixed<7, 3, 1, LeafFilter<7, 3, 1>::kUnroll, true>>;
    case 2: return (const void *)bz_kernel<Fixed<7, 3, 2, LeafFilter<7, 3, 2>::kUnroll, true>>;
    case 3: return (const void *)bz_kernel<Fixed<7, 3, 3, LeafFilter<7, 3, 3>::kUnroll, true>>;
    case 4: return (const void *)bz_kernel<Fixed<7, 3, 4, LeafFilter<7, 3, 4>::kUnroll, true>>;
    default: return nullptr;
  }
}
const void *pair_table_kernel_p7(int W) {
  switch (W) {
    case 1: return (const void *)pair_table_kernel<7, 3, 1>;
    case 2: return (const void *)pair_table_kernel<7, 3, 2>;
    case 3: return (const void *)pair_table_kernel<7, 3, 3>;
    case 4: return (const void *)pair_table_kernel<7, 3, 4>;
    default: return nullptr;
  }
}
}  // namespace fpk
