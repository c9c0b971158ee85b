// fp_k_p3.cu -- enumeration kernels for p = 3 (one per word count W), with
// pair-leaf passes.
#include "fp_kernel.cuh"
#include "fp_kernels.h"

namespace fpk {
const void *kernel_p3(int W) {
  switch (W) {
    case 1: return (const void *)bz_kernel<Fixed<3, 2, 1, LeafFilter<3, 2, 1>::kUnroll, true>>;
    case 2: return (const void *)bz_kernel<Fixed<3, 2, 2, LeafFilter<3, 2, 2>::kUnroll, true>>;
    case 3: return (const void *)bz_kernel<Fixed<3, 2, 3, LeafFilter<3, 2, 3>::kUnroll, true>>;
    case 4: return (const void *)bz_kernel<Fixed<3, 2, 4, LeafFilter<3, 2, 4>::kUnroll, true>>;
    default: return nullptr;
  }
}
const void *pair_table_kernel_p3(int W) {
  switch (W) {
    case 1: return (const void *)pair_table_kernel<3, 2, 1>;
    case 2: return (const void *)pair_table_kernel<3, 2, 2>;
    case 3: return (const void *)pair_table_kernel<3, 2, 3>;
    case 4: return (const void *)pair_table_kernel<3, 2, 4>;
    default: return nullptr;
  }
}
}  // namespace fpk
