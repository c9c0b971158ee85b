// fp_k_mersenne.cu -- enumeration kernels for the Mersenne primes p = 31
// (r = 5) and p = 127 (r = 7): the exact add in its end-around-carry form,
// the leaf filter by isometric subtraction, W = 1..4 words per slice.
#include "fp_kernel.cuh"
#include "fp_kernels.h"

namespace fpk {
template <int P, int R>
static const void *pick_m(int W) {
  switch (W) {
    case 1: return (const void *)bz_kernel<Fixed<P, R, 1>>;
    case 2: return (const void *)bz_kernel<Fixed<P, R, 2>>;
    case 3: return (const void *)bz_kernel<Fixed<P, R, 3>>;
    case 4: return (const void *)bz_kernel<Fixed<P, R, 4>>;
    default: return nullptr;
  }
}
const void *kernel_mersenne(int p, int W) {
  return p == 31 ? pick_m<31, 5>(W) : p == 127 ? pick_m<127, 7>(W) : nullptr;
}
}  // namespace fpk
