// fp_k_generic.cu -- enumeration kernels for the other odd primes p < 256
// (runtime p, r = 4..8 bits per symbol, W = 1..4 words per slice).
#include "fp_kernel.cuh"
#include "fp_kernels.h"

namespace fpk {
template <int R>
static const void *pick(int W) {
  switch (W) {
    case 1: return (const void *)bz_kernel<Fixed<0, R, 1>>;
    case 2: return (const void *)bz_kernel<Fixed<0, R, 2>>;
    case 3: return (const void *)bz_kernel<Fixed<0, R, 3>>;
    case 4: return (const void *)bz_kernel<Fixed<0, R, 4>>;
    default: return nullptr;
  }
}
const void *kernel_generic(int r, int W) {
  switch (r) {
    case 4: return pick<4>(W);
    case 5: return pick<5>(W);
    case 6: return pick<6>(W);
    case 7: return pick<7>(W);
    case 8: return pick<8>(W);
    default: return nullptr;
  }
}
}  // namespace fpk
