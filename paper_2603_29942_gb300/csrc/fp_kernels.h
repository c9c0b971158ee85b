// fp_kernels.h -- host stubs of the enumeration kernel instantiations.
#pragma once

namespace fpk {
// Kernel for one (prime class, words) variant; nullptr if not built.
const void *kernel_p3(int W);
const void *kernel_p5(int W);
const void *kernel_p7(int W);
const void *kernel_generic(int r, int W);
const void *kernel_mersenne(int p, int W);  // p = 31 or 127
// Test hook: the pair-table builder of the p = 3 / 7 kernels, alone.
const void *pair_table_kernel_p3(int W);
const void *pair_table_kernel_p7(int W);
// Batched kernel dispatching per task over p in {3, 5, 7}, W in 1..4.
const void *kernel_multi357_narrow();  // W <= 2
const void *kernel_multi357_wide();    // W <= 4
inline const void *kernel_multi357(int W) { return W <= 2 ? kernel_multi357_narrow() : kernel_multi357_wide(); }
}  // namespace fpk
