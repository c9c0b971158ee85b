// fp_driver.h -- host-side driver helpers shared by the launch paths
// (single codes, batches, serving).
#pragma once
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/fpcode.h"
#include "fp_enum.cuh"
#include "fp_kernel.cuh"

namespace fpd {

// Per-device context: SM count, the binomial table, the shared workspace.
struct DevCtx {
  bool ready = false;
  int sms = 0;
  fpenum::Binom *binom = nullptr;  // device copy
  std::mutex ws_mu;                // guards the workspace below
  char *ws = nullptr;
  size_t ws_bytes = 0;
  char *ws_pinned = nullptr;
  size_t ws_pinned_bytes = 0;
  void *ev0 = nullptr, *ev1 = nullptr;  // cudaEvent_t around the kernel of a workspace search
};

// Context of the current device (created on first use).
int get_ctx(DevCtx **out);
// Kernel of one (prime class, words) variant.
const void *kernel_for(int variant);
// CTAs per SM for `fn` with `smem` bytes of dynamic shared memory.
int occupancy(const void *fn, int smem, int override_per_sm, int *per_sm);
// Per-launch limits from the options.
fpk::KParams kparams(const fpcode_opts &o, int serve);

}  // namespace fpd
