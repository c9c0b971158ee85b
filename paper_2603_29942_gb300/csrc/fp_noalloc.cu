// fp_noalloc.cu -- fpcode_min_distance_noalloc: the certified-distance
// search without any device or pinned-host allocation.
//
// Who needs it: code that runs where cudaMalloc is not available or not
// allowed -- inside a host callback or a library that must not touch the
// CUDA allocator, or under a memory budget fixed at start-up -- can still
// certify a distance.  The search state, the pass schedule, the bit-sliced
// row multiples and the binomial table live in one file-scope device array
// (g_noalloc_scratch, kNoallocScratchBytes = 512 KiB) that every GPU loading
// this library holds until the process exits.
//
// Host code never uses the array's name as an address: on the first call
// on a device (with that device current) the address is fetched once with
// cudaGetSymbolAddress and cached per device; that first call should
// therefore come before any stream capture, and a cudaDeviceReset after it
// is not supported.  Every call shares the array
// and it keeps the last call's contents, so calls that overlap on the GPU
// (different streams or threads on the same device) race; a mutex
// serialises calls from this process on the host side.  The state words the
// kernel expects to start at zero are cleared by every call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fpcode.h"
#include "fp_driver.h"
#include "fp_internal.h"
#include "fp_kernel.cuh"
#include "fp_kernels.h"

namespace {

constexpr size_t kNoallocScratchBytes = 512 * 1024;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;               // one call at a time (they share the array)
bool g_noalloc_ready[kMaxDevices];
unsigned char *g_noalloc_ptr[kMaxDevices];  // device address of the array, per device

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

#define NA_CUDA(call)                                                           \
  do {                                                                          \
    cudaError_t _e = (call);                                                    \
    if (_e != cudaSuccess) {                                                    \
      fph::set_error(std::string(#call) + ": " + cudaGetErrorString(_e));       \
      return FPCODE_ECUDA;                                                      \
    }                                                                           \
  } while (0)

// Once per device, with the device current: fetch the array's device
// address and write the binomial table at its start.  The address and the
// table are kept for the life of the device's context: a cudaDeviceReset
// after the first call on that device is not supported (the table written
// once would be gone).
int noalloc_setup(int dev, unsigned char **out) {
  if (!g_noalloc_ready[dev]) {
    void *ptr = nullptr;
    NA_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    NA_CUDA(cudaMemcpy(ptr, &fph::binom(), sizeof(fpenum::Binom), cudaMemcpyHostToDevice));
    g_noalloc_ptr[dev] = static_cast<unsigned char *>(ptr);
    g_noalloc_ready[dev] = true;
  }
  *out = g_noalloc_ptr[dev];
  return FPCODE_OK;
}


}  // namespace

extern "C" int fpcode_min_distance_noalloc(int p, int n, int k, const uint8_t *G, void *stream, int *d,
                                           uint8_t *witness) {
  if (!d) return FPCODE_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  fpcode_opts o;
  fpcode_opts_default(&o);
  fph::Prepared P;
  int s = fph::prepare(p, n, k, G, o, &P);
  if (s) return s;

  // layout inside the array: [binom][CtlStatic][SlotDesc][passes, segments][table][state][dyn][aux][flags].
  // The pair-leaf plan (made below, for the grid) has at most one segment
  // per block (h, q) of each pass.
  size_t max_segs = 0;
  if (P.pair)
    for (const auto &pd : P.passes)
      if (pd.g >= 2) max_segs += pd.g == 2 ? 1 : (size_t)((P.p - 1) / 2) * (size_t)(P.k - 2 - (pd.g - 3));
  const size_t off_ctl = a256(sizeof(fpenum::Binom));
  const size_t off_slot = a256(off_ctl + sizeof(fpk::CtlStatic));
  const size_t off_pass = a256(off_slot + sizeof(fpk::SlotDesc));
  const size_t off_table =
      a256(off_pass + P.passes.size() * sizeof(fpk::PassDesc) + max_segs * sizeof(fpk::PairSeg));
  const size_t off_state = a256(off_table + P.table.size() * sizeof(uint32_t));
  const size_t dyn_bytes = a256(sizeof(fpk::SlotState) + sizeof(fpk::CtlDyn));
  const size_t off_aux = off_state + dyn_bytes;
  const size_t off_flags = off_aux + a256(sizeof(fpk::SlotAux));
  const size_t aux_bytes = off_flags - off_aux + 256;  // per-pass bookkeeping, then the slot's flag word
  if (off_aux + aux_bytes > kNoallocScratchBytes) {
    fph::set_error("fpcode_min_distance_noalloc: the code needs " + std::to_string(off_aux + aux_bytes) +
                   " bytes of device scratch, above the fixed 524288; use fpcode_min_distance");
    return FPCODE_EINVAL;
  }

  int dev = 0;
  NA_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    fph::set_error("fpcode_min_distance_noalloc: device index out of range");
    return FPCODE_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  unsigned char *base = nullptr;
  s = noalloc_setup(dev, &base);
  if (s) return s;

  const void *fn = fpd::kernel_for(P.variant);
  if (!fn) {
    fph::set_error("fpcode_min_distance_noalloc: no kernel for this (p, n - k)");
    return FPCODE_EINVAL;
  }
  const int smem = (int)(((std::max<size_t>(16, P.smem_bytes_per_set()) + 15) & ~(size_t)15) + fpk::kBinomBytes);
  int per_sm = 0, sms = 0;
  s = fpd::occupancy(fn, smem, P.opts.ctas_per_sm, &per_sm);  // sets the message when nothing fits
  if (s) return s;
  NA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int ctas = sms * per_sm;
  fph::plan_tasks(&P, ctas, 0, fph::kMinStepsSingle, true);
  if (P.segs.size() > max_segs) {
    fph::set_error("internal: pair-leaf plan larger than its bound");
    return FPCODE_EINVAL;
  }

  // host image of the static part (starting at off_ctl)
  std::vector<unsigned char> img(off_state - off_ctl, 0);
  fpk::CtlStatic cs{};
  cs.binom = reinterpret_cast<const fpenum::Binom *>(base);
  cs.aux = reinterpret_cast<fpk::SlotAux *>(base + off_aux);
  cs.slot_flags = reinterpret_cast<uint32_t *>(base + off_flags);
  cs.nslots = 1;
  cs.serve = 0;
  std::memcpy(&img[0], &cs, sizeof(cs));
  fpk::SlotDesc sd{};
  sd.p = P.p;
  sd.n = P.n;
  sd.k = P.k;
  sd.r = P.r;
  sd.W = P.W;
  sd.rwpad = P.rwpad;
  sd.m = P.m;
  sd.npasses = (int)P.passes.size();
  sd.variant = P.variant;
  sd.per_round_check = P.opts.per_round_check;
  sd.mid_pass_exit = P.opts.mid_pass_exit;
  sd.complete = P.complete;
  sd.seed_u = P.seed_u;
  sd.pair_sigp = P.pair ? P.pair_sigp : 0;
  sd.pair_quick_max = P.pair_quick_max;
  sd.nsegs = (int)P.segs.size();
  sd.table = reinterpret_cast<const uint32_t *>(base + off_table);
  sd.passes = reinterpret_cast<const fpk::PassDesc *>(base + off_pass);
  std::memcpy(&img[off_slot - off_ctl], &sd, sizeof(sd));
  std::memcpy(&img[off_pass - off_ctl], P.passes.data(), P.passes.size() * sizeof(fpk::PassDesc));
  if (!P.segs.empty())  // pair-leaf segments right after the passes
    std::memcpy(&img[off_pass - off_ctl + P.passes.size() * sizeof(fpk::PassDesc)], P.segs.data(),
                P.segs.size() * sizeof(fpk::PairSeg));
  std::memcpy(&img[off_table - off_ctl], P.table.data(), P.table.size() * sizeof(uint32_t));

  NA_CUDA(cudaMemcpyAsync(base + off_ctl, img.data(), img.size(), cudaMemcpyHostToDevice, st));
  NA_CUDA(cudaMemsetAsync(base + off_state, 0, dyn_bytes + aux_bytes, st));  // state starts at zero
  if (!P.passes.empty()) {
    const fpk::SlotDesc *slots = reinterpret_cast<const fpk::SlotDesc *>(base + off_slot);
    fpk::SlotState *states = reinterpret_cast<fpk::SlotState *>(base + off_state);
    const fpk::CtlStatic *ctl = reinterpret_cast<const fpk::CtlStatic *>(base + off_ctl);
    fpk::CtlDyn *dyn = reinterpret_cast<fpk::CtlDyn *>(base + off_state + dyn_bytes - sizeof(fpk::CtlDyn));
    fpk::KParams kp = fpd::kparams(o, 0);  // the same limits as the allocating entry point
    void *args[] = {(void *)&slots, (void *)&states, (void *)&ctl, (void *)&dyn, (void *)&kp};
    NA_CUDA(cudaLaunchKernel(fn, dim3(ctas), dim3(fpk::kThreads), args, (size_t)smem, st));
  }
  fpk::SlotState state{};
  NA_CUDA(cudaMemcpyAsync(&state, base + off_state, sizeof(state), cudaMemcpyDeviceToHost, st));
  NA_CUDA(cudaStreamSynchronize(st));

  fph::DeviceOutcome oc{};
  oc.best_key = ~(uint64_t)state.best_key;
  oc.enumerated = state.finished ? state.entered : state.enumerated;
  if (P.passes.empty()) {
    oc.best_key = fpk::kNoKey;
    oc.status = FPCODE_EBUDGET;
    oc.stop_pass = -1;
  } else if (state.finished) {
    oc.status = state.status & 0xFF;
    oc.stop_pass = state.stop_pass;
  } else {
    oc.status = -1;
    oc.stop_pass = (int)((state.word >> 40) & 0xFF) - 1;
  }
  fpcode_result res;
  s = fph::decode_result(P, oc, &res, witness);
  if (s) return s;
  *d = res.d;
  return FPCODE_OK;
}
