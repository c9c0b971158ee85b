// fp_api.cu -- the C ABI of libfpcode on top of the persistent enumeration
// kernel: device context, uploads, launches, read-back, batching, and the
// device self-test and integer-rate microbenchmark entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <thread>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/fpcode.h"
#include "../../include/fpcode_testing.h"
#include "fp_internal.h"
#include "fp_kernel.cuh"
#include "fp_kernels.h"
#include "fp_driver.h"

using fpk::CtlDyn;
using fpk::CtlStatic;
using fpk::KParams;
using fpk::PassDesc;
using fpk::SlotDesc;
using fpk::SlotState;

using fpd::DevCtx;

#define FP_CUDA(call)                                                                           \
  do {                                                                                           \
    cudaError_t _e = (call);                                                                     \
    if (_e != cudaSuccess) {                                                                     \
      fph::set_error(std::string(#call) + ": " + cudaGetErrorString(_e));                        \
      return FPCODE_ECUDA;                                                                       \
    }                                                                                            \
  } while (0)

namespace fph {

int device_identity(int *sms, char *name, size_t name_len) {
  int dev = 0;
  FP_CUDA(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  FP_CUDA(cudaGetDeviceProperties(&prop, dev));
  *sms = prop.multiProcessorCount;
  std::snprintf(name, name_len, "%s", prop.name);
  return FPCODE_OK;
}

}  // namespace fph

namespace fpd {

std::mutex g_ctx_mu;
DevCtx g_ctx[64];

int get_ctx(DevCtx **out) {
  int dev = 0;
  FP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    fph::set_error("device index out of range");
    return FPCODE_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_ctx_mu);
  DevCtx &c = g_ctx[dev];
  if (!c.ready) {
    FP_CUDA(cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev));
    FP_CUDA(cudaMalloc(&c.binom, sizeof(fpenum::Binom)));
    FP_CUDA(cudaMemcpy(c.binom, &fph::binom(), sizeof(fpenum::Binom), cudaMemcpyHostToDevice));
    c.ready = true;
  }
  *out = &c;
  return FPCODE_OK;
}

// Grow-only device + pinned buffers (caller holds ws_mu).
int ws_reserve(DevCtx &c, size_t dev_bytes, size_t pinned_bytes) {
  if (dev_bytes > c.ws_bytes) {
    if (c.ws) cudaFree(c.ws);
    c.ws = nullptr;
    c.ws_bytes = 0;
    size_t want = std::max(dev_bytes, (size_t)1 << 20);
    FP_CUDA(cudaMalloc(&c.ws, want));
    c.ws_bytes = want;
  }
  if (pinned_bytes > c.ws_pinned_bytes) {
    if (c.ws_pinned) cudaFreeHost(c.ws_pinned);
    c.ws_pinned = nullptr;
    c.ws_pinned_bytes = 0;
    size_t want = std::max(pinned_bytes, (size_t)1 << 20);
    FP_CUDA(cudaHostAlloc(&c.ws_pinned, want, cudaHostAllocMapped));  // mapped: kernels write outcomes into it
    c.ws_pinned_bytes = want;
  }
  return FPCODE_OK;
}

const void *kernel_for(int variant) {
  const int cls = variant / 4, W = variant % 4 + 1;
  switch (cls) {
    case 0: return fpk::kernel_p3(W);
    case 1: return fpk::kernel_p5(W);
    case 2: return fpk::kernel_p7(W);
    case 8: return fpk::kernel_mersenne(31, W);
    case 9: return fpk::kernel_mersenne(127, W);
    default: return fpk::kernel_generic(cls - 3 + 4, W);
  }
}

// CTAs per SM for a kernel with `smem` bytes of dynamic shared memory.
int occupancy(const void *fn, int smem, int override_per_sm, int *per_sm) {
  cudaFuncAttributes fa{};
  FP_CUDA(cudaFuncGetAttributes(&fa, fn));
  // dynamic and static shared memory together past 48 KiB need the opt-in
  if ((size_t)smem + fa.sharedSizeBytes > 48 * 1024)
    FP_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int n = 0;
  FP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, fpk::kThreads, (size_t)smem));
  if (n < 1) {
    fph::set_error("kernel cannot be resident (shared memory or registers)");
    return FPCODE_EINVAL;
  }
  *per_sm = override_per_sm > 0 ? std::min(override_per_sm, n) : n;
  return FPCODE_OK;
}

KParams kparams(const fpcode_opts &o, int serve) {
  KParams kp{};
  const double wait = o.wait_limit_s > 0 ? o.wait_limit_s : 10.0;
  kp.wait_limit_ns = (unsigned long long)(wait * 1e9);
  kp.timeout_ns = o.timeout_s > 0 ? (unsigned long long)(o.timeout_s * 1e9) : 0ull;
  kp.idle_limit_ns = serve ? 20000000ull : 0ull;
  kp.mid_pass = o.mid_pass_exit ? 1 : 0;
  kp.lookahead = o.lookahead ? 1 : 0;
  return kp;
}

}  // namespace fpd

namespace {

using fpd::get_ctx;
using fpd::kernel_for;
using fpd::kparams;
using fpd::occupancy;
using fpd::ws_reserve;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// ---------------------------------------------------------------------------
// Layout of a launch over several codes:
//   static  [CtlStatic][SlotDesc x ns][PassDesc ...][tables ...]
//   dynamic [SlotState x ns][CtlDyn]
// ---------------------------------------------------------------------------
struct Layout {
  size_t off_ctl = 0, off_slots = 0, off_passes = 0, off_tables = 0, static_bytes = 0;
  size_t off_states = 0, dyn_bytes = 0, off_aux = 0, aux_bytes = 0, off_flags = 0, off_times = 0, total = 0;
  std::vector<size_t> pass_off, table_off;
};

Layout make_layout(const std::vector<const fph::Prepared *> &codes) {
  Layout L;
  const size_t ns = codes.size();
  size_t o = 0;
  L.off_ctl = o;
  o = align256(o + sizeof(CtlStatic));
  L.off_slots = o;
  o = align256(o + ns * sizeof(SlotDesc));
  L.off_passes = o;
  for (auto *P : codes) {  // each code's passes, then its pair-leaf segments (read as passes + npasses)
    L.pass_off.push_back(o);
    o = align256(o + P->passes.size() * sizeof(PassDesc) + P->segs.size() * sizeof(fpk::PairSeg));
  }
  L.off_tables = o;
  for (auto *P : codes) {
    L.table_off.push_back(o);
    o = align256(o + P->table.size() * sizeof(uint32_t));
  }
  L.static_bytes = o;
  L.off_states = o;
  L.dyn_bytes = align256(ns * sizeof(SlotState) + sizeof(CtlDyn));  // read back after a search
  L.off_aux = o + L.dyn_bytes;
  L.off_flags = L.off_aux + align256(ns * sizeof(fpk::SlotAux));
  L.aux_bytes = L.off_flags - L.off_aux + align256((ns + 3) / 4 * 16);  // aux and flags: zeroed, never read back
  L.off_times = L.off_aux + L.aux_bytes;  // per-pass end times of a single code (diagnostics)
  L.total = L.off_times + (fpk::kMaxPasses + 1) * sizeof(unsigned long long);
  return L;
}

// Write the static part for `codes` into host staging `h` (device base `d`).
// outcome: for one code, the device address of a host-mapped copy of its
// dynamic state ([SlotState][CtlDyn], L.dyn_bytes): the kernel's last CTA
// writes it there and zeroes the state for the next launch (else null: the
// caller zeroes the state before and copies it back after each launch).
void fill_static(const Layout &L, const std::vector<const fph::Prepared *> &codes, const DevCtx &c, char *h,
                 char *d, int serve, char *outcome = nullptr) {
  CtlStatic cs{};
  cs.binom = c.binom;
  cs.aux = reinterpret_cast<fpk::SlotAux *>(d + L.off_aux);
  cs.slot_flags = reinterpret_cast<uint32_t *>(d + L.off_flags);
  cs.nslots = (int)codes.size();
  cs.serve = serve;
  if (outcome && codes.size() == 1 && !serve) {
    cs.outcome = outcome;
    cs.dyn_bytes = (uint32_t)L.dyn_bytes;
    cs.clean_bytes = (uint32_t)(L.off_times - L.off_states);
  }
  std::memcpy(h + L.off_ctl, &cs, sizeof(cs));
  for (size_t i = 0; i < codes.size(); ++i) {
    const fph::Prepared &P = *codes[i];
    SlotDesc sd{};
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
    sd.table = reinterpret_cast<const uint32_t *>(d + L.table_off[i]);
    sd.passes = reinterpret_cast<const PassDesc *>(d + L.pass_off[i]);
    std::memcpy(h + L.off_slots + i * sizeof(SlotDesc), &sd, sizeof(sd));
    std::memcpy(h + L.pass_off[i], P.passes.data(), P.passes.size() * sizeof(PassDesc));
    if (!P.segs.empty())
      std::memcpy(h + L.pass_off[i] + P.passes.size() * sizeof(PassDesc), P.segs.data(),
                  P.segs.size() * sizeof(fpk::PairSeg));
    std::memcpy(h + L.table_off[i], P.table.data(), P.table.size() * sizeof(uint32_t));
  }
}

fph::DeviceOutcome outcome_of(const SlotState &s, const CtlDyn &dyn) {
  fph::DeviceOutcome o{};
  o.best_key = ~(uint64_t)s.best_key;
  o.enumerated = s.finished ? s.entered : s.enumerated;
  if (s.finished) {
    o.status = s.status & 0xFF;
    o.stop_pass = s.stop_pass;
  } else {
    o.status = -1;  // timed out or a wait gave up
    o.stop_pass = (int)((s.word >> 40) & 0xFF) - 1;
  }
  (void)dyn;
  return o;
}

int launch(const void *fn, int ctas, int smem, cudaStream_t st, char *d, const Layout &L, const KParams &kp) {
  const SlotDesc *slots = reinterpret_cast<const SlotDesc *>(d + L.off_slots);
  SlotState *states = reinterpret_cast<SlotState *>(d + L.off_states);
  const CtlStatic *ctl = reinterpret_cast<const CtlStatic *>(d + L.off_ctl);
  CtlDyn *dyn = reinterpret_cast<CtlDyn *>(d + L.off_states + L.dyn_bytes - sizeof(CtlDyn));
  KParams kpv = kp;
  void *args[] = {(void *)&slots, (void *)&states, (void *)&ctl, (void *)&dyn, (void *)&kpv};
  FP_CUDA(cudaLaunchKernel(fn, dim3(ctas), dim3(fpk::kThreads), args, (size_t)smem, st));
  return FPCODE_OK;
}

// Dynamic shared memory of a launch: binomial columns + the largest table
// of one information set.
int smem_for(const std::vector<const fph::Prepared *> &codes) {
  size_t s = 16;
  for (auto *P : codes) s = std::max(s, P->smem_bytes_per_set());
  return (int)(((s + 15) & ~(size_t)15) + fpk::kBinomBytes);
}

// with_state: the host image also holds the first state (zeroed
// bookkeeping, the bound in the best key) and one copy takes both, so the
// next search needs no reset of its own.
// Grid and task plan of one code (before its layout: the plan's pair-leaf
// segments are part of the static image).
int plan_one(fpcode_prepared *prep, const DevCtx &c) {
  fph::Prepared &P = prep->host;
  const void *fn = kernel_for(P.variant);
  if (!fn) {
    fph::set_error("no kernel for this (p, n - k)");
    return FPCODE_EINVAL;
  }
  prep->smem = smem_for({&P});
  int per_sm = 0;
  int s = occupancy(fn, prep->smem, P.opts.ctas_per_sm, &per_sm);
  if (s) return s;
  prep->ctas = c.sms * per_sm;
  fph::plan_tasks(&P, prep->ctas, P.opts.prefixes_per_lane, P.opts.min_steps > 0 ? P.opts.min_steps : fph::kMinStepsSingle,
                  true);
  if (prep->slice_hi > 0) {  // a slice of the one pass: its tasks under the same plan
    fpk::PassDesc &d = P.passes[0];
    const uint64_t hi = std::min<uint64_t>(prep->slice_hi, d.ntasks);
    const uint64_t lo = std::min<uint64_t>(prep->slice_lo, hi);
    d.task_off = (uint32_t)lo;
    d.ntasks = (uint32_t)(hi - lo);
  }
  return FPCODE_OK;
}

// Upload one planned code (plan_one) into device buffer `d` via pinned
// staging `h`.
// readback: the host-mapped buffer the kernel copies the outcome into.
int upload_one(fpcode_prepared *prep, cudaStream_t st, DevCtx &c, char *d, char *h, char *readback,
               bool with_state = false) {
  fph::Prepared &P = prep->host;
  Layout L = make_layout({&P});
  prep->off_ctl = L.off_ctl;
  prep->off_slot = L.off_slots;
  prep->off_pass = L.off_passes;
  prep->off_table = L.off_tables;
  prep->off_state = L.off_states;
  prep->dyn_bytes = L.dyn_bytes;
  prep->dev_bytes = L.total;
  char *outcome = nullptr;
  if (readback && cudaHostGetDevicePointer((void **)&outcome, readback, 0) != cudaSuccess) {
    (void)cudaGetLastError();  // not mapped: the state is reset and copied back per search instead
    outcome = nullptr;
  }
  prep->mapped_outcome = outcome != nullptr;
  fill_static(L, {&P}, c, h, d, 0, outcome);
  SlotDesc *sd = reinterpret_cast<SlotDesc *>(h + L.off_slots);
  sd->pass_times = reinterpret_cast<unsigned long long *>(d + L.off_times);
  size_t bytes = L.static_bytes;
  prep->state_clean = false;
  if (with_state) {
    std::memset(h + L.off_states, 0, L.off_times - L.off_states);
    bytes = L.off_times;
    prep->state_clean = true;
  }
  FP_CUDA(cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, st));
  return FPCODE_OK;
}

int enqueue_one(fpcode_prepared *prep, cudaStream_t st, const fpcode_opts &o) {
  fph::Prepared &P = prep->host;
  Layout L = make_layout({&P});
  // the state is zero after the upload that wrote it and after every
  // search whose kernel cleaned up behind itself (mapped outcome); else reset it
  const bool clean = prep->state_clean;
  prep->state_clean = false;  // until this search has finished
  if (!clean) FP_CUDA(cudaMemsetAsync(prep->dev + L.off_states, 0, L.dyn_bytes + L.aux_bytes, st));
  const bool resumed = prep->resume_from > 0;
  // the first state's values, staged in pinned memory (a copy from pageable
  // memory would wait for the stream)
  struct Stage {
    unsigned long long word, key, bound;
    int32_t frontier, useq;
  };
  Stage *sg = reinterpret_cast<Stage *>(prep->pinned + prep->stage_off);
  static_assert(sizeof(Stage) <= 64, "staging block");
  char *stp = prep->dev + L.off_states;
  if (resumed) {  // continue after a checkpoint: next task, frontier, bound
    const fpk::PassDesc &d = P.passes[prep->resume_from];
    sg->word = (unsigned long long)d.task_base;
    sg->key = prep->resume_key == fpk::kNoKey ? 0ull : ~prep->resume_key;
    sg->frontier = prep->resume_from;
    sg->useq = prep->resume_key == fpk::kNoKey ? 0 : (int32_t)fpk::key_weight(prep->resume_key);
    FP_CUDA(cudaMemcpyAsync(stp + offsetof(SlotState, word), &sg->word, 8, cudaMemcpyHostToDevice, st));
    FP_CUDA(cudaMemcpyAsync(stp + offsetof(SlotState, best_key), &sg->key, 8, cudaMemcpyHostToDevice, st));
    FP_CUDA(cudaMemcpyAsync(stp + offsetof(SlotState, frontier), &sg->frontier, 4, cudaMemcpyHostToDevice, st));
    FP_CUDA(cudaMemcpyAsync(prep->dev + L.off_aux + offsetof(fpk::SlotAux, useq_after) +
                                (size_t)(prep->resume_from - 1) * sizeof(int32_t),
                            &sg->useq, 4, cudaMemcpyHostToDevice, st));
    prep->resume_from = 0;  // one search
  }
  // the probe's bound as a key past every real one (pass 255), stored inverted
  if (prep->init_u > 0) {
    sg->bound = ~fph::bound_key((uint32_t)prep->init_u);
    FP_CUDA(cudaMemcpyAsync(stp + offsetof(SlotState, best_key), &sg->bound, 8, cudaMemcpyHostToDevice, st));
  }
  if (!P.passes.empty()) {
    FP_CUDA(cudaEventRecord((cudaEvent_t)prep->ev0, st));
    int s = launch(kernel_for(P.variant), prep->ctas, prep->smem, st, prep->dev, L, kparams(o, 0));
    if (s) return s;
    FP_CUDA(cudaEventRecord((cudaEvent_t)prep->ev1, st));
  }
  if (!prep->mapped_outcome || P.passes.empty())
    FP_CUDA(cudaMemcpyAsync(prep->pinned, prep->dev + L.off_states, L.dyn_bytes, cudaMemcpyDeviceToHost, st));
  prep->run_opts = o;
  return FPCODE_OK;
}

int finish_one(fpcode_prepared *prep, cudaStream_t st, fpcode_result *res, uint8_t *witness) {
  FP_CUDA(cudaStreamSynchronize(st));
  const fph::Prepared &P = prep->host;
  prep->state_clean = prep->mapped_outcome && !P.passes.empty();  // the kernel's last CTA zeroed it
  if (P.passes.empty()) {  // budget below the first pass
    fph::DeviceOutcome o{fpk::kNoKey, 0, FPCODE_EBUDGET, -1};
    return fph::decode_result(P, o, res, witness);
  }
  SlotState s;
  CtlDyn dyn;
  std::memcpy(&s, prep->pinned, sizeof(s));
  std::memcpy(&dyn, prep->pinned + prep->dyn_bytes - sizeof(CtlDyn), sizeof(dyn));
  const fph::DeviceOutcome oc = outcome_of(s, dyn);
  prep->last_status = oc.status;
  prep->last_stop = oc.stop_pass;
  prep->last_key = oc.best_key;
  int rc = fph::decode_result(P, oc, res, witness);
  float ms = 0;
  if (cudaEventElapsedTime(&ms, (cudaEvent_t)prep->ev0, (cudaEvent_t)prep->ev1) == cudaSuccess) res->t_kernel_ms = ms;
  return rc;
}

int ensure_events(fpcode_prepared *prep) {
  if (!prep->ev0) {
    cudaEvent_t a, b;
    FP_CUDA(cudaEventCreate(&a));
    FP_CUDA(cudaEventCreate(&b));
    prep->ev0 = a;
    prep->ev1 = b;
  }
  return FPCODE_OK;
}

double ms_since(std::chrono::steady_clock::time_point t) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t).count();
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void fpcode_opts_default(fpcode_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->per_round_check = 0;
  o->defer = 1;
  o->mid_pass_exit = 1;
  o->lookahead = 1;
  o->wait_limit_s = 10.0;
  o->pair_leaves = 2;
}

const char *fpcode_last_error(void) { return fph::last_error(); }

int fpcode_prepare(int p, int n, int k, const uint8_t *G, const fpcode_opts *opts, fpcode_prepared **out) {
  if (!out) return FPCODE_EINVAL;
  *out = nullptr;
  fpcode_opts o;
  fpcode_opts_default(&o);
  if (opts) o = *opts;
  fpcode_prepared *prep = new (std::nothrow) fpcode_prepared();
  if (!prep) return FPCODE_ENOMEM;
  int s = fph::prepare(p, n, k, G, o, &prep->host);
  if (s) {
    delete prep;
    return s;
  }
  *out = prep;
  return FPCODE_OK;
}

int fpcode_prepared_single_pass(const fpcode_prepared *src, int pass, int u_init, fpcode_prepared **out) {
  if (!out) return FPCODE_EINVAL;
  *out = nullptr;
  if (!src || pass < 0 || pass >= (int)src->host.passes.size() || u_init < 0 || u_init > fpk::kMaxN) {
    fph::set_error("fpcode_prepared_single_pass: no such pass, or a bound outside 0..255");
    return FPCODE_EINVAL;
  }
  fpcode_prepared *prep = new (std::nothrow) fpcode_prepared();
  if (!prep) return FPCODE_ENOMEM;
  prep->host = src->host;
  fpk::PassDesc d = src->host.passes[pass];
  d.L_before = 0;  // no bound ever reaches U: every task runs, nothing is certified
  d.L_after = 0;
  d.round_end = 1;
  d.task_base = 0;
  prep->host.passes.assign(1, d);
  prep->host.complete = 0;
  prep->host.seed_u = 0;  // the probe's bound is u_init
  prep->init_u = u_init;
  *out = prep;
  return FPCODE_OK;
}

int fpcode_prepared_pass_slice(const fpcode_prepared *src, int pass, uint64_t task_lo, uint64_t task_hi, int u_init,
                               fpcode_prepared **out) {
  if (!out) return FPCODE_EINVAL;
  *out = nullptr;
  if (!src || task_hi <= task_lo) {
    fph::set_error("fpcode_prepared_pass_slice: need a prepared code and task_lo < task_hi");
    return FPCODE_EINVAL;
  }
  fpcode_prepared *prep = nullptr;
  int s = fpcode_prepared_single_pass(src, pass, u_init, &prep);
  if (s) return s;
  prep->slice_lo = task_lo;
  prep->slice_hi = task_hi;
  // the slice's tasks are those of the pass in the source's plan: the share
  // of a pass depends on whether passes follow it in the source schedule
  prep->host.opts.task_share = fph::task_share_of(src->host.opts, pass + 1 == (int)src->host.passes.size());
  *out = prep;
  return FPCODE_OK;
}

int fpcode_prepared_set_bound(fpcode_prepared *slice, int u_init) {
  if (!slice || slice->slice_hi == 0 || u_init < 0 || u_init > fpk::kMaxN) {
    fph::set_error("fpcode_prepared_set_bound: need a pass slice and a bound in 0..255");
    return FPCODE_EINVAL;
  }
  slice->init_u = u_init;
  return FPCODE_OK;
}

void fpcode_prepared_free(fpcode_prepared *prep) {
  if (!prep) return;
  if (!prep->external) {
    if (prep->dev) cudaFree(prep->dev);
    if (prep->pinned) cudaFreeHost(prep->pinned);
  }
  if (prep->ev0) cudaEventDestroy((cudaEvent_t)prep->ev0);
  if (prep->ev1) cudaEventDestroy((cudaEvent_t)prep->ev1);
  delete prep;
}

int fpcode_prepared_upload(fpcode_prepared *prep, void *stream) {
  if (!prep) return FPCODE_EINVAL;
  if (prep->uploaded) return FPCODE_OK;
  cudaStream_t st = (cudaStream_t)stream;
  DevCtx *c;
  int s = get_ctx(&c);
  if (s) return s;
  s = ensure_events(prep);
  if (s) return s;
  FP_CUDA(cudaGetDevice(&prep->device));
  s = plan_one(prep, *c);
  if (s) return s;
  Layout L = make_layout({&prep->host});
  FP_CUDA(cudaMalloc(&prep->dev, L.total));
  prep->stage_off = align256(std::max(L.static_bytes, L.dyn_bytes));
  FP_CUDA(cudaHostAlloc(&prep->pinned, prep->stage_off + 64, cudaHostAllocMapped));  // mapped: the outcome lands here
  s = upload_one(prep, st, *c, prep->dev, prep->pinned, prep->pinned);
  if (s) return s;
  FP_CUDA(cudaStreamSynchronize(st));
  prep->uploaded = true;
  return FPCODE_OK;
}

int fpcode_search_enqueue(fpcode_prepared *prep, void *stream, const fpcode_opts *opts) {
  if (!prep || !prep->uploaded) {
    fph::set_error("fpcode_search_enqueue: not uploaded");
    return FPCODE_EINVAL;
  }
  return enqueue_one(prep, (cudaStream_t)stream, opts ? *opts : prep->host.opts);
}

int fpcode_search_checkpoint(const fpcode_prepared *prep, fpcode_checkpoint *out) {
  if (!prep || !out) return FPCODE_EINVAL;
  const fph::Prepared &P = prep->host;
  // a search that ran every pass of its schedule and stopped at the budget
  if (prep->last_status != FPCODE_EBUDGET || prep->last_stop + 1 != (int)P.passes.size() || P.complete) {
    fph::set_error("fpcode_search_checkpoint: the last search did not stop at its budget after its last pass");
    return FPCODE_EINVAL;
  }
  std::memset(out, 0, sizeof(*out));
  out->p = P.p;
  out->n = P.n;
  out->k = P.k;
  out->passes_done = prep->last_stop + 1;
  out->best_key = prep->last_key;
  out->code_hash = P.code_hash;
  return FPCODE_OK;
}

int fpcode_search_resume(fpcode_prepared *prep, const fpcode_checkpoint *ck, void *stream, const fpcode_opts *opts) {
  if (!prep || !ck) return FPCODE_EINVAL;
  const fph::Prepared &P = prep->host;
  if (ck->p != P.p || ck->n != P.n || ck->k != P.k || ck->code_hash != P.code_hash) {
    fph::set_error("fpcode_search_resume: the checkpoint is of another code or other schedule options");
    return FPCODE_EINVAL;
  }
  if (ck->passes_done < 1 || ck->passes_done >= (int)P.passes.size()) {
    fph::set_error("fpcode_search_resume: the schedule has no pass after the checkpoint (raise the budget)");
    return FPCODE_EINVAL;
  }
  if (ck->best_key != fpk::kNoKey && (int)fpk::key_pass(ck->best_key) >= ck->passes_done) {
    fph::set_error("fpcode_search_resume: the checkpoint's best key is not of a completed pass");
    return FPCODE_EINVAL;
  }
  if (!prep->uploaded) {
    fph::set_error("fpcode_search_resume: not uploaded");
    return FPCODE_EINVAL;
  }
  prep->resume_from = ck->passes_done;
  prep->resume_key = ck->best_key;
  return enqueue_one(prep, (cudaStream_t)stream, opts ? *opts : P.opts);
}

int fpcode_search_finish(fpcode_prepared *prep, void *stream, fpcode_result *res, uint8_t *witness) {
  if (!prep || !res) return FPCODE_EINVAL;
  return finish_one(prep, (cudaStream_t)stream, res, witness);
}

int fpcode_min_distance_ex(fpcode_prepared *prep, void *stream, const fpcode_opts *opts, fpcode_result *res,
                           uint8_t *witness) {
  if (!prep || !res) return FPCODE_EINVAL;
  auto t0 = std::chrono::steady_clock::now();
  int s = fpcode_prepared_upload(prep, stream);
  if (s) return s;
  s = fpcode_search_enqueue(prep, stream, opts);
  if (s) return s;
  s = fpcode_search_finish(prep, stream, res, witness);
  res->t_total_ms = ms_since(t0);
  return s;
}

int fpcode_min_distance(int p, int n, int k, const uint8_t *G, void *stream, int *d, uint8_t *witness) {
  if (!d) return FPCODE_EINVAL;
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = (cudaStream_t)stream;
  fpcode_opts o;
  fpcode_opts_default(&o);
  fpcode_prepared prep;
  int s = fph::prepare(p, n, k, G, o, &prep.host);
  if (s) return s;
  DevCtx *c;
  s = get_ctx(&c);
  if (s) return s;
  std::lock_guard<std::mutex> lk(c->ws_mu);
  s = plan_one(&prep, *c);
  if (s) return s;
  Layout L = make_layout({&prep.host});
  // pinned: [static image and first state][read-back][staging], so nothing
  // waits between the upload and the launch
  const size_t rb_off = align256(L.off_times), stage_off = rb_off + align256(L.dyn_bytes);
  s = ws_reserve(*c, L.total, stage_off + 64);
  if (s) return s;
  if (!c->ev0) {  // events of the workspace searches, made once per device
    cudaEvent_t a, b;
    FP_CUDA(cudaEventCreate(&a));
    FP_CUDA(cudaEventCreate(&b));
    c->ev0 = a;
    c->ev1 = b;
  }
  prep.ev0 = c->ev0;
  prep.ev1 = c->ev1;
  prep.external = true;
  prep.dev = c->ws;
  s = upload_one(&prep, st, *c, prep.dev, c->ws_pinned, c->ws_pinned + rb_off, true);
  if (s) return s;
  prep.pinned = c->ws_pinned + rb_off;
  prep.stage_off = stage_off - rb_off;
  prep.uploaded = true;
  s = enqueue_one(&prep, st, o);
  if (s) return s;
  fpcode_result res;
  s = finish_one(&prep, st, &res, witness);
  prep.ev0 = prep.ev1 = nullptr;  // the context's
  (void)t0;
  if (s) return s;
  *d = res.d;
  return FPCODE_OK;
}

int fpcode_min_distance_batch(int num, const fpcode_desc *codes, void *stream, const fpcode_opts *opts,
                              fpcode_result *results, uint8_t *witnesses) {
  if (num < 0 || (num > 0 && (!codes || !results))) return FPCODE_EINVAL;
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = (cudaStream_t)stream;
  fpcode_opts o;
  fpcode_opts_default(&o);
  if (opts) o = *opts;
  std::vector<std::unique_ptr<fph::Prepared>> preps(num);
  std::vector<int> status(num, FPCODE_OK);
  // batch_words 1: one launch per kernel variant (prime class and words per
  // slice), each of the single-code kernels, which also run pair-leaf
  // codes; else the batched kernels over p in {3, 5, 7}
  const bool per_variant = o.batch_words == 1;
  {
    // host preparation of the codes, spread over the host's cores
    const int nth = std::max(1, std::min<int>((int)std::thread::hardware_concurrency(), (num + 7) / 8));
    std::atomic<int> next{0};
    auto work = [&]() {
      for (;;) {
        const int i = next.fetch_add(1);
        if (i >= num) break;
        preps[i].reset(new fph::Prepared());
        fpcode_opts oi = o;
        if (!per_variant) oi.pair_leaves = 0;  // the batched kernels take one-row leaves
        if (codes[i].budget) oi.budget = codes[i].budget;
        status[i] = fph::prepare(codes[i].p, codes[i].n, codes[i].k, codes[i].G, oi, preps[i].get());
      }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nth; ++t) pool.emplace_back(work);
    work();
    for (auto &th : pool) th.join();
  }
  const double t_prep = ms_since(t0);
  DevCtx *c;
  int s = get_ctx(&c);
  if (s) return s;
  // groups: the batched kernels for p in {3,5,7} (narrow: W <= 2, wide:
  // W <= 4); one launch per other variant
  std::vector<std::vector<int>> groups;
  {
    std::vector<int> narrow, wide;
    std::vector<std::vector<int>> other(64);
    const int narrow_w = o.batch_words == 4 ? 0 : 2;
    for (int i = 0; i < num; ++i) {
      if (status[i] != FPCODE_OK) continue;
      if (preps[i]->variant < 12 && !per_variant) (preps[i]->W <= narrow_w ? narrow : wide).push_back(i);
      else other[preps[i]->variant].push_back(i);
    }
    if (!narrow.empty()) groups.push_back(narrow);
    if (!wide.empty()) groups.push_back(wide);
    for (auto &g : other)
      if (!g.empty()) groups.push_back(g);
  }
  std::vector<size_t> woff(num + 1, 0);
  for (int i = 0; i < num; ++i) woff[i + 1] = woff[i] + (size_t)codes[i].n;
  std::lock_guard<std::mutex> lk(c->ws_mu);
  // Every group is planned and laid out first, at its own offset in the
  // workspace and in the pinned staging; then all uploads, launches and
  // read-backs go onto the stream back to back, with one synchronisation at
  // the end, so the GPU does not wait for the host between groups.
  struct Launch {
    std::vector<const fph::Prepared *> codesv;
    std::vector<int> idx;
    const void *fn = nullptr;
    int smem = 0, ctas = 0;
    Layout L;
    size_t dev_off = 0, pin_off = 0, rb_off = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
  };
  std::vector<Launch> ls;
  size_t dev_total = 0, pin_total = 0;
  for (auto &grp : groups) {
    Launch g;
    for (int i : grp)
      if (!preps[i]->passes.empty()) {
        g.codesv.push_back(preps[i].get());
        g.idx.push_back(i);
      }
    if (g.codesv.empty()) continue;
    const bool multi = g.codesv[0]->variant < 12 && !per_variant;
    int wmax = 1;
    for (auto *P : g.codesv) wmax = std::max(wmax, P->W);
    g.fn = multi ? fpk::kernel_multi357(wmax) : kernel_for(g.codesv[0]->variant);
    g.smem = smem_for(g.codesv);
    int per_sm = 0;
    s = occupancy(g.fn, g.smem, o.ctas_per_sm, &per_sm);
    if (s) return s;
    g.ctas = c->sms * per_sm;
    const bool many = g.idx.size() > 1;
    for (int i : g.idx)
      fph::plan_tasks(preps[i].get(), g.ctas, o.prefixes_per_lane,
                      o.min_steps > 0 ? o.min_steps : many ? fph::kMinStepsBatch : fph::kMinStepsSingle, !many);
    g.L = make_layout(g.codesv);
    g.dev_off = dev_total;
    dev_total += align256(g.L.total);
    g.pin_off = pin_total;
    g.rb_off = pin_total + align256(g.L.static_bytes);
    pin_total = g.rb_off + align256(g.L.dyn_bytes);
    ls.push_back(std::move(g));
  }
  s = ws_reserve(*c, std::max<size_t>(dev_total, 256), std::max<size_t>(pin_total, 256));
  if (s) return s;
  int err = FPCODE_OK;
  for (auto &g : ls) {
    char *d = c->ws + g.dev_off;
    fill_static(g.L, g.codesv, *c, c->ws_pinned + g.pin_off, d, 0);
    if (cudaEventCreate(&g.e0) != cudaSuccess || cudaEventCreate(&g.e1) != cudaSuccess) {
      err = FPCODE_ECUDA;
      break;
    }
    if (cudaMemcpyAsync(d, c->ws_pinned + g.pin_off, g.L.static_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(d + g.L.off_states, 0, g.L.dyn_bytes + g.L.aux_bytes, st) != cudaSuccess ||
        cudaEventRecord(g.e0, st) != cudaSuccess) {
      err = FPCODE_ECUDA;
      break;
    }
    if ((err = launch(g.fn, g.ctas, g.smem, st, d, g.L, kparams(o, 0))) != FPCODE_OK) break;
    if (cudaEventRecord(g.e1, st) != cudaSuccess ||
        cudaMemcpyAsync(c->ws_pinned + g.rb_off, d + g.L.off_states, g.L.dyn_bytes, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess) {
      err = FPCODE_ECUDA;
      break;
    }
  }
  if (!err && cudaStreamSynchronize(st) != cudaSuccess) err = FPCODE_ECUDA;
  int nlaunch = -1;
  for (auto &g : ls) {
    if (!err && g.e1) {
      ++nlaunch;
      float ms = 0;
      cudaEventElapsedTime(&ms, g.e0, g.e1);
      const SlotState *states = reinterpret_cast<const SlotState *>(c->ws_pinned + g.rb_off);
      CtlDyn dyn;
      std::memcpy(&dyn, c->ws_pinned + g.rb_off + g.L.dyn_bytes - sizeof(CtlDyn), sizeof(dyn));
      for (size_t q = 0; q < g.idx.size(); ++q) {
        const int i = g.idx[q];
        uint8_t *w = witnesses ? witnesses + woff[i] : nullptr;
        fph::decode_result(*preps[i], outcome_of(states[q], dyn), &results[i], w);
        results[i].t_kernel_ms = ms;
        results[i].launch = nlaunch;
        results[i].t_prepare_ms = t_prep;
      }
    }
    if (g.e0) cudaEventDestroy(g.e0);
    if (g.e1) cudaEventDestroy(g.e1);
  }
  if (err) {
    fph::set_error("fpcode_min_distance_batch: a CUDA call failed");
    return err;
  }
  for (int i = 0; i < num; ++i) {
    if (status[i] != FPCODE_OK) {
      std::memset(&results[i], 0, sizeof(results[i]));
      results[i].status = status[i];
      results[i].d = -1;
    } else if (preps[i]->passes.empty()) {
      fph::DeviceOutcome oc{fpk::kNoKey, 0, FPCODE_EBUDGET, -1};
      fph::decode_result(*preps[i], oc, &results[i], nullptr);
    }
    results[i].t_total_ms = ms_since(t0);
  }
  return FPCODE_OK;
}

}  // extern "C"

// ===========================================================================
// Device self-test of the bit-sliced operations and the integer-rate
// microbenchmark.
// ===========================================================================
namespace {

template <int R>
__global__ void bitslice_kernel(int op, int p, int count, const uint32_t *a, const uint32_t *b, uint32_t *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const uint32_t *x = a + (size_t)i * R;
  const uint32_t *y = b + (size_t)i * R;
  uint32_t *z = out + (size_t)i * R;
  uint32_t xa[R], ya[R], za[R];
  for (int q = 0; q < R; ++q) {
    xa[q] = x[q];
    ya[q] = y[q];
    za[q] = 0;
  }
  switch (op) {
    case FPCODE_OP_ADD:
      if (p == 3) fpbs::add_exact<3, R>(xa, ya, za, p);
      else if (p == 7) fpbs::add_exact<7, R>(xa, ya, za, p);
      else if (p == 31 || p == 127) fpbs::add_mersenne<R>(xa, ya, za);  // R = r of p here
      else fpbs::add_generic<R>(xa, ya, za, p);
      for (int q = 0; q < R; ++q) z[q] = za[q];
      break;
    case FPCODE_OP_NZ_SUB: out[i] = fpbs::nz_sub<R>(xa, ya); break;
    case FPCODE_OP_NZ_ADD:
      out[i] = (p == 3) ? fpbs::nz_add_p3(xa[0], xa[1], ya[0], ya[1]) : fpbs::nz_add_mersenne<R>(xa, ya);
      break;
    case FPCODE_OP_NEG:
      fpbs::neg_mersenne<R>(xa, za);
      for (int q = 0; q < R; ++q) z[q] = za[q];
      break;
    case FPCODE_OP_MUL2:
      fpbs::mul_pow2_mersenne<R>(xa, za, 1);
      for (int q = 0; q < R; ++q) z[q] = za[q];
      break;
  }
}

// Independent chains of one instruction kind: op 0 LOP3, 1 POPC, 2 IADD.
template <int OP>
__global__ void intpeak_kernel(uint32_t *sink, long long *cycles, int iters, uint32_t seed) {
  uint32_t v[8];
  for (int q = 0; q < 8; ++q) v[q] = (threadIdx.x + 1u) * (2u * q + 3u) ^ seed;
  const uint32_t k1 = seed * 0x9E3779B9u, k2 = seed ^ 0x5bd1e995u;
  long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (OP == 0) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(v[q]) : "r"(k1), "r"(k2));
      if (OP == 1) asm volatile("popc.b32 %0, %0;" : "+r"(v[q]));
      if (OP == 2) asm volatile("add.u32 %0, %0, %1;" : "+r"(v[q]) : "r"(k1));
    }
  }
  long long t1 = clock64();
  uint32_t acc = 0;
  for (int q = 0; q < 8; ++q) acc ^= v[q];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace

extern "C" {

int fpcode_test_pass_times(fpcode_prepared *prep, void *stream, double *us, int max) {
  if (!prep || !prep->uploaded || !us) return -1;
  Layout L = make_layout({&prep->host});
  std::vector<unsigned long long> t(fpk::kMaxPasses + 1);
  FP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  FP_CUDA(cudaMemcpy(t.data(), prep->dev + L.off_times, t.size() * sizeof(unsigned long long),
                     cudaMemcpyDeviceToHost));
  const int n = std::min<int>(max, (int)prep->host.passes.size());
  for (int i = 0; i < n; ++i) us[i] = t[i] >= t[fpk::kMaxPasses] ? (double)(t[i] - t[fpk::kMaxPasses]) * 1e-3 : -1.0;
  return n;
}

int fpcode_test_pair_table_device(const fpcode_prepared *prep, int j, uint32_t *out, int max_words) {
  const fph::Prepared *P = prep ? &prep->host : nullptr;
  if (!P || !P->pair || j < 0 || j >= P->m || !out || max_words < 0) return -FPCODE_EINVAL;
  const int words = (int)P->pair_words_per_set();
  if (words > max_words) return -FPCODE_EINVAL;
  const void *fn = P->p == 3 ? fpk::pair_table_kernel_p3(P->W) : fpk::pair_table_kernel_p7(P->W);
  if (!fn) return -FPCODE_EINVAL;
  const size_t mw = P->table_words_per_set();
  const int smem = (int)P->smem_bytes_per_set();
  uint32_t *d_rows = nullptr, *d_out = nullptr;
  cudaError_t e = cudaMalloc(&d_rows, mw * 4);
  if (e == cudaSuccess) e = cudaMalloc(&d_out, (size_t)words * 4 + 4);
  if (e == cudaSuccess) e = cudaMemcpy(d_rows, &P->table[(size_t)j * mw], mw * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && smem > 48 * 1024) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) {
    const uint32_t *rows = d_rows;
    int k = P->k, rwpad = P->rwpad, sigp = P->pair_sigp, ow = words;
    void *args[] = {(void *)&rows, (void *)&k, (void *)&rwpad, (void *)&sigp, (void *)&d_out, (void *)&ow};
    e = cudaLaunchKernel(fn, dim3(1), dim3(fpk::kThreads), args, (size_t)smem, 0);
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, d_out, (size_t)words * 4, cudaMemcpyDeviceToHost);
  if (d_rows) cudaFree(d_rows);
  if (d_out) cudaFree(d_out);
  if (e != cudaSuccess) {
    fph::set_error(cudaGetErrorString(e));
    return -FPCODE_ECUDA;
  }
  return words;
}

int fpcode_prepared_bytes(const fpcode_prepared *prep, uint64_t *h2d, uint64_t *d2h) {
  if (!prep) return FPCODE_EINVAL;
  Layout L = make_layout({&prep->host});
  if (h2d) *h2d = L.off_times;  // tables, descriptors, the first state and the zeroed bookkeeping
  if (d2h) *d2h = L.dyn_bytes;
  return FPCODE_OK;
}

int fpcode_test_bitslice_device(int op, int p, int count, const uint32_t *a, const uint32_t *b, uint32_t *out) {
  if (!fph::is_odd_prime(p) || count < 0 || !a || !b || !out) return FPCODE_EINVAL;
  const bool mersenne = ((p + 1) & p) == 0;
  if ((op == FPCODE_OP_NEG || op == FPCODE_OP_MUL2 || op == FPCODE_OP_NZ_ADD) && !mersenne) return FPCODE_EINVAL;
  if (op < FPCODE_OP_ADD || op > FPCODE_OP_MUL2) return FPCODE_EINVAL;
  if (count == 0) return FPCODE_OK;
  const int r = fpbs::bits_for(p);
  const size_t in_words = (size_t)count * r;
  const size_t out_words = (op == FPCODE_OP_NZ_SUB || op == FPCODE_OP_NZ_ADD) ? (size_t)count : in_words;
  uint32_t *da = nullptr, *db = nullptr, *dout = nullptr;
  FP_CUDA(cudaMalloc(&da, in_words * 4));
  FP_CUDA(cudaMalloc(&db, in_words * 4));
  FP_CUDA(cudaMalloc(&dout, in_words * 4));
  FP_CUDA(cudaMemcpy(da, a, in_words * 4, cudaMemcpyHostToDevice));
  FP_CUDA(cudaMemcpy(db, b, in_words * 4, cudaMemcpyHostToDevice));
  const int threads = 128, blocks = (count + threads - 1) / threads;
  switch (r) {
    case 2: bitslice_kernel<2><<<blocks, threads>>>(op, p, count, da, db, dout); break;
    case 3: bitslice_kernel<3><<<blocks, threads>>>(op, p, count, da, db, dout); break;
    case 4: bitslice_kernel<4><<<blocks, threads>>>(op, p, count, da, db, dout); break;
    case 5: bitslice_kernel<5><<<blocks, threads>>>(op, p, count, da, db, dout); break;
    case 6: bitslice_kernel<6><<<blocks, threads>>>(op, p, count, da, db, dout); break;
    case 7: bitslice_kernel<7><<<blocks, threads>>>(op, p, count, da, db, dout); break;
    default: bitslice_kernel<8><<<blocks, threads>>>(op, p, count, da, db, dout); break;
  }
  FP_CUDA(cudaGetLastError());
  FP_CUDA(cudaMemcpy(out, dout, out_words * 4, cudaMemcpyDeviceToHost));
  cudaFree(da);
  cudaFree(db);
  cudaFree(dout);
  return FPCODE_OK;
}

int fpcode_int_peaks(void *stream, double *rates) {
  if (!rates) return FPCODE_EINVAL;
  DevCtx *c;
  int s = get_ctx(&c);
  if (s) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = c->sms * 8, threads = 256, iters = 4096;
  uint32_t *sink = nullptr;
  long long *cyc = nullptr;
  FP_CUDA(cudaMalloc(&sink, sizeof(uint32_t) * blocks * threads));
  FP_CUDA(cudaMalloc(&cyc, sizeof(long long) * blocks));
  std::vector<long long> h(blocks);
  cudaEvent_t e0, e1;
  FP_CUDA(cudaEventCreate(&e0));
  FP_CUDA(cudaEventCreate(&e1));
  double per_clk[3] = {0, 0, 0}, per_s[3] = {0, 0, 0}, mhz = 0;
  for (int op = 0; op < 3; ++op) {
    for (int rep = 0; rep < 2; ++rep) {  // first run warms up
      cudaEventRecord(e0, st);
      if (op == 0) intpeak_kernel<0><<<blocks, threads, 0, st>>>(sink, cyc, iters, 7u);
      if (op == 1) intpeak_kernel<1><<<blocks, threads, 0, st>>>(sink, cyc, iters, 7u);
      if (op == 2) intpeak_kernel<2><<<blocks, threads, 0, st>>>(sink, cyc, iters, 7u);
      cudaEventRecord(e1, st);
    }
    FP_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    FP_CUDA(cudaMemcpy(h.data(), cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost));
    long long mx = 1;
    for (long long x : h) mx = std::max(mx, x);
    const double ops = (double)blocks * threads * iters * 8.0;
    per_clk[op] = ops / c->sms / (double)mx;
    per_s[op] = ops / (ms * 1e-3);
    if (op == 0) mhz = (double)mx / (ms * 1e3);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  cudaFree(cyc);
  rates[0] = per_clk[0];
  rates[1] = per_clk[1];
  rates[2] = per_clk[2];
  rates[3] = per_s[0];
  rates[4] = per_s[1];
  rates[5] = mhz;
  return FPCODE_OK;
}

}  // extern "C"
