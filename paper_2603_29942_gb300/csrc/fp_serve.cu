// fp_serve.cu -- serving: continuous batching of minimum-distance requests
// on the persistent enumeration kernel.
//
// A server owns one device block: a table of S slots (descriptor, pass
// schedule, state), a first-fit arena for the bit-sliced row tables, and a
// host-mapped array of completion records.  submit() prepares a code on the
// host, takes a free slot and arena space (FPCODE_EBUSY if either is
// missing: admission by device memory), and writes the slot on a private
// non-blocking copy stream -- tables, schedule and descriptor first, the
// zeroed state after them and the task counter that makes it claimable
// last, so a running kernel only sees a slot once it is complete.  The kernel (serving mode) keeps claiming tasks of every live
// slot, interleaving old and new codes; when a code certifies, its CTA
// writes the outcome to the mapped completion record, which poll() reads
// without any CUDA call.  The kernel exits after a short idle period and
// submit()/poll() relaunch it when codes are waiting.
//
// One thread drives a server; calls on one server are not thread-safe.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "../../include/fpcode.h"
#include "fp_driver.h"
#include "fp_internal.h"
#include "fp_kernels.h"

namespace {

#define SV_CUDA(call)                                                           \
  do {                                                                          \
    cudaError_t _e = (call);                                                    \
    if (_e != cudaSuccess) {                                                    \
      fph::set_error(std::string(#call) + ": " + cudaGetErrorString(_e));       \
      return FPCODE_ECUDA;                                                      \
    }                                                                           \
  } while (0)

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr int kMaxPassesPerSlot = fpk::kMaxPasses;
constexpr size_t kServeTableSet = 32 * 1024;      // shared memory per CTA: largest table of one set
constexpr size_t kServeTableCode = 256 * 1024;    // largest table of one code

// A slot is handed to the next code as soon as its completion is posted.
// The kernel posts it only once no other claim of the slot is in flight
// (the per-slot count in `inflight`, see conclude in fp_kernel.cuh): tasks
// of later passes that ran ahead of the termination test have stopped and
// counted themselves off by then, so none of them can write into the next
// code's bookkeeping.  A code whose wait for them gave up reports
// FPCODE_ETIMEOUT, and its slot stays out of use until the kernel exits.
//
// The task counter that makes a slot claimable is written in two steps: a
// transition value first (the new generation with a task index no schedule
// reaches, so claims that read it find nothing to do and never wrap into a
// real index), then the rest of the fresh state, then the counter at task
// 0, then the slot's flag word.  A claim therefore never sees a claimable
// counter next to a state that is still being written.
constexpr uint64_t kTaskTransit = 1ull << 39;

struct Slot {
  bool busy = false;
  bool held = false;  // its last code's drain timed out: unusable until the kernel has exited
  uint64_t ticket = 0;
  size_t arena_off = 0, arena_bytes = 0;
  std::unique_ptr<fph::Prepared> prep;
};

}  // namespace

struct fpcode_server {
  fpcode_serve_opts o{};
  fpd::DevCtx *ctx = nullptr;
  cudaStream_t kst = nullptr;  // kernel stream (the caller's)
  cudaStream_t cst = nullptr;  // admissions
  cudaEvent_t copies_done = nullptr, kernel_done = nullptr;
  bool kernel_live = false;
  const void *fn = nullptr;
  int smem = 0, ctas = 0, S = 0;
  char *dev = nullptr;
  size_t off_ctl = 0, off_slots = 0, off_passes = 0, off_arena = 0, arena_bytes = 0, off_states = 0,
         off_dyn = 0, off_aux = 0, off_flags = 0, off_inflight = 0, total = 0;
  fpk::Completion *done_host = nullptr, *done_dev = nullptr;
  char *staging = nullptr;  // pinned, one region per slot
  char *zeros = nullptr;    // pinned, never written: the source that clears a slot's bookkeeping
  size_t stage_per_slot = 0;
  std::vector<Slot> slots;
  std::vector<std::pair<size_t, size_t>> free_ext;  // arena extents (offset, bytes), sorted
  uint64_t next_ticket = 1;
  uint64_t launches = 0;  // kernel launches so far
  int running = 0;
  std::vector<std::pair<uint64_t, std::unique_ptr<fph::Prepared>>> host_done;  // nothing to run on the device
};

namespace {

bool arena_alloc(fpcode_server *s, size_t bytes, size_t *off) {
  bytes = a256(bytes);
  for (size_t i = 0; i < s->free_ext.size(); ++i) {
    auto &e = s->free_ext[i];
    if (e.second >= bytes) {
      *off = e.first;
      e.first += bytes;
      e.second -= bytes;
      if (e.second == 0) s->free_ext.erase(s->free_ext.begin() + (long)i);
      return true;
    }
  }
  return false;
}

void arena_free(fpcode_server *s, size_t off, size_t bytes) {
  bytes = a256(bytes);
  auto &v = s->free_ext;
  auto it = std::lower_bound(v.begin(), v.end(), std::make_pair(off, (size_t)0));
  it = v.insert(it, {off, bytes});
  size_t i = (size_t)(it - v.begin());
  if (i + 1 < v.size() && v[i].first + v[i].second == v[i + 1].first) {  // merge right
    v[i].second += v[i + 1].second;
    v.erase(v.begin() + (long)i + 1);
  }
  if (i > 0 && v[i - 1].first + v[i - 1].second == v[i].first) {  // merge left
    v[i - 1].second += v[i].second;
    v.erase(v.begin() + (long)i);
  }
}

// (Re)launch the serving kernel if it has exited while codes are waiting.
int ensure_kernel(fpcode_server *s) {
  if (s->kernel_live) {
    cudaError_t q = cudaEventQuery(s->kernel_done);
    if (q == cudaSuccess) s->kernel_live = false;
    else if (q != cudaErrorNotReady) SV_CUDA(q);
  }
  if (!s->kernel_live)  // no task of any code is in flight: held slots are free again
    for (auto &sl : s->slots) sl.held = false;
  if (s->kernel_live || s->running == 0) return FPCODE_OK;
  SV_CUDA(cudaStreamWaitEvent(s->kst, s->copies_done, 0));
  SV_CUDA(cudaMemsetAsync(s->dev + s->off_dyn, 0, sizeof(fpk::CtlDyn), s->kst));
  const fpk::SlotDesc *slots = reinterpret_cast<const fpk::SlotDesc *>(s->dev + s->off_slots);
  fpk::SlotState *states = reinterpret_cast<fpk::SlotState *>(s->dev + s->off_states);
  const fpk::CtlStatic *ctl = reinterpret_cast<const fpk::CtlStatic *>(s->dev + s->off_ctl);
  fpk::CtlDyn *dyn = reinterpret_cast<fpk::CtlDyn *>(s->dev + s->off_dyn);
  fpk::KParams kp = fpd::kparams(s->o.search, 1);
  const double idle = s->o.idle_exit_s > 0 ? s->o.idle_exit_s : 0.02;
  kp.idle_limit_ns = (unsigned long long)(idle * 1e9);
  kp.timeout_ns = 0;
  void *args[] = {(void *)&slots, (void *)&states, (void *)&ctl, (void *)&dyn, (void *)&kp};
  SV_CUDA(cudaLaunchKernel(s->fn, dim3(s->ctas), dim3(fpk::kThreads), args, (size_t)s->smem, s->kst));
  SV_CUDA(cudaEventRecord(s->kernel_done, s->kst));
  s->kernel_live = true;
  ++s->launches;
  return FPCODE_OK;
}

}  // namespace

extern "C" {

void fpcode_serve_opts_default(fpcode_serve_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->slots = 64;
  o->ctas_per_sm = 0;
  o->device_bytes = (size_t)64 << 20;
  o->idle_exit_s = 0.02;
  o->max_words = 2;
  fpcode_opts_default(&o->search);
}

int fpcode_serve_create(const fpcode_serve_opts *opts, void *stream, fpcode_server **out) {
  if (!out) return FPCODE_EINVAL;
  *out = nullptr;
  fpcode_serve_opts o;
  fpcode_serve_opts_default(&o);
  if (opts) o = *opts;
  if (o.slots < 1 || o.slots > 4096 || o.device_bytes < 4096 || (o.max_words != 2 && o.max_words != 4)) {
    fph::set_error("serve: need 1..4096 slots, some device memory and max_words 2 or 4");
    return FPCODE_EINVAL;
  }
  std::unique_ptr<fpcode_server> s(new fpcode_server());
  s->o = o;
  s->kst = (cudaStream_t)stream;
  int st = fpd::get_ctx(&s->ctx);
  if (st) return st;
  s->fn = fpk::kernel_multi357(o.max_words);
  s->smem = (int)kServeTableSet + fpk::kBinomBytes;
  int per_sm = 0;
  st = fpd::occupancy(s->fn, s->smem, o.ctas_per_sm, &per_sm);
  if (st) return st;
  s->ctas = s->ctx->sms * per_sm;
  s->S = o.slots;
  const size_t S = (size_t)s->S;
  size_t off = 0;
  s->off_ctl = off;
  off = a256(off + sizeof(fpk::CtlStatic));
  s->off_slots = off;
  off = a256(off + S * sizeof(fpk::SlotDesc));
  s->off_passes = off;
  off = a256(off + S * kMaxPassesPerSlot * sizeof(fpk::PassDesc));
  s->off_arena = off;
  s->arena_bytes = a256(o.device_bytes);
  off += s->arena_bytes;
  s->off_states = off;
  off = a256(off + S * sizeof(fpk::SlotState));
  s->off_dyn = off;
  off = a256(off + sizeof(fpk::CtlDyn));
  s->off_aux = off;
  off = a256(off + S * sizeof(fpk::SlotAux));
  s->off_flags = off;
  off = a256(off + (S + 3) / 4 * 16);
  s->off_inflight = off;
  off = a256(off + S * fpk::kInflightStride * sizeof(uint32_t));
  s->total = off;
  SV_CUDA(cudaMalloc(&s->dev, s->total));
  SV_CUDA(cudaHostAlloc(&s->done_host, S * sizeof(fpk::Completion), cudaHostAllocMapped));
  std::memset(s->done_host, 0, S * sizeof(fpk::Completion));
  SV_CUDA(cudaHostGetDevicePointer((void **)&s->done_dev, s->done_host, 0));
  s->stage_per_slot =
      a256(sizeof(fpk::SlotDesc)) + a256(kMaxPassesPerSlot * sizeof(fpk::PassDesc)) + a256(sizeof(fpk::SlotState) + 32) +
      kServeTableCode;
  const size_t init_bytes = s->off_arena;  // ctl + descriptors + schedules
  const size_t flag_bytes = (S + 3) / 4 * 16;
  SV_CUDA(cudaMallocHost(&s->staging, std::max(S * s->stage_per_slot,
                                               init_bytes + S * sizeof(fpk::SlotState) + flag_bytes)));
  SV_CUDA(cudaHostAlloc(&s->zeros, sizeof(fpk::SlotAux), cudaHostAllocDefault));
  std::memset(s->zeros, 0, sizeof(fpk::SlotAux));
  SV_CUDA(cudaStreamCreateWithFlags(&s->cst, cudaStreamNonBlocking));
  SV_CUDA(cudaEventCreateWithFlags(&s->copies_done, cudaEventDisableTiming));
  SV_CUDA(cudaEventCreateWithFlags(&s->kernel_done, cudaEventDisableTiming));
  // initial image: control block, empty descriptors, every state "finished"
  std::memset(s->staging, 0, init_bytes);
  fpk::CtlStatic cs{};
  cs.binom = s->ctx->binom;
  cs.done_host = s->done_dev;
  cs.aux = reinterpret_cast<fpk::SlotAux *>(s->dev + s->off_aux);
  cs.slot_flags = reinterpret_cast<uint32_t *>(s->dev + s->off_flags);
  cs.inflight = reinterpret_cast<uint32_t *>(s->dev + s->off_inflight);
  cs.nslots = s->S;
  cs.serve = 1;
  std::memcpy(s->staging + s->off_ctl, &cs, sizeof(cs));
  SV_CUDA(cudaMemcpyAsync(s->dev, s->staging, init_bytes, cudaMemcpyHostToDevice, s->cst));
  std::vector<fpk::SlotState> states(S);
  std::memset(states.data(), 0, S * sizeof(fpk::SlotState));
  for (auto &x : states) x.finished = 1;
  std::memcpy(s->staging + init_bytes, states.data(), S * sizeof(fpk::SlotState));
  SV_CUDA(cudaMemcpyAsync(s->dev + s->off_states, s->staging + init_bytes, S * sizeof(fpk::SlotState),
                          cudaMemcpyHostToDevice, s->cst));
  uint32_t *flags = reinterpret_cast<uint32_t *>(s->staging + init_bytes + S * sizeof(fpk::SlotState));
  for (size_t i = 0; i < flag_bytes / 4; ++i) flags[i] = fpk::kSlotFinished;  // no code in any slot
  SV_CUDA(cudaMemcpyAsync(s->dev + s->off_flags, flags, flag_bytes, cudaMemcpyHostToDevice, s->cst));
  SV_CUDA(cudaMemsetAsync(s->dev + s->off_dyn, 0, sizeof(fpk::CtlDyn), s->cst));
  // in-flight claim counts: zero once, never reset while the server lives
  SV_CUDA(cudaMemsetAsync(s->dev + s->off_inflight, 0, S * fpk::kInflightStride * sizeof(uint32_t), s->cst));
  SV_CUDA(cudaStreamSynchronize(s->cst));
  s->slots.resize(S);
  s->free_ext.push_back({0, s->arena_bytes});
  *out = s.release();
  return FPCODE_OK;
}

int fpcode_serve_submit(fpcode_server *s, const fpcode_desc *code, uint64_t *ticket) {
  if (!s || !code || !ticket) return FPCODE_EINVAL;
  fpcode_opts o = s->o.search;
  o.pair_leaves = 0;  // the serving kernels take one-row leaves
  if (code->budget) o.budget = code->budget;
  std::unique_ptr<fph::Prepared> P(new fph::Prepared());
  int st = fph::prepare(code->p, code->n, code->k, code->G, o, P.get());
  if (st) return st;
  if (P->variant >= 12) {
    fph::set_error("serve: p must be 3, 5 or 7");
    return FPCODE_EINVAL;
  }
  if (P->W > s->o.max_words) {
    fph::set_error("serve: n - k needs more words per slice than the server's max_words");
    return FPCODE_EINVAL;
  }
  const size_t table_bytes = P->table.size() * sizeof(uint32_t);
  if (P->smem_bytes_per_set() > kServeTableSet || table_bytes > kServeTableCode) {
    fph::set_error("serve: code tables too large for a serving slot");
    return FPCODE_EINVAL;
  }
  if (P->passes.empty()) {  // the budget stops it before the first pass
    *ticket = s->next_ticket++;
    s->host_done.emplace_back(*ticket, std::move(P));
    return FPCODE_OK;
  }
  int slot = -1;
  for (int i = 0; i < s->S; ++i)
    if (!s->slots[i].busy && !s->slots[i].held) {
      slot = i;
      break;
    }
  if (slot < 0) {
    fph::set_error("serve: no free slot");
    return FPCODE_EBUSY;
  }
  size_t aoff = 0;
  if (!arena_alloc(s, table_bytes, &aoff)) {
    fph::set_error("serve: no device memory free for the tables");
    return FPCODE_EBUSY;
  }
  fph::plan_tasks(P.get(), s->ctas, o.prefixes_per_lane, o.min_steps > 0 ? o.min_steps : fph::kMinStepsServe, true);
  const uint64_t tk = s->next_ticket++;
  char *stg = s->staging + (size_t)slot * s->stage_per_slot;
  const size_t o_pass = a256(sizeof(fpk::SlotDesc));
  const size_t o_state = o_pass + a256(kMaxPassesPerSlot * sizeof(fpk::PassDesc));
  const size_t o_tab = o_state + a256(sizeof(fpk::SlotState) + 32);
  char *d_desc = s->dev + s->off_slots + (size_t)slot * sizeof(fpk::SlotDesc);
  char *d_pass = s->dev + s->off_passes + (size_t)slot * kMaxPassesPerSlot * sizeof(fpk::PassDesc);
  char *d_tab = s->dev + s->off_arena + aoff;
  fpk::SlotDesc sd{};
  sd.p = P->p;
  sd.n = P->n;
  sd.k = P->k;
  sd.r = P->r;
  sd.W = P->W;
  sd.rwpad = P->rwpad;
  sd.m = P->m;
  sd.npasses = (int)P->passes.size();
  sd.variant = P->variant;
  sd.per_round_check = P->opts.per_round_check;
  sd.mid_pass_exit = P->opts.mid_pass_exit;
  sd.complete = P->complete;
  sd.seed_u = P->seed_u;
  sd.pair_sigp = 0;
  sd.table = reinterpret_cast<const uint32_t *>(d_tab);
  sd.passes = reinterpret_cast<const fpk::PassDesc *>(d_pass);
  sd.seq = tk;
  std::memcpy(stg, &sd, sizeof(sd));
  std::memcpy(stg + o_pass, P->passes.data(), P->passes.size() * sizeof(fpk::PassDesc));
  std::memcpy(stg + o_tab, P->table.data(), table_bytes);
  // tables, schedule, descriptor; the zeroed state last (it makes the slot live)
  SV_CUDA(cudaMemcpyAsync(d_tab, stg + o_tab, table_bytes, cudaMemcpyHostToDevice, s->cst));
  SV_CUDA(cudaMemcpyAsync(d_pass, stg + o_pass, P->passes.size() * sizeof(fpk::PassDesc), cudaMemcpyHostToDevice,
                          s->cst));
  SV_CUDA(cudaMemcpyAsync(d_desc, stg, sizeof(sd), cudaMemcpyHostToDevice, s->cst));
  // the task counter at the transition value: claims that read it find no
  // task (and do not touch the slot's bookkeeping)
  char *d_state = s->dev + s->off_states + (size_t)slot * sizeof(fpk::SlotState);
  fpk::SlotState fresh{};
  fresh.word = ((unsigned long long)(tk & fpk::kGenMask) << fpk::kGenShift) | kTaskTransit;
  std::memcpy(stg + o_state, &fresh, sizeof(fresh));
  SV_CUDA(cudaMemcpyAsync(d_state, stg + o_state, sizeof(fresh.word), cudaMemcpyHostToDevice, s->cst));
  // per-pass minima and counts, and the rest of the state.  Admissions use
  // copies only: a memset is a kernel, and it could not start while the
  // serving kernel holds every SM.
  SV_CUDA(cudaMemcpyAsync(s->dev + s->off_aux + (size_t)slot * sizeof(fpk::SlotAux), s->zeros,
                          sizeof(fpk::SlotAux), cudaMemcpyHostToDevice, s->cst));
  constexpr size_t kRest = offsetof(fpk::SlotState, best_key);  // the lines after the counter's
  SV_CUDA(cudaMemcpyAsync(d_state + kRest, stg + o_state + kRest, sizeof(fpk::SlotState) - kRest,
                          cudaMemcpyHostToDevice, s->cst));
  // then the counter at task 0: the code is claimable from here on
  unsigned long long *w0 = reinterpret_cast<unsigned long long *>(stg + o_state + sizeof(fpk::SlotState));
  *w0 = (unsigned long long)(tk & fpk::kGenMask) << fpk::kGenShift;
  SV_CUDA(cudaMemcpyAsync(d_state, w0, sizeof(*w0), cudaMemcpyHostToDevice, s->cst));
  // the flag word last: until it changes, slot scans skip the slot
  uint32_t *flag = reinterpret_cast<uint32_t *>(stg + o_state + sizeof(fpk::SlotState) + 8);
  *flag = fpk::slot_flag_gen(tk & fpk::kGenMask);
  SV_CUDA(cudaMemcpyAsync(s->dev + s->off_flags + (size_t)slot * 4, flag, sizeof(*flag), cudaMemcpyHostToDevice,
                          s->cst));
  SV_CUDA(cudaEventRecord(s->copies_done, s->cst));
  Slot &sl = s->slots[slot];
  sl.busy = true;
  sl.ticket = tk;
  sl.arena_off = aoff;
  sl.arena_bytes = table_bytes;
  sl.prep = std::move(P);
  ++s->running;
  *ticket = tk;
  return ensure_kernel(s);
}

int fpcode_serve_poll(fpcode_server *s, fpcode_result *out, uint64_t *tickets, uint8_t *witnesses, int max,
                      int *n_out) {
  if (!s || !n_out || max < 0 || (max > 0 && (!out || !tickets))) return FPCODE_EINVAL;
  int n = 0;
  while (n < max && !s->host_done.empty()) {
    auto &h = s->host_done.back();
    fph::DeviceOutcome oc{fpk::kNoKey, 0, FPCODE_EBUDGET, -1};
    fph::decode_result(*h.second, oc, &out[n], witnesses ? witnesses + (size_t)n * FPCODE_MAX_N : nullptr);
    tickets[n++] = h.first;
    s->host_done.pop_back();
  }
  for (int i = 0; i < s->S && n < max; ++i) {
    Slot &sl = s->slots[i];
    if (!sl.busy) continue;
    volatile fpk::Completion *c = s->done_host + i;
    if (c->seq != sl.ticket) continue;
    std::atomic_thread_fence(std::memory_order_acquire);
    fph::DeviceOutcome oc{};
    oc.best_key = c->best_key;
    oc.enumerated = c->enumerated;
    oc.status = c->status;
    oc.stop_pass = c->stop_pass;
    fph::decode_result(*sl.prep, oc, &out[n], witnesses ? witnesses + (size_t)n * FPCODE_MAX_N : nullptr);
    tickets[n++] = sl.ticket;
    // posted after the slot's claims drained: its tables are no longer read
    arena_free(s, sl.arena_off, sl.arena_bytes);
    sl.busy = false;
    sl.held = oc.status == FPCODE_ETIMEOUT;
    sl.prep.reset();
    --s->running;
  }
  *n_out = n;
  return ensure_kernel(s);
}

int fpcode_serve_drain(fpcode_server *s, int timeout_ms) {
  if (!s) return FPCODE_EINVAL;
  auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    int st = ensure_kernel(s);
    if (st) return st;
    bool all = true;
    for (int i = 0; i < s->S; ++i) {
      const Slot &sl = s->slots[i];
      if (sl.busy && ((volatile fpk::Completion *)(s->done_host + i))->seq != sl.ticket) {
        all = false;
        break;
      }
    }
    if (all) return FPCODE_OK;
    if (timeout_ms >= 0 &&
        std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms)) {
      fph::set_error("serve: drain timed out");
      return FPCODE_ETIMEOUT;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

int fpcode_serve_launches(const fpcode_server *s, uint64_t *n) {
  if (!s || !n) return FPCODE_EINVAL;
  *n = s->launches;
  return FPCODE_OK;
}

void fpcode_serve_destroy(fpcode_server *s) {
  if (!s) return;
  if (s->kst || s->kernel_live) cudaStreamSynchronize(s->kst);  // the kernel exits once idle
  if (s->cst) {
    cudaStreamSynchronize(s->cst);
    cudaStreamDestroy(s->cst);
  }
  if (s->copies_done) cudaEventDestroy(s->copies_done);
  if (s->kernel_done) cudaEventDestroy(s->kernel_done);
  if (s->dev) cudaFree(s->dev);
  if (s->done_host) cudaFreeHost(s->done_host);
  if (s->staging) cudaFreeHost(s->staging);
  if (s->zeros) cudaFreeHost(s->zeros);
  delete s;
}

}  // extern "C"
