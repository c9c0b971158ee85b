// fp_internal.h -- host-side structures of libfpcode shared by the
// preparation code (fp_host.cpp) and the CUDA driver (fp_api.cu).
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fpcode.h"
#include "fp_enum.cuh"
#include "fp_types.h"

namespace fph {

// Thread-local error text behind fpcode_last_error().
void set_error(const std::string &msg);
const char *last_error();

const fpenum::Binom &binom();  // host binomial table

bool is_odd_prime(int p);

// A bound u with no codeword behind it: the largest key of weight u, its
// pass field past every pass.  Any record of weight <= u replaces it, and
// the skip rule (which needs a key from a pass already entered) never fires
// on it.
inline uint64_t bound_key(uint32_t u) { return ((uint64_t)u << fpk::kKeyW) | ((1ull << fpk::kKeyW) - 1); }

// Digit width of the packed coefficient counter for prime p (the kernels
// use the same: 1 bit for p = 3, 4 for p = 5, 7, 8 otherwise).
int digit_bits_of(int p);

struct Prepared {
  int p = 0, n = 0, k = 0, r = 0, W = 0, rwpad = 0, m = 0, variant = 0;
  fpcode_opts opts{};
  std::vector<int> kj;           // fresh pivots of each Gamma_j
  std::vector<uint8_t> gam;      // m * k * n: Gamma_j, rows in pivot order
  std::vector<int> piv;          // m * k pivot columns (increasing)
  std::vector<int> red;          // m * (n - k) non-pivot columns (increasing)
  std::vector<uint32_t> table;   // per set: k * (p-1) * rwpad bit-sliced multiples, then (one-row leaves) the row signatures
  std::vector<fpk::PassDesc> passes;
  // Pair leaves (fp_types.h): passes with g >= 2 read a table of pair
  // signatures of A[y] + c A[x] and the segments of the task plan.
  bool pair = false;
  int pair_sigp = 0;             // words per pair entry (a power of two)
  std::vector<fpk::PairSeg> segs;  // all passes' segments (PassDesc.seg_off, nseg)
  int complete = 0;              // schedule reaches the last level
  uint64_t code_hash = 0;        // hash of (p, n, k, per_round_check, defer, pair) and G: schedule and key layout
  int seed_u = 0;                // least weight of the g = 1 passes (rows of the Gamma_j), 0: none;
                                 // a search starts with it as its bound (SlotDesc.seed_u)
  int L0 = 0;                    // lower bound before any pass
  double t_prepare_ms = 0;
  size_t pair_entries() const { return (size_t)(p - 1) * ((size_t)k * (k - 1) / 2); }
  // pair signatures (pair_sigp words an entry), then slice 0 of each entry
  // (W words), each part padded to whole 16-byte vectors
  size_t pair_words_per_set() const {
    return pair ? ((pair_entries() * (size_t)pair_sigp + 3) & ~(size_t)3) + ((pair_entries() * (size_t)W + 3) & ~(size_t)3)
                : 0;
  }
  int pair_quick_max = 0;        // thresholds up to this take the one-popcount pair bound
  // Words of one information set in the uploaded table: the multiples, and
  // for one-row leaves the row signatures.  Pair leaves upload only the
  // multiples; the kernel builds the pair table from them in shared memory.
  size_t table_words_per_set() const {
    return pair ? (size_t)k * (size_t)(p - 1) * rwpad
                : (size_t)k * ((size_t)(p - 1) * rwpad + fpk::sig_words(p, r, W));
  }
  size_t table_bytes_per_set() const { return table_words_per_set() * 4; }
  // Shared memory one staged information set takes (with the pair table).
  size_t smem_bytes_per_set() const { return (table_words_per_set() + pair_words_per_set()) * 4; }
};

// Guided share of a pair-leaf pass (task_share, or its default for a pass
// that is (last) or is not the last of its launch).
int task_share_of(const fpcode_opts &o, bool last);

// Elimination, information sets, multiples, schedule.  Returns an fpcode
// status; the error text is set on failure.
int prepare(int p, int n, int k, const uint8_t *G, const fpcode_opts &opts, Prepared *out);

// Tasks and prefixes per lane of every pass for a grid of `ctas` CTAs.
// fixed_pl > 0: tasks of fixed_pl prefixes per lane everywhere.  Else a pass
// too small to give every lane of the grid min_steps prefixes gets fixed
// tasks of min_steps prefixes per lane (fewer tasks than CTAs), the others
// guided tasks.  min_steps trades the latency of one small code (1: spread
// each pass over the whole grid) against throughput (a lane's setup cost
// shared by more prefixes).  spread_tiny: a pass under one prefix unit per
// lane of the grid still gets one unit per lane (the first passes of a
// search run with a loose threshold, many exact leaves each, and sit on the
// path to the first termination tests).
void plan_tasks(Prepared *P, int ctas, int fixed_pl, int min_steps, bool spread_tiny);

// Pair-leaf table limit per information set: with the binomial columns it
// keeps four 256-thread CTAs resident per SM.
constexpr size_t kPairTableMaxBytes = 40 * 1024;
constexpr int kMinStepsSingle = 8;   // one code per launch
constexpr int kMinStepsBatch = 32;   // many codes share the grid
constexpr int kMinStepsServe = 1;    // streamed codes: latency first

// Name and SM count of the current device (fp_api.cu).  Returns an fpcode status.
int device_identity(int *sms, char *name, size_t name_len);

// Fill a result from the final device state of one code.
struct DeviceOutcome {
  uint64_t best_key;     // kNoKey if none
  uint64_t enumerated;
  int status;            // fpcode status; -1: did not finish
  int stop_pass;         // last pass entered (-1: none)
};
int decode_result(const Prepared &P, const DeviceOutcome &o, fpcode_result *res, uint8_t *witness);
// Coefficients (length k) of the codeword a packed key stands for, with its
// level and information set; false if the key names none.
bool key_coefficients(const Prepared &P, uint64_t key, int *g_out, int *j_out, std::vector<int> &coef);

}  // namespace fph

// The opaque handle of the C ABI: host preparation plus its device copy.
struct fpcode_prepared {
  fph::Prepared host;
  int device = -1;
  int ctas = 0;         // grid the tasks were planned for
  int smem = 0;         // dynamic shared memory of one launch
  int init_u = 0;       // > 0: the search starts with this upper bound (single-pass probes)
  int resume_from = 0;  // > 0: the next search starts at this pass (fpcode_search_resume)
  uint64_t slice_lo = 0, slice_hi = 0;  // slice_hi > 0: only tasks [slice_lo, slice_hi) of the one pass
  uint64_t resume_key = ~0ull;  // ... with this best key
  int last_status = -100;       // outcome of the last finished search (for checkpoints)
  int last_stop = -1;
  uint64_t last_key = ~0ull;
  bool uploaded = false;
  bool external = false;  // device/pinned buffers borrowed from a workspace
  char *dev = nullptr;    // [CtlStatic][SlotDesc][PassDesc...][table] [SlotState][CtlDyn]
  size_t dev_bytes = 0;
  size_t off_ctl = 0, off_slot = 0, off_pass = 0, off_table = 0, off_state = 0, dyn_bytes = 0;
  char *pinned = nullptr; // read-back of the dynamic part
  size_t stage_off = 0;   // pinned + stage_off: 64 bytes staging the first state's values (bound, resume)
  bool state_clean = false;     // the dynamic state is zero (upload with state, or a kernel that cleaned up)
  bool mapped_outcome = false;  // the kernel writes its outcome into `pinned` and zeroes its state
  void *ev0 = nullptr, *ev1 = nullptr;  // cudaEvent_t around the kernel
  fpcode_opts run_opts{};
};
