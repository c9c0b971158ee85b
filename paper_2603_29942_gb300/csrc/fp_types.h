// fp_types.h -- data shared by the host driver and the enumeration kernels.
#pragma once
#include <stddef.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define FPK_HD __host__ __device__ inline
#else
#define FPK_HD inline
#endif

namespace fpk {

#ifndef FPK_THREADS
#define FPK_THREADS 256
#endif
constexpr int kThreads = FPK_THREADS;  // threads per CTA (256: 8 warps)
constexpr int kWarps = kThreads / 32;
constexpr int kMaxK = 64;            // rows: subsets are 64-bit masks
constexpr int kMaxW = 4;             // 32-bit words per slice: n - k <= 128
constexpr int kMaxPasses = 255;      // pass index fits 8 bits of the key
constexpr int kMaxN = 255;           // weight fits 8 bits of the key
constexpr uint64_t kMaxPrefix = 1ull << 34;  // prefix index fits 34 bits

// Packed witness key: (weight, pass, prefix index, leaf row, leaf coefficient).
// atomicMin on it keeps the lowest weight and, among equal weights, the
// first codeword in enumeration order.
constexpr int kKeyW = 56, kKeyP = 48, kKeyI = 14, kKeyX = 8;
constexpr uint64_t kNoKey = ~0ull;

FPK_HD uint64_t make_key(uint32_t weight, uint32_t pass, uint64_t I, uint32_t x, uint32_t c) {
  return ((uint64_t)weight << kKeyW) | ((uint64_t)pass << kKeyP) | (I << kKeyI) | ((uint64_t)x << kKeyX) |
         (uint64_t)c;
}
FPK_HD uint32_t key_weight(uint64_t key) { return (uint32_t)(key >> kKeyW); }
FPK_HD uint32_t key_pass(uint64_t key) { return (uint32_t)(key >> kKeyP) & 0xFFu; }
FPK_HD uint64_t key_prefix(uint64_t key) { return (key >> kKeyI) & ((1ull << 34) - 1); }
FPK_HD uint32_t key_leaf(uint64_t key) { return (uint32_t)(key >> kKeyX) & 63u; }
FPK_HD uint32_t key_coef(uint64_t key) { return (uint32_t)key & 0xFFu; }

// One pass (g, j) of the schedule.
struct PassDesc {
  int32_t g, j;
  int32_t L_before;   // lower bound before the pass (valid: earlier passes complete)
  int32_t L_after;    // lower bound once the pass is complete
  int32_t round_end;  // last pass of round g (per-round termination check)
  int32_t pl;         // > 0: fixed tasks of kThreads * pl units; 0: guided
  uint32_t ntasks;    // CTA tasks in the pass
  uint32_t phases;    // guided: number of phases (guided_phases), 0: fixed tasks of kThreads units
  uint64_t nprefix;   // prefixes (g >= 2) or rows (g == 1)
  uint64_t size;      // codewords in the pass: C(k,g)(p-1)^(g-1)
  uint64_t NC;        // (p-1)^(g-2) coefficient vectors per prefix subset
  uint32_t plan_ctas; // guided: tasks per phase
  uint32_t unit;      // prefixes per work unit: b^t, aligned to the coefficient counter
  // Tasks of all passes form one sequence: CTAs take them in order, so a
  // pass's tasks are handed out as soon as the previous pass has none left.
  uint32_t task_base;      // tasks of all earlier passes
  uint32_t seg_off;        // pair-leaf passes: first segment of the pass in the code's segment list
  uint32_t nseg;           // pair-leaf passes: its segments (0: a one-row-leaf pass)
  uint32_t task_off;       // a slice of the pass (fpcode_prepared_pass_slice): its first task in the pass's plan
};

// Words per row of the pair-signature table (Mersenne p = 3, 7): for each
// pair {c, -c} (representatives c = 1 for p = 3; 1, 2, 4 for p = 7) and
// word w, the r-1 words y_i xor y_{i+1} of y = c * A[row] (0 otherwise).
FPK_HD int sig_words(int p, int r, int W) {
  const int raw = p == 3 ? W * (r - 1) : p == 7 ? 3 * W * (r - 1) : 0;
  return (raw + 3) & ~3;
}
FPK_HD int pair_rep(int p, int q) { return p == 7 ? (1 << q) : q + 1; }

// Variant id: prime class * 4 + (W - 1); classes 0: p = 3, 1: p = 5,
// 2: p = 7, 3 + (r - 4): other primes with r bits (r = 4..8), 8: p = 31,
// 9: p = 127 (the Mersenne primes above 7, with their own exact add).
FPK_HD int variant_id(int p, int r, int W) {
  int cls = p == 3 ? 0 : p == 5 ? 1 : p == 7 ? 2 : p == 31 ? 8 : p == 127 ? 9 : 3 + (r - 4);
  return cls * 4 + (W - 1);
}

// Guided tasks of a pass work in rows of kThreads units (one unit per lane
// of a CTA), so every lane of a task but those of the pass's last row is
// busy.  While more than C = plan_ctas rows are left, a phase gives each of
// C tasks ceil(left / 2C) rows (tasks shrink as the pass drains); the last
// rows go one per task.  Calls f(phase tasks, rows per task) per phase
// until it returns true; returns the tasks of the pass.
template <class F>
FPK_HD uint64_t guided_phases(uint64_t rows, uint64_t C, F f) {
  uint64_t left = rows, tasks = 0;
  while (left > C) {
    const uint64_t per = (left + 2 * C - 1) / (2 * C);  // >= 1 here
    if (f(C, per)) return tasks;
    tasks += C;
    left -= C * per;
  }
  f(left, (uint64_t)1);
  return tasks + left;
}

// Unit range [lo, hi) of CTA task t of a pass with g >= 2 (a unit is
// d.unit consecutive prefixes; every unit starts where the lowest digits of
// the coefficient counter are zero, so all lanes of a warp take the same
// Gray steps): fixed tasks of kThreads * pl units, or guided rows.
FPK_HD void task_range(const PassDesc &d, uint64_t t, uint64_t *lo, uint64_t *hi) {
  const uint64_t N = d.nprefix / d.unit;
  if (d.pl > 0 || d.phases == 0) {
    const uint64_t chunk = (uint64_t)kThreads * (uint64_t)(d.pl > 0 ? d.pl : 1);
    *lo = t * chunk;
    *hi = *lo + chunk < N ? *lo + chunk : N;
    return;
  }
  const uint64_t rows = (N + kThreads - 1) / kThreads;
  uint64_t row0 = 0, nrow = 1;
  guided_phases(rows, d.plan_ctas, [&](uint64_t tasks, uint64_t per) {
    if (t < tasks) {
      row0 += t * per;
      nrow = per;
      return true;
    }
    t -= tasks;
    row0 += tasks * per;
    return false;
  });
  *lo = row0 * kThreads;
  *hi = (row0 + nrow) * kThreads < N ? (row0 + nrow) * kThreads : N;
}
static_assert(sizeof(PassDesc) == 80, "PassDesc layout");

// ---------------------------------------------------------------------------
// Pair leaves (p = 3, 7).  A codeword of pass g >= 3 with rows T splits into
// its two largest rows y < x and the stem Q (the other g - 2 rows, largest
// q).  The table holds, for every pair y < x and c in [1, p), the pair
// signature of B = A[y] + c A[x]; the lane holds the exact stem sum S, and
// one popcount bounds both S + B and S - B (the pair filter).  S - B is -1
// times the codeword with stem coefficients -c_Q, so stems take only half
// the coefficients of q (h in [1, (p-1)/2]) and every class is met once.
// Stem J of a pass: h = J / N1 + 1, and J % N1 is a prefix index of the
// one-row-leaf enumeration over rows 0..k-2 at level g - 1 (largest row q,
// the rest R with its coefficient counter).  Pass g = 2 has one empty stem
// (S = 0) whose entries are the codewords themselves.
//
// Entry order: pairs by y descending, then x ascending, then c; the
// entries with y > q are the first (p-1) C(k-1-q, 2).  After the signatures
// the table holds slice 0 of every B (W words an entry): with the
// signatures it gives B exactly (slice i+1 = slice i xor signature word i,
// for the natural encoding of p = 2^r - 1), for the exact path.
// ---------------------------------------------------------------------------

// One segment of a pair-leaf pass: stems from the block (h, q) on, cut into
// tasks of 256 >> lsplit groups of lanes, each group taking spg stems and
// its 1 << lsplit lanes splitting each stem's entries.
struct PairSeg {
  uint32_t task_end;  // tasks of the pass up to the end of this segment
  uint16_t spg;       // stems per group per task
  uint8_t q;          // largest stem row of the first block (255: the empty stem of g = 2)
  uint8_t hsplit;     // (h - 1) << 4 | lsplit
};
static_assert(sizeof(PairSeg) == 8, "PairSeg layout");

// Packed key of a pair-leaf codeword: (weight, pass, stem J (33 bits),
// entry e (14 bits), sign (S + B: 0, S - B: 1)).
constexpr int kPairKeyJ = 15, kPairKeyE = 1;
FPK_HD uint64_t make_pair_key(uint32_t weight, uint32_t pass, uint64_t J, uint32_t e, uint32_t sign) {
  return ((uint64_t)weight << kKeyW) | ((uint64_t)pass << kKeyP) | (J << kPairKeyJ) | ((uint64_t)e << kPairKeyE) |
         (uint64_t)sign;
}
FPK_HD uint64_t pair_key_stem(uint64_t key) { return (key >> kPairKeyJ) & ((1ull << 33) - 1); }
FPK_HD uint32_t pair_key_entry(uint64_t key) { return (uint32_t)(key >> kPairKeyE) & 0x3FFFu; }
FPK_HD uint32_t pair_key_sign(uint64_t key) { return (uint32_t)key & 1u; }

// Entries of the pairs with y > q: (p - 1) C(k - 1 - q, 2) (q = -1: all).
FPK_HD uint32_t pair_entries_above(int k, int q, int b) {
  const uint32_t t = (uint32_t)(k - 1 - q);
  return (uint32_t)b * (t * (t - 1) / 2);
}
// Entry e -> (y, x, c).  Pair index P = e / b; with t = k - 1 - y the pairs
// above y number C(t, 2), so t is the largest with C(t, 2) <= P.
FPK_HD void pair_entry_rows(int k, int b, uint32_t e, int *y, int *x, int *c) {
  const uint32_t P = e / (uint32_t)b;
  *c = (int)(e - P * (uint32_t)b) + 1;
  uint32_t t = 1;
  while ((t + 1) * t / 2 <= P) ++t;
  *y = k - 1 - (int)t;
  *x = *y + 1 + (int)(P - t * (t - 1) / 2);
}

// First stem of segment s of pair-leaf pass d (B(n, t) = C(n, t)).  Stems
// of the blocks before (h, q): (h - 1) N1 + C(q, g - 2) (p-1)^(g-3), with
// N1 = C(k - 2, g - 2) (p-1)^(g-3) the stems per h.
template <class BT>
FPK_HD uint64_t pair_seg_first(const PassDesc &d, const PairSeg &s, int k, const BT &B) {
  if (s.q == 255) return 0;
  const uint64_t N1 = B(k - 2, d.g - 2) * d.NC;
  return (uint64_t)(s.hsplit >> 4) * N1 + B(s.q, d.g - 2) * d.NC;
}

// Stem range [Ja, Jb) and entry split of task t of pair-leaf pass d, whose
// segments are seg[0 .. d.nseg) (device: a shared-memory copy; host: the
// plan itself).  The segment is the first whose task_end exceeds t.  Group
// g of the task takes stems [Ja + g spg, Ja + (g + 1) spg) within [Ja, Jb).
template <class BT>
FPK_HD void pair_task(const PassDesc &d, const PairSeg *seg, int k, const BT &B, uint64_t t, uint64_t *Ja,
                      uint64_t *Jb, int *lsplit, int *spg = nullptr) {
  int lo = 0, hi = (int)d.nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (seg[mid].task_end > t) hi = mid;
    else lo = mid + 1;
  }
  const uint64_t t0 = lo > 0 ? seg[lo - 1].task_end : 0;
  const uint64_t J0 = pair_seg_first(d, seg[lo], k, B);
  const uint64_t J1 = lo + 1 < (int)d.nseg ? pair_seg_first(d, seg[lo + 1], k, B) : d.nprefix;
  *lsplit = seg[lo].hsplit & 15;
  if (spg) *spg = seg[lo].spg;
  const uint64_t per = (uint64_t)(kThreads >> *lsplit) * seg[lo].spg;
  *Ja = J0 + (t - t0) * per;
  *Jb = *Ja + per < J1 ? *Ja + per : J1;
}

// Static description of one code as the kernel sees it.
struct SlotDesc {
  int32_t p, n, k, r, W, rwpad;  // rwpad: words per stored multiple (r*W rounded up to 4)
  int32_t m, npasses;
  int32_t variant;               // kernel variant (prime and words)
  int32_t per_round_check;
  int32_t mid_pass_exit;
  int32_t complete;              // 1: the schedule runs to the last level
  int32_t seed_u;                // > 0: least weight of the g = 1 passes, the search's first bound
  int32_t pair_sigp;             // > 0: pair-leaf passes (g >= 2), words per pair-table entry; 0: one-row leaves
  int32_t pair_quick_max;        // pair leaves: thresholds up to this take the one-popcount bound
  int32_t nsegs;                 // pair leaves: segments of all passes (after the pass descriptors)
  const uint32_t *table;         // m * k * (p-1) * rwpad words, device
  const PassDesc *passes;        // npasses entries, device
  uint64_t seq;                  // serving: ticket of the code in this slot
  unsigned long long *pass_times;  // optional: %globaltimer at each pass end (device)
};
static_assert(sizeof(SlotDesc) == 96, "SlotDesc layout");

// Dynamic state of one code, device memory (all zero = fresh).  Three
// 128-byte lines keep apart what is written at different rates: the task
// counter (an atomic per claim), the best key and finished flag (written
// rarely, read by every claim and every warp's threshold refresh), and the
// accounting written once per task or at the end.  On one line, the reads
// queued behind the claims' atomics at the L2.
struct alignas(128) SlotState {
  unsigned long long word;        // (generation << 48) | next task of the whole schedule
  unsigned long long pad_w[15];
  unsigned long long best_key;    // inverted packed witness key (0: none yet)
  int32_t finished;               // 0 while running; fin_tag(generation) once nothing is left to do
  int32_t pad_k[29];
  unsigned long long enumerated;  // codewords evaluated, passes past the stop included
  unsigned long long entered;     // codewords evaluated in the passes up to stop_pass
  int32_t frontier;               // next pass whose termination test is pending
  int32_t pad0;
  int32_t status;                 // 0 while running, then kDoneFlag | fpcode status
  int32_t stop_pass;              // last pass entered
  int32_t pad_a[24];
};
static_assert(sizeof(SlotState) == 384 && offsetof(SlotState, best_key) == 128 && offsetof(SlotState, enumerated) == 256,
              "SlotState lines");

// Per-pass bookkeeping of one code (zeroed with the state): the least
// weight recorded in each pass (stored as 256 - w, 0: none), the running
// minimum after each tested pass, tasks done and codewords evaluated.
struct SlotAux {
  int32_t pass_min[256];
  int32_t useq_after[256];  // least weight recorded in passes <= P (written by the test of pass P)
  uint32_t pass_done[256];
  unsigned long long pass_count[256];
};

// Serving: the finaliser of a code posts its outcome to host-mapped memory
// (seq written last, after a system-scope fence).
struct Completion {
  unsigned long long seq;
  unsigned long long best_key;   // packed key (kNoKey: none)
  unsigned long long enumerated; // codewords evaluated in the passes entered
  int32_t status;                // fpcode status
  int32_t stop_pass;
};

constexpr int32_t kRunning = -1;
// SlotState.word = (generation << 48) | task index over all passes; the
// generation is the low 16 bits of SlotDesc.seq (0 outside serving).
constexpr uint64_t kTaskMask = (1ull << 40) - 1;
constexpr int kGenShift = 48;
constexpr uint64_t kGenMask = 0xFFFFull;

// SlotState.finished of a concluded code: its generation in the high half,
// so that a claim of the next code in the slot never reads a predecessor's
// flag as its own (one-shot launches: generation 0, the value 1).
FPK_HD int32_t fin_tag(uint64_t gen) { return (int32_t)(((gen & kGenMask) << 16) | 1u); }

// Serving: per-slot count of claims in flight, on its own 32-byte sector.
// It is never reset while the server lives: every claim adds one before it
// reads the finished flag and takes it back after its last write, so the
// count stays balanced across the codes that follow one another in a slot.
constexpr int kInflightStride = 8;  // u32 words per slot

}  // namespace fpk
