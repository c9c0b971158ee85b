// fp_kernel.cuh -- persistent Brouwer-Zimmermann enumeration kernel (sm_103a).
//
// One launch serves a table of codes ("slots").  Every CTA loops: thread 0
// claims a task -- a contiguous range of kThreads * pl prefixes of the
// current pass of some code -- by atomicAdd on the code's (pass, task)
// word; the CTA stages that information set's bit-sliced row multiples into
// shared memory (coalesced 128-bit loads) and runs the task.  The CTA that
// completes the last task of a pass decides, on the device, whether the
// code is certified (L >= U, Sec. 3.1 Alg. 6) or hands out the next pass.
// No CTA ever waits on another except for the bounded wait at a pass
// hand-off, so single codes, batches and a stream of served codes share
// this one loop.
//
// Inside a task each lane walks its prefixes in Gray order (one exact
// bit-sliced add per step, Sec. 2.1 Alg. 3 / Alg. 4 or the generic form)
// and, for every leaf row x > m and coefficient c, evaluates the weight of
// S + c A[x] without forming it: the isometric subtraction of Sec. 4.3,
// popc(OR_i (S_i xor (p-c)A[x]_i)) per word.  All lanes of a warp share the
// leaf loop, so the leaf operand is a shared-memory broadcast.  A lane whose
// candidate could lower the bound takes a rare slow path that recomputes
// the weight exactly and folds a packed (weight, pass, prefix, leaf)
// key into the code's atomicMin upper bound; the bound is polled at every
// task for the early exit of Sec. 4.4.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fp_bitslice.cuh"
#include "fp_enum.cuh"
#include "fp_types.h"

namespace fpk {

// Launch-wide constants (device memory, written by the host).
struct CtlStatic {
  const fpenum::Binom *binom;
  Completion *done_host;  // serving: host-mapped completion records (else null)
  SlotAux *aux;           // per-slot pass minima and counts (zeroed with the states)
  uint32_t *slot_flags;   // per slot, padded to a multiple of four: see kSlotFinished
  uint32_t *inflight;     // serving: claims in flight per slot (kInflightStride apart); null otherwise
  char *outcome;          // one-code launches: host-mapped copy of the dynamic state (else null), see below
  int32_t nslots;
  int32_t serve;          // serving: slots appear while the kernel runs
  uint32_t dyn_bytes;     // outcome: bytes of [SlotState][CtlDyn] copied out
  uint32_t clean_bytes;   // outcome: bytes of the dynamic state (states, aux, flags) zeroed for the next launch
};

// A slot's flag word: (generation << 16) | kSlotFinished | kSlotExhausted.
// Claims read the flags four slots per 16-byte load and skip the slots
// with a bit set.  The host writes generation << 16 when it installs a
// code (zero for one-shot launches); a CTA that finds the code's task
// sequence used up sets kSlotExhausted by compare-and-swap on that exact
// value, so a late writer from an earlier code cannot mark its successor.
constexpr uint32_t kSlotFinished = 1u;
constexpr uint32_t kSlotExhausted = 2u;
__host__ __device__ inline uint32_t slot_flag_gen(unsigned long long gen) { return (uint32_t)(gen & 0xFFFFull) << 16; }

// Per-launch limits, passed by value.
struct KParams {
  unsigned long long wait_limit_ns;  // longest single wait at a pass hand-off
  unsigned long long timeout_ns;     // 0: none; else per-launch time limit
  unsigned long long idle_limit_ns;  // serving: exit after this long idle
  int32_t mid_pass;                  // -1: per code; 0 / 1: override
  int32_t lookahead;                 // 1: take tasks of later passes while earlier ones drain
};

// Launch-wide dynamic flags (zeroed before each launch).
struct CtlDyn {
  int32_t err;      // 1: a hand-off wait gave up; 2: time limit reached
  int32_t leaving;  // serving: the kernel is retiring (idle); claims exit, the host launches again
  unsigned long long last_busy;  // serving: %globaltimer of a recent claim that found work (max over CTAs)
  uint32_t exited;  // one-code launches with an outcome copy: CTAs that have left
  uint32_t pad;
};

// Shared memory: binomial columns C(n, t), t < kBinomCols, then the staged
// table of one information set.
constexpr int kBinomCols = fpenum::kBinomCols;
constexpr int kBinomBytes = kBinomCols * (fpenum::kMaxK + 1) * 8;  // 12480, a multiple of 16

// Words of one information set's table in global memory: the multiples,
// then (one-row leaves) the row signatures.  Pair leaves keep only the
// multiples there; the CTA builds the pair table after them in shared
// memory when it stages the set (build_pairs).
__device__ __forceinline__ int table_words(const SlotDesc &sd) {
  if (sd.pair_sigp > 0) return sd.k * (sd.p - 1) * sd.rwpad;
  return sd.k * ((sd.p - 1) * sd.rwpad + sig_words(sd.p, sd.r, sd.W));
}

// SlotState.status while a code is running is 0; the finaliser stores
// kDoneFlag | fpcode status.
constexpr int32_t kDoneFlag = 0x100;

template <int R, int W>
struct Shape {
  static constexpr int RW = R * W;
  static constexpr int RWP = (RW + 3) & ~3;
};

__device__ __forceinline__ unsigned long long ld_vol(const unsigned long long *p) {
  return *(volatile const unsigned long long *)p;
}
__device__ __forceinline__ int ld_vol(const int32_t *p) { return *(volatile const int32_t *)p; }
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Coherent (L2) copy of a descriptor: slots are rewritten by the host while
// a serving kernel runs, so descriptors never come from L1.
// Through the non-coherent (L1) path: for data that no thread of the
// launch writes.
template <class T>
__device__ __forceinline__ T load_nc(const T *p) {
  static_assert(sizeof(T) % 16 == 0, "16-byte multiple");
  T out;
  const uint4 *src = reinterpret_cast<const uint4 *>(p);
  uint4 *dst = reinterpret_cast<uint4 *>(&out);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(T) / 16); ++i) dst[i] = __ldg(src + i);
  return out;
}

template <class T>
__device__ __forceinline__ T load_cg(const T *p) {
  static_assert(sizeof(T) % 16 == 0, "16-byte multiple");
  T out;
  const uint4 *src = reinterpret_cast<const uint4 *>(p);
  uint4 *dst = reinterpret_cast<uint4 *>(&out);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(T) / 16); ++i) dst[i] = __ldcg(src + i);
  return out;
}

// Acquire-release fence at GPU scope: orders this thread's accesses before
// and after it (a release before a flag write, an acquire after a flag
// read).  Cheaper than the sequentially consistent __threadfence(), which
// only the store-then-load handshakes need (one side writes a flag and reads
// the other's, the other the reverse).
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// The best key is stored inverted (~key) so that an all-zero state means
// "no codeword yet" and atomicMax keeps the minimum key.
__device__ __forceinline__ uint64_t best_key(const SlotState *st) { return ~ld_vol(&st->best_key); }

template <int RWP>
__device__ __forceinline__ void load_entry(const uint32_t *tab, int idx, uint32_t (&e)[RWP]) {
  const uint4 *src = reinterpret_cast<const uint4 *>(tab + idx * RWP);
#pragma unroll
  for (int q = 0; q < RWP / 4; ++q) {
    uint4 v = src[q];
    e[4 * q] = v.x;
    e[4 * q + 1] = v.y;
    e[4 * q + 2] = v.z;
    e[4 * q + 3] = v.w;
  }
}

// s += multiple v of row t (exact, word by word).  Entry layout: word-major,
// e[w * R + i] = slice i of word w.
template <int P, int R, int W>
__device__ __forceinline__ void add_row(uint32_t (&s)[R * W], const uint32_t *tab, int t, int v, int p) {
  constexpr int RWP = Shape<R, W>::RWP;
  uint32_t e[RWP];
  load_entry<RWP>(tab, t * (p - 1) + (v - 1), e);
#pragma unroll
  for (int w = 0; w < W; ++w) fpbs::add_exact<P, R>(&s[w * R], &e[w * R], &s[w * R], p);
}

template <int P, int R, int W>
__device__ __forceinline__ void set_row(uint32_t (&s)[R * W], const uint32_t *tab, int t, int v, int p) {
  constexpr int RWP = Shape<R, W>::RWP;
  uint32_t e[RWP];
  load_entry<RWP>(tab, t * (p - 1) + (v - 1), e);
#pragma unroll
  for (int q = 0; q < R * W; ++q) s[q] = e[q];
}

// Exact sum of a prefix: A[m] (coefficient 1) + sum over the slots of Q.
// Rows of Q by slot, 6 bits each, for the first kSlotRows slots (a Gray
// step then finds its row with one shift instead of a walk over Q).
constexpr int kSlotRows = 10;

template <int P, int R, int W, int DB>
__device__ __forceinline__ void build_sum(uint32_t (&s)[R * W], const uint32_t *tab, const fpenum::Prefix &pf,
                                          int L, int b, int p, uint64_t &qrows, int hm = 1) {
  set_row<P, R, W>(s, tab, pf.m, hm, p);  // the largest row, coefficient hm (1 for a one-row-leaf prefix)
  uint64_t Q = pf.Q;
  qrows = 0;
  for (int slot = 0; slot < L; ++slot) {
    int q = fpenum::ctz64(Q);
    Q &= Q - 1;
    if (slot < kSlotRows) qrows |= (uint64_t)q << (6 * slot);
    int coef = fpenum::gray_digit<DB>(pf.d, slot, b, L) + 1;
    add_row<P, R, W>(s, tab, q, coef, p);
  }
}

// Weight of the redundant part of S + c A[x] via the stored multiple
// (p - c) A[x] = -c A[x]: isometric subtraction, one popc per word.
template <int R, int W>
__device__ __forceinline__ int leaf_weight(const uint32_t (&s)[R * W], const uint32_t *e) {
  int wsum = 0;
#pragma unroll
  for (int w = 0; w < W; ++w) wsum += __popc(fpbs::nz_sub<R>(&s[w * R], &e[w * R]));
  return wsum;
}

// Record a candidate codeword: the code's packed best key and the least
// weight of its pass.  Both are reductions whose result is not waited for:
// the caller lowers its own bound to the recorded weight and takes up the
// other CTAs' records when it next reads the best key.
__device__ __forceinline__ void record(SlotState *st, SlotAux *ax, int pass, uint64_t key) {
  atomicMax(&ax->pass_min[pass], 256 - (int)key_weight(key));
  atomicMax(&st->best_key, (unsigned long long)~key);
}

// ---------------------------------------------------------------------------
// Task of a pass with g == 1: the k rows themselves (coefficient 1).
// ---------------------------------------------------------------------------
template <int P, int R, int W>
__device__ void task_rows(const SlotDesc &sd, int pass, const uint32_t *tab, int U, SlotState *st, SlotAux *ax,
                          unsigned long long &count) {
  constexpr int RWP = Shape<R, W>::RWP;
  const int x = threadIdx.x;
  const int p = P ? P : sd.p;
  if (x < sd.k) {
    uint32_t e[RWP];
    load_entry<RWP>(tab, x * (p - 1), e);
    int wsum = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) wsum += __popc(fpbs::nz<R>(&e[w * R]));
    int weight = 1 + wsum;
    if (weight <= U) record(st, ax, pass, make_key((uint32_t)weight, (uint32_t)pass, 0, (uint32_t)x, 1));
    count += 1;
  }
}

// ---------------------------------------------------------------------------
// Task of a pass with g >= 2.
//
// Leaf filter.  For a leaf row x and a pair of coefficients {c, p-c}, the
// positions where BOTH S + cA[x] and S - cA[x] are nonzero give a lower
// bound on either weight.  For p = 2^r - 1, with y = cA[x] and d = S xor y,
// S + y = 0 iff d is all ones and S - y = 0 iff d is all zeros (negation is
// the bitwise complement), so that mask is OR_i (d_i xor d_{i+1}) =
// OR_i ((S_i xor S_{i+1}) xor (y_i xor y_{i+1})): the prefix keeps its r-1
// "signature" words, the row table stores the leaf's.  Other primes AND the
// two isometric subtractions.  One POPC per word covers two codewords (for
// p = 3 both leaf coefficients); only a pair whose bound is below the
// current threshold is evaluated exactly (slow path).
// ---------------------------------------------------------------------------
template <int P, int R, int W>
struct LeafFilter {
  static constexpr bool kMersenne = (P == 3 || P == 7);
  static constexpr int kSigW = kMersenne ? (((P == 3 ? W * (R - 1) : 3 * W * (R - 1)) + 3) & ~3) : 0;
  static constexpr int kPrefSig = kMersenne ? W * (R - 1) : 1;
  // leaves evaluated per vote: as many as the registers allow
  static constexpr int kUnroll = !kMersenne ? 1 : kSigW <= 4 ? 4 : kSigW <= 8 ? 2 : 1;
  // The one-popcount bound of W > 1 words (popc of the words' OR) is used
  // while the threshold is at most this: about 32 (1 - q^W) - 8, eight
  // under the bound's mean for random symbols, where q is the chance that
  // a position is zero in a word's pair mask (5/9 for p = 3, 13/49 for p = 7).
  static constexpr int kQuickMax = P == 3 ? (W == 2 ? 14 : W == 3 ? 18 : 21) : P == 7 ? (W == 2 ? 21 : 23) : 0;
};

// Lower bound on the redundant weight of S + c A[x] over every nonzero
// leaf coefficient c: the least bound of the pairs {c, p - c}.
template <bool B>
struct BoolTag {
  static constexpr bool value = B;
};

template <int P, int R, int W, bool QUICK, int NA>
__device__ __forceinline__ int pair_bound(const uint32_t (&s)[R * W], const uint32_t (&a)[NA], const uint32_t *sig,
                                          const uint32_t *tab, int x, int p) {
  using F = LeafFilter<P, R, W>;
  constexpr int RWP = Shape<R, W>::RWP;
  int best = 1 << 20;
  if constexpr (F::kMersenne) {
    uint32_t e[F::kSigW];
    load_entry<F::kSigW>(sig, x, e);
    constexpr int NP = (P - 1) / 2;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      if constexpr (W > 1 && QUICK) {
        // OR the words' masks before one popcount: popc(f_0 | f_1 | ...) is
        // at most sum_w popc(f_w), so it is a lower bound too; weaker, so
        // it is used only while the threshold is well under its mean
        uint32_t u = 0;
#pragma unroll
        for (int w = 0; w < W; ++w)
#pragma unroll
          for (int i = 0; i + 1 < R; ++i) u |= a[w * (R - 1) + i] ^ e[(q * W + w) * (R - 1) + i];
        best = min(best, __popc(u));
      } else {
        int lb = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
          uint32_t f = 0;
#pragma unroll
          for (int i = 0; i + 1 < R; ++i) f |= a[w * (R - 1) + i] ^ e[(q * W + w) * (R - 1) + i];
          lb += __popc(f);
        }
        best = min(best, lb);
      }
    }
  } else {
    const int b = p - 1;
    for (int q = 0; q < (p - 1) / 2; ++q) {
      const int c = q + 1;
      uint32_t e1[RWP], e2[RWP];
      load_entry<RWP>(tab, x * b + (p - c - 1), e1);  // (p - c) A = -c A
      load_entry<RWP>(tab, x * b + (c - 1), e2);      // c A = -(p - c) A
      int lb = 0;
#pragma unroll
      for (int w = 0; w < W; ++w)
        lb += __popc(fpbs::nz_sub<R>(&s[w * R], &e1[w * R]) & fpbs::nz_sub<R>(&s[w * R], &e2[w * R]));
      best = min(best, lb);
    }
  }
  return best;
}

// Slow path of leaf x: the exact redundant weight of S + c A[x] for every
// c, recording those below the lane's threshold (which then drops to it).
template <int P, int R, int W>
__device__ __forceinline__ void leaf_exact(const uint32_t (&s)[R * W], const uint32_t *tab, int x, int p, int g,
                                        int pass, uint64_t I, int &thr, SlotState *st, SlotAux *ax) {
  constexpr int RWP = Shape<R, W>::RWP;
  const int b = p - 1;
  for (int c = 1; c < p; ++c) {
    uint32_t e[RWP];
    load_entry<RWP>(tab, x * b + (p - c - 1), e);
    const int wr = leaf_weight<R, W>(s, e);
    if (wr < thr) {  // weights up to g + wr stay of interest: ties decide the witness by key
      record(st, ax, pass, make_key((uint32_t)(g + wr), (uint32_t)pass, I, (uint32_t)x, (uint32_t)c));
      thr = wr + 1;
    }
  }
}

template <int R, int W, int NA>
__device__ __forceinline__ void prefix_signature(const uint32_t (&s)[R * W], uint32_t (&a)[NA]) {
  static_assert(NA >= W * (R - 1), "signature size");
#pragma unroll
  for (int w = 0; w < W; ++w)
#pragma unroll
    for (int i = 0; i + 1 < R; ++i) a[w * (R - 1) + i] = s[w * R + i] ^ s[w * R + i + 1];
}

template <int P, int R, int W, int DB, int UNR>
__device__ void task_prefixes(const SlotDesc &sd, const PassDesc &pd, int pass, const uint32_t *tab,
                              const fpenum::BinomCols &B, uint64_t ulo, uint64_t uhi, int U, SlotState *st,
                              SlotAux *ax, unsigned long long &count) {
  constexpr int RW = R * W;
  constexpr int RWP = Shape<R, W>::RWP;
  using F = LeafFilter<P, R, W>;
  const int p = P ? P : sd.p;
  const int b = p - 1;
  const int k = sd.k;
  const int g = pd.g;
  const int L = g - 2;
  const uint32_t *sig = tab + k * b * RWP;  // pair signatures (Mersenne p)
  const uint64_t pu = (uhi - ulo + kThreads - 1) / kThreads;  // units per lane, same for the CTA
  const uint64_t unit = pd.unit;
  const uint64_t pl = pu * unit;                               // prefix steps
  uint64_t I = (ulo + (uint64_t)threadIdx.x * pu) * unit;
  const uint64_t Iend = min(I + pl, pd.nprefix < uhi * unit ? pd.nprefix : uhi * unit);
  int thr = U - g + 1;  // record weights <= U: redundant weight < U - g + 1

  uint32_t s[RW];
#pragma unroll
  for (int q = 0; q < RW; ++q) s[q] = 0;
  uint32_t a[F::kPrefSig];
#pragma unroll
  for (int q = 0; q < F::kPrefSig; ++q) a[q] = 0;
  fpenum::Prefix pf;
  pf.m = k;
  pf.qi = 0;
  pf.Q = 0;
  pf.d = 0;
  uint64_t ci = 0, nq = 1, qrows = 0;
  if (I < Iend) {
    pf = fpenum::prefix_unrank<DB>(B, I, k, g, b);
    ci = (I - fpenum::prefixes_below(B, pf.m, g, pd.NC)) - pf.qi * pd.NC;
    nq = B(pf.m, L);
    build_sum<P, R, W, DB>(s, tab, pf, L, b, p, qrows);
    if constexpr (F::kMersenne) prefix_signature<R, W>(s, a);
  }

  // prefixes left to this lane (the current one included); its index is Iend - left
  uint32_t left = I < Iend ? (uint32_t)(Iend - I) : 0u;
  const uint32_t nsteps = (uint32_t)pl;
  uint32_t cw = (uint32_t)(k - 1 - pf.m) * (uint32_t)b;  // codewords of the current prefix (set at rebuilds)
  uint32_t count32 = 0;                                   // codewords of this lane, flushed every 16 steps
  for (uint32_t base = 0; base < nsteps; base += 16) {
   if (base) {
      // a finished code only has tasks of passes past its stop left: drop
      // them; else take up the best weight recorded anywhere since
      int fin = 0, ub = 0;
      if ((threadIdx.x & 31) == 0) {
        fin = ld_vol(&st->finished);
        const uint64_t key = best_key(st);
        ub = key == kNoKey ? 255 : (int)key_weight(key);
      }
      if (__shfl_sync(0xffffffffu, fin, 0)) break;
      thr = min(thr, __shfl_sync(0xffffffffu, ub, 0) - g + 1);
    }
    count += count32;
    count32 = 0;
    const uint32_t end = min(base + 16u, nsteps);
   for (uint32_t step = base; step < end; ++step) {
    const bool act = left > 0;
    const int mlane = act ? pf.m : k;
    const int xs = (int)__reduce_min_sync(0xffffffffu, (unsigned)mlane) + 1;
    // the leaves of this step, with the one-popcount bound (QUICK) or the
    // per-word sum; the mode is picked once per step from the threshold
    auto leaves = [&](auto quick_tag) {
      constexpr bool QUICK = decltype(quick_tag)::value;
      if constexpr (UNR == 1) {
        for (int x = xs; x < k; ++x) {  // lanes whose prefix reaches above x sit it out
          const int tx = x > mlane ? thr : 0;
          if (__any_sync(0xffffffffu, pair_bound<P, R, W, QUICK>(s, a, sig, tab, x, p) < tx)) {
            if (x > mlane) leaf_exact<P, R, W>(s, tab, x, p, g, pass, Iend - left, thr, st, ax);
            thr = (int)__reduce_min_sync(0xffffffffu, (unsigned)thr);
          }
        }
      } else {
        // leaves above every active lane's largest row: no per-lane test needed
        const int xu = max(xs, (int)__reduce_max_sync(0xffffffffu, (unsigned)(act ? pf.m + 1 : 0)));
        for (int x = xs; x < xu; ++x) {  // lanes whose prefix reaches above x sit these out
          const int tx = x > mlane ? thr : 0;
          if (__any_sync(0xffffffffu, pair_bound<P, R, W, QUICK>(s, a, sig, tab, x, p) < tx)) {
            if (x > mlane) leaf_exact<P, R, W>(s, tab, x, p, g, pass, Iend - left, thr, st, ax);
            thr = (int)__reduce_min_sync(0xffffffffu, (unsigned)thr);
          }
        }
        int x = xu;
        for (; x + UNR <= k; x += UNR) {
          int lb[UNR];
#pragma unroll
          for (int u = 0; u < UNR; ++u) lb[u] = pair_bound<P, R, W, QUICK>(s, a, sig, tab, x + u, p);
          int lbm = lb[0];
#pragma unroll
          for (int u = 1; u < UNR; ++u) lbm = min(lbm, lb[u]);
          if (__any_sync(0xffffffffu, act && lbm < thr)) {
            if (act) {
#pragma unroll
              for (int u = 0; u < UNR; ++u)
                if (lb[u] < thr) leaf_exact<P, R, W>(s, tab, x + u, p, g, pass, Iend - left, thr, st, ax);
            }
            thr = (int)__reduce_min_sync(0xffffffffu, (unsigned)thr);
          }
        }
        for (; x < k; ++x) {
          if (__any_sync(0xffffffffu, act && pair_bound<P, R, W, QUICK>(s, a, sig, tab, x, p) < thr)) {
            if (act) leaf_exact<P, R, W>(s, tab, x, p, g, pass, Iend - left, thr, st, ax);
            thr = (int)__reduce_min_sync(0xffffffffu, (unsigned)thr);
          }
        }
      }
    };
    if constexpr (W > 1 && UNR > 1) {  // single-code kernels; the batched ones keep one copy
      if (thr <= F::kQuickMax) leaves(BoolTag<true>{});  // thr is the same on every lane here
      else leaves(BoolTag<false>{});
    } else {
      leaves(BoolTag<false>{});
    }
    if (act) count32 += cw;
    // advance to the next prefix
    if (left > 1) {
      int dir;
      const int slot = fpenum::prefix_advance<DB>(B, pf, ci, nq, pd.NC, b, L, &dir);
      if (slot >= 0) {
        const int q = slot < kSlotRows ? (int)(qrows >> (6 * slot)) & 63 : fpenum::nth_member(pf.Q, slot);
        add_row<P, R, W>(s, tab, q, dir > 0 ? 1 : b, p);  // c -> c+1: +A; c -> c-1: +(p-1)A
      } else {
        build_sum<P, R, W, DB>(s, tab, pf, L, b, p, qrows);
        cw = (uint32_t)(k - 1 - pf.m) * (uint32_t)b;
      }
      if constexpr (F::kMersenne) prefix_signature<R, W>(s, a);
    }
    left -= left > 0 ? 1u : 0u;
   }
  }
  count += count32;
}

// ---------------------------------------------------------------------------
// Task of a pair-leaf pass (g >= 2, p = 3 or 7; the enumeration is described
// in fp_types.h).  The CTA's stems [Ja, Jb) go to 256 >> lsplit groups of
// 1 << lsplit lanes, a contiguous run of stems per group; the lanes of a
// group hold the same exact stem sum S and split the stem's pair entries in
// interleaved chunks (lane sub takes chunks sub, sub + 2^lsplit, ...), so a
// warp's table loads are broadcasts or consecutive words.  Per entry: one
// pair bound (LOP3s and one popcount) for the two codewords S + B and S - B;
// the warp votes every few loads, and only a vote that finds a bound under
// the threshold runs the exact path, whose candidates are reduced to one
// key per warp before the atomic record.  The best weight recorded anywhere
// is read once per stem (the load issued before the stem's entries, used
// after them).
// ---------------------------------------------------------------------------
// Pair table of the staged information set, built by the CTA in shared
// memory from the set's staged multiples (tab): entries run over pairs
// y < x of rows by y descending, then x, then c in [1, p); entry (y, x, c)
// holds the pair signature words B_i xor B_{i+1} of B = A[y] + c A[x] (the
// exact add), zero-padded to sigp words, and, after all signatures (padded
// to 16 bytes), B's slice 0.  The same table the host hook
// fpcode_test_pair_entry computes, entry by entry.
template <int P, int R, int W>
__device__ __noinline__ void build_pairs(uint32_t *tab, int k, int rwpad, int sigp) {
  constexpr int b = P - 1;
  const int ne = b * (k * (k - 1) / 2);
  uint32_t *pt = tab + k * b * rwpad;
  uint32_t *p0 = pt + ((ne * sigp + 3) & ~3);
  for (int e = threadIdx.x; e < ne; e += kThreads) {
    // e = b P + (c - 1); pair P counts down the triangle: t = k - 1 - y rows
    // above y, the largest t with t (t - 1) / 2 <= P
    const uint32_t Pq = (uint32_t)e / (uint32_t)b;
    const int c = e - (int)Pq * b + 1;
    uint32_t t = (uint32_t)((1.0f + sqrtf(8.0f * (float)Pq + 1.0f)) * 0.5f);
    while (t > 1 && t * (t - 1) / 2 > Pq) --t;
    while ((t + 1) * t / 2 <= Pq) ++t;
    const int y = k - 1 - (int)t;
    const int x = y + 1 + (int)(Pq - t * (t - 1) / 2);
    const uint32_t *ay = tab + y * b * rwpad;
    const uint32_t *ax = tab + (x * b + (c - 1)) * rwpad;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      uint32_t sum[R];
      fpbs::add_exact<P, R>(ay + w * R, ax + w * R, sum, P);
#pragma unroll
      for (int i = 0; i + 1 < R; ++i) pt[e * sigp + w * (R - 1) + i] = sum[i] ^ sum[i + 1];
      p0[e * W + w] = sum[0];
    }
    for (int q = W * (R - 1); q < sigp; ++q) pt[e * sigp + q] = 0u;
  }
}

// Test hook kernel: one CTA of kThreads stages the multiples of one
// information set (k (p-1) rwpad words at rows) into shared memory, builds
// its pair table there (build_pairs) and copies the pair table out.
template <int P, int R, int W>
__global__ void __launch_bounds__(kThreads) pair_table_kernel(const uint32_t *rows, int k, int rwpad, int sigp,
                                                             uint32_t *out, int out_words) {
  extern __shared__ uint4 smem_pairs[];
  uint32_t *tab = reinterpret_cast<uint32_t *>(smem_pairs);
  const int mw = k * (P - 1) * rwpad;
  for (int i = threadIdx.x; i < mw; i += kThreads) tab[i] = rows[i];
  __syncthreads();
  build_pairs<P, R, W>(tab, k, rwpad, sigp);
  __syncthreads();
  for (int i = threadIdx.x; i < out_words; i += kThreads) out[i] = tab[mw + i];
}

template <int P, int R, int W>
struct PairShape {
  static constexpr int SW = W * (R - 1);                                    // signature words of an entry
  static constexpr int SP = SW <= 1 ? 1 : SW <= 2 ? 2 : SW <= 4 ? 4 : 8;  // padded (the host's pair_sigp)
  static constexpr int EPL = SP <= 2 ? 2 : 1;                               // entries per load
  static constexpr int LW = SP * EPL;                                       // words per load
  static constexpr int UNR = LW <= 4 ? 4 : 2;                               // loads per vote
  static_assert(UNR * EPL <= 8, "PairQueue holds 8 entries per lane per vote");
};

// A warp's queue of pair-leaf candidates: (entry << 5) | lane.
struct PairQueue {
  uint32_t n;
  uint32_t item[32 * 8 + 32];  // fewer than 32 left over, then 32 lanes x at most 8 entries of one vote
};

template <int LW>
__device__ __forceinline__ void load_words(const uint32_t *tab, uint32_t i, uint32_t (&e)[LW]) {
  if constexpr (LW == 2) {
    const uint2 v = reinterpret_cast<const uint2 *>(tab)[i];
    e[0] = v.x;
    e[1] = v.y;
  } else {
    load_entry<LW>(tab, (int)i, e);
  }
}

// Pair bound of S (signature a) and entry signature e: positions where both
// S + B and S - B are nonzero; QUICK: one popcount of the words' OR (weaker,
// used while the threshold is well under the bound's mean).
template <int R, int W, bool QUICK>
__device__ __forceinline__ int pair_lb(const uint32_t (&a)[W * (R - 1)], const uint32_t *e) {
  if constexpr (QUICK && W > 1) {
    uint32_t u = 0;
#pragma unroll
    for (int q = 0; q < W * (R - 1); ++q) u |= a[q] ^ e[q];
    return __popc(u);
  } else {
    int lb = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      uint32_t f = 0;
#pragma unroll
      for (int i = 0; i + 1 < R; ++i) f |= a[w * (R - 1) + i] ^ e[w * (R - 1) + i];
      lb += __popc(f);
    }
    return lb;
  }
}

// Exact path of entry e of stem J: B from its signature words `sig` and
// its slice 0 (`b0`, W words): slice i+1 = slice i xor signature word i.
// The redundant weights of S + B (isometric subtraction against -B, the
// complement of B where it is nonzero) and S - B; the least key under the
// threshold joins `best`.
template <int P, int R, int W>
__device__ __forceinline__ void pair_exact(const uint32_t (&s)[R * W], const uint32_t *sig, const uint32_t *b0, int g,
                                           int pass, uint64_t J, uint32_t e, int thr, uint64_t &best) {
  int wp = 0, wm = 0;
#pragma unroll
  for (int w = 0; w < W; ++w) {
    uint32_t Bw[R], nb[R];
    Bw[0] = b0[w];
#pragma unroll
    for (int i = 0; i + 1 < R; ++i) Bw[i + 1] = Bw[i] ^ sig[w * (R - 1) + i];
    fpbs::neg_mersenne<R>(Bw, nb);
    wp += __popc(fpbs::nz_sub<R>(&s[w * R], nb));
    wm += __popc(fpbs::nz_sub<R>(&s[w * R], Bw));
  }
  if (wp < thr) best = min(best, (uint64_t)make_pair_key((uint32_t)(g + wp), (uint32_t)pass, J, e, 0));
  if (g >= 3 && wm < thr) best = min(best, (uint64_t)make_pair_key((uint32_t)(g + wm), (uint32_t)pass, J, e, 1));
}

template <int P, int R, int W, int DB>
__device__ void task_pairs(const SlotDesc &sd, const PassDesc &pd, int pass, const uint32_t *tab,
                           const fpenum::BinomCols &B, uint64_t Ja, uint64_t Jb, int shape, int U, SlotState *st,
                           SlotAux *ax, unsigned long long &count) {
  using S = PairShape<P, R, W>;
  constexpr int RW = R * W;
  constexpr int SW = S::SW, SP = S::SP, EPL = S::EPL, LW = S::LW, UNR = S::UNR;
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int b = P - 1;
  const int k = sd.k;
  const int g = pd.g;
  const int lane = threadIdx.x & 31;
  const uint32_t *ptab = tab + k * b * sd.rwpad;  // pair signatures
  const uint32_t *p0tab = ptab + (((b * (k * (k - 1) / 2)) * SP + 3) & ~3);  // slice 0 of each entry
  const int lsplit = shape & 15;
  const int sub = (int)threadIdx.x & ((1 << lsplit) - 1);
  const uint64_t spg = (uint64_t)(shape >> 4);  // the plan's stems per group: aligned to the coefficient counter
  uint64_t J = Ja + (uint64_t)(threadIdx.x >> lsplit) * spg;
  const uint64_t Jend = J + spg < Jb ? J + spg : Jb;
  const uint32_t nstem = J < Jend ? (uint32_t)(Jend - J) : 0u;
  int thr = U - g + 1;  // record weights <= U: redundant weight < U - g + 1

  uint32_t s[RW];
#pragma unroll
  for (int q = 0; q < RW; ++q) s[q] = 0;
  uint32_t a[SW];
#pragma unroll
  for (int q = 0; q < SW; ++q) a[q] = 0;
  // the stem: h and the prefix over rows 0..k-2 at level g - 1 (g >= 3)
  const int L = g - 3;
  const uint64_t NC = pd.NC;
  const uint64_t N1 = g >= 3 ? B(k - 2, g - 2) * NC : 1;
  fpenum::Prefix pf;
  pf.m = -1;
  pf.qi = 0;
  pf.Q = 0;
  pf.d = 0;
  uint64_t ci = 0, nq = 1, qrows = 0, I1 = 0;
  int h = 1;
  if (nstem && g >= 3) {
    h = (int)(J / N1) + 1;
    I1 = J - (uint64_t)(h - 1) * N1;
    pf = fpenum::prefix_unrank<DB>(B, I1, k - 1, g - 1, b);
    ci = I1 - fpenum::prefixes_below(B, pf.m, g - 1, NC) - pf.qi * NC;
    nq = B(pf.m, L);
    build_sum<P, R, W, DB>(s, tab, pf, L, b, P, qrows, h);
  }
  const unsigned long long cpe = g >= 3 ? 2ull : 1ull;  // codewords per entry
  const uint32_t nmax = __reduce_max_sync(FULL, nstem);
  // the warp's candidate queue: up to UNR * EPL entries per lane per vote
  __shared__ PairQueue s_pq[kWarps];
  PairQueue *wq = &s_pq[threadIdx.x >> 5];
  if (lane == 0) wq->n = 0;
  __syncwarp();
  // the code's finished flag and best key, read by lane 0 and taken up once
  // the warp has done kPollWork entries since (the loads' latency hides
  // behind them)
  constexpr uint32_t kPollWork = 192;
  int pfin = 0;
  unsigned long long pkey = 0;
  if (lane == 0) {
    pfin = ld_vol(&st->finished);
    pkey = ld_vol(&st->best_key);
  }
  uint32_t since = 0;
  for (uint32_t it = 0; it < nmax; ++it) {
    const bool act = it < nstem;
    if constexpr (SW > 0) prefix_signature<R, W>(s, a);
    const uint32_t E = act ? pair_entries_above(k, pf.m, b) : 0u;  // pf.m = -1 for g = 2
    const uint32_t nch = E / EPL;  // E is a multiple of EPL: even for p = 3, a multiple of 6 for p = 7
    const uint32_t its = nch > (uint32_t)sub ? ((nch - (uint32_t)sub + (1u << lsplit) - 1) >> lsplit) : 0u;
    const uint32_t its_lo = __reduce_min_sync(FULL, its), its_hi = __reduce_max_sync(FULL, its);
    // Candidates (entries whose bound is under the threshold) go to the
    // warp's queue as (entry, lane); the warp checks them 32 at a time, each
    // lane taking one and fetching the owner's stem sum by shuffle, so the
    // exact path costs the warp one pass per 32 candidates instead of one
    // per vote that found any.  One record per warp, only if some lane found
    // a codeword under the threshold.
    auto check = [&](uint32_t first, uint32_t cnt) {
      const bool have = (uint32_t)lane < cnt;
      const uint32_t item = have ? wq->item[first + lane] : 0u;
      const int src = (int)(item & 31u);
      const uint32_t ec = item >> 5;
      uint32_t so[RW];
#pragma unroll
      for (int q = 0; q < RW; ++q) so[q] = __shfl_sync(FULL, s[q], src);
      const uint64_t Jo = (uint64_t)__shfl_sync(FULL, (unsigned long long)J, src);
      uint64_t best = kNoKey;
      if (have) {
        uint32_t ew[SP];
#pragma unroll
        for (int q = 0; q < SP; ++q) ew[q] = ptab[ec * SP + q];
        pair_exact<P, R, W>(so, ew, p0tab + ec * W, g, pass, Jo, ec, thr, best);
      }
      if (__any_sync(FULL, best != kNoKey)) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = min(best, (uint64_t)__shfl_xor_sync(FULL, (unsigned long long)best, o));
        if (lane == 0) record(st, ax, pass, best);
        thr = min(thr, (int)key_weight(best) - g + 1);
      }
    };
    // after a vote that found candidates: check full rounds of 32 from the
    // queue's end, keep the rest for the stem's end
    auto drain_full = [&]() {
      __syncwarp();
      uint32_t n = wq->n;
      while (n >= 32) {
        n -= 32;
        check(n, 32);
      }
      __syncwarp();
      if (lane == 0) wq->n = n;
      __syncwarp();
    };
    auto push = [&](uint32_t e) { wq->item[atomicAdd(&wq->n, 1u)] = (e << 5) | (uint32_t)lane; };
    auto entries = [&](auto quick_tag) {
      constexpr bool QUICK = decltype(quick_tag)::value;
      uint32_t i = 0;
      for (; i + UNR <= its_lo; i += UNR) {  // every lane has UNR more loads
        int lb[UNR * EPL];
        int lbm = 1 << 20;
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
          uint32_t e[LW];
          load_words<LW>(ptab, (uint32_t)sub + ((i + u) << lsplit), e);
#pragma unroll
          for (int v = 0; v < EPL; ++v) {
            lb[u * EPL + v] = pair_lb<R, W, QUICK>(a, &e[v * SP]);
            lbm = min(lbm, lb[u * EPL + v]);
          }
        }
        if (__any_sync(FULL, lbm < thr)) {
          if (lbm < thr) {
#pragma unroll
            for (int u = 0; u < UNR; ++u)
#pragma unroll
              for (int v = 0; v < EPL; ++v)
                if (lb[u * EPL + v] < thr) push(((uint32_t)sub + ((i + u) << lsplit)) * EPL + v);
          }
          drain_full();
        }
      }
      for (; i < its_hi; ++i) {  // the rest: lanes with fewer loads sit out
        const bool on = i < its;
        const uint32_t ch = on ? (uint32_t)sub + (i << lsplit) : 0u;
        uint32_t e[LW];
        load_words<LW>(ptab, ch, e);
        int lb[EPL];
        int lbm = 1 << 20;
#pragma unroll
        for (int v = 0; v < EPL; ++v) {
          lb[v] = on ? pair_lb<R, W, QUICK>(a, &e[v * SP]) : (1 << 20);
          lbm = min(lbm, lb[v]);
        }
        if (__any_sync(FULL, lbm < thr)) {
#pragma unroll
          for (int v = 0; v < EPL; ++v)
            if (lb[v] < thr) push(ch * EPL + v);
          drain_full();
        }
      }
    };
    if constexpr (W > 1) {
      if (thr <= sd.pair_quick_max) entries(BoolTag<true>{});  // thr is the same on every lane of the warp
      else entries(BoolTag<false>{});
    } else {
      entries(BoolTag<false>{});
    }
    // the stem's last candidates (the queue refers to this stem's sums)
    __syncwarp();
    if (const uint32_t n = wq->n) {
      check(0, n);
      __syncwarp();
      if (lane == 0) wq->n = 0;
      __syncwarp();
    }
    if (act && sub == 0) count += (unsigned long long)E * cpe;
    since += its_hi * EPL + 8;
    if (since >= kPollWork) {
      // the code finished: drop the rest; else take up the best weight recorded anywhere
      if (__shfl_sync(FULL, pfin, 0)) break;
      const uint64_t key = ~(uint64_t)__shfl_sync(FULL, pkey, 0);
      if (key != kNoKey) thr = min(thr, (int)key_weight(key) - g + 1);
      if (lane == 0) {
        pfin = ld_vol(&st->finished);
        pkey = ld_vol(&st->best_key);
      }
      since = 0;
    }
    // next stem
    if (act && it + 1 < nstem) {
      if (I1 + 1 < N1) {
        int dir;
        const int slot = fpenum::prefix_advance<DB>(B, pf, ci, nq, NC, b, L, &dir);
        if (slot >= 0) {
          const int qq = slot < kSlotRows ? (int)(qrows >> (6 * slot)) & 63 : fpenum::nth_member(pf.Q, slot);
          add_row<P, R, W>(s, tab, qq, dir > 0 ? 1 : b, P);  // c -> c+1: +A; c -> c-1: +(p-1)A
        } else {
          build_sum<P, R, W, DB>(s, tab, pf, L, b, P, qrows, h);
        }
        ++I1;
      } else {  // next h: the first prefix again, largest row coefficient h + 1
        ++h;
        I1 = 0;
        pf = fpenum::prefix_unrank<DB>(B, 0, k - 1, g - 1, b);
        ci = 0;
        nq = B(pf.m, L);
        build_sum<P, R, W, DB>(s, tab, pf, L, b, P, qrows, h);
      }
      ++J;
    }
  }
}

// One kernel variant: prime P (0: any, from the descriptor), r slices, W
// words per slice; UNR leaves per vote in the leaf loop (1: the plain loop,
// whose smaller code suits the batched kernels); PAIRS: pair-leaf passes
// for codes prepared with them (p = 3, 7, single-code kernels).
template <int P, int R, int W, int UNR = LeafFilter<P, R, W>::kUnroll, bool PAIRS = false>
struct Fixed {
  static constexpr int DB = P == 3 ? 1 : (P == 5 || P == 7) ? 4 : 8;  // as the host's digit width
  static constexpr int kSegCache = PAIRS ? 768 : 1;  // pair-leaf segments held in shared memory
  static constexpr int kPassCache = 24;                // pass descriptors held in shared memory (one code)
  // after staging a set: its pair table (pair-leaf codes), built in shared memory
  static __device__ __forceinline__ void stage_pairs(uint32_t *tab, const SlotDesc &sd) {
    if constexpr (PAIRS && (P == 3 || P == 7)) {
      if (sd.pair_sigp > 0) build_pairs<P, R, W>(tab, sd.k, sd.rwpad, sd.pair_sigp);
    }
  }
  static __device__ __forceinline__ void run(const SlotDesc &sd, const PassDesc &pd, int pass, const uint32_t *tab,
                                             const fpenum::BinomCols &B, uint64_t ulo, uint64_t uhi, int lsplit,
                                             int U, SlotState *st, SlotAux *ax, unsigned long long &count) {
    if constexpr (PAIRS && (P == 3 || P == 7)) {
      if (sd.pair_sigp > 0 && pd.g >= 2) {
        task_pairs<P, R, W, DB>(sd, pd, pass, tab, B, ulo, uhi, lsplit, U, st, ax, count);
        return;
      }
    }
    (void)lsplit;
    if (pd.g == 1) {
      if (ulo == 0) task_rows<P, R, W>(sd, pass, tab, U, st, ax, count);
    } else {
      task_prefixes<P, R, W, DB, UNR>(sd, pd, pass, tab, B, ulo, uhi, U, st, ax, count);
    }
  }
};


// Batched launches over codes with p in {3, 5, 7}: dispatch per task.  The
// narrow kernel (WMAX = 2: n - k <= 64) holds half the variants and so
// fits its registers without spilling; the wide one (WMAX = 4) takes the
// rest.
template <int WMAX>
struct Multi357 {
  static constexpr int kSegCache = 1;  // batches take one-row leaves
  static constexpr int kPassCache = 1;  // and read their pass descriptors from global memory
  static __device__ __forceinline__ void stage_pairs(uint32_t *, const SlotDesc &) {}  // one-row leaves only
  static __device__ __forceinline__ void run(const SlotDesc &sd, const PassDesc &pd, int pass, const uint32_t *tab,
                                             const fpenum::BinomCols &B, uint64_t ulo, uint64_t uhi, int lsplit,
                                             int U, SlotState *st, SlotAux *ax, unsigned long long &count) {
    switch (sd.variant) {
#define FPK_CASE(id, P, R, W) \
  case id: if constexpr (W <= WMAX) Fixed<P, R, W, 1>::run(sd, pd, pass, tab, B, ulo, uhi, lsplit, U, st, ax, count); break;
      FPK_CASE(0, 3, 2, 1)
      FPK_CASE(1, 3, 2, 2)
      FPK_CASE(2, 3, 2, 3)
      FPK_CASE(3, 3, 2, 4)
      FPK_CASE(4, 5, 3, 1)
      FPK_CASE(5, 5, 3, 2)
      FPK_CASE(6, 5, 3, 3)
      FPK_CASE(7, 5, 3, 4)
      FPK_CASE(8, 7, 3, 1)
      FPK_CASE(9, 7, 3, 2)
      FPK_CASE(10, 7, 3, 3)
      FPK_CASE(11, 7, 3, 4)
#undef FPK_CASE
      default: break;
    }
  }
};

enum { kCmdRun = 0, kCmdWait = 1, kCmdExit = 2 };

// What thread 0 hands to its CTA for one task.
struct Claim {  // the task taken (its code's and pass's descriptors: the ClaimCache)
  unsigned long long task;  // task index within the pass
  uint64_t ulo, uhi;        // its unit range (g >= 2; pair-leaf passes: stems; g == 1: task, task + 1)
  int slot, pass, U, skip;
  unsigned int ndone;       // tasks of the pass this claim completes (skipped runs: more than one)
  int lsplit;               // pair-leaf passes: lanes per stem (log2, low 4 bits) | stems per group << 4
};

// Shared-memory copy of pair-leaf segments: for a one-code launch, the
// whole list of the code (staged by the CTA at its start, pass = -2), else
// those of the pass thread 0 claims from (at most (p-1)/2 (k-2) <= 186).
constexpr int kSegPass = 192;
template <int N>
struct SegCache {
  PairSeg seg[N];
  int slot, pass;               // whose (-1: none; pass -2: the whole list)
  unsigned long long gen;
};

// Thread 0's cache of the descriptors it read last (one slot and pass), so
// that an idle probe costs two loads: the finished flag and the task word.
struct ClaimCache {
  int slot;  // -1: empty
  unsigned long long gen;
  int P;     // pass whose descriptor is cached (-1: none)
  SlotDesc sd;
  PassDesc pd;
  unsigned int sleep_ns;
  unsigned long long busy_note;  // serving: when this CTA last raised last_busy
};

// Pass of global task t: the cached pass, the next one, else a binary
// search over the passes' task_base fields.  pc: the launch's copy of its
// first npc pass descriptors in shared memory (one-code launches; 0 for
// the others), the rest come from global memory.
__device__ __forceinline__ bool locate(ClaimCache &cc, const PassDesc *pc, int npc, unsigned long long t) {
  auto tbase = [&](int i) -> unsigned long long {
    return i < npc ? (unsigned long long)pc[i].task_base : (unsigned long long)__ldcg(&cc.sd.passes[i].task_base);
  };
  auto tend = [&](int i) -> unsigned long long {
    return i < npc ? (unsigned long long)pc[i].task_base + pc[i].ntasks
                   : (unsigned long long)__ldcg(&cc.sd.passes[i].task_base) + __ldcg(&cc.sd.passes[i].ntasks);
  };
  auto take_pass = [&](int i) {
    cc.P = i;
    if (i < npc) cc.pd = pc[i];
    else cc.pd = load_cg(&cc.sd.passes[i]);
  };
  if (cc.P >= 0 && t >= cc.pd.task_base) {
    if (t < (unsigned long long)cc.pd.task_base + cc.pd.ntasks) return true;
    if (cc.P + 1 >= cc.sd.npasses) return false;
    if (t < tend(cc.P + 1)) {
      take_pass(cc.P + 1);
      return true;
    }
  }
  const int last = cc.sd.npasses - 1;
  if (t >= tend(last)) {
    take_pass(last);
    return false;
  }
  int lo = 0, hi = last;  // the pass with the largest task_base <= t
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tbase(mid) <= t) lo = mid;
    else hi = mid - 1;
  }
  take_pass(lo);
  return true;
}

// Mark the slot's task sequence used up, for the code of generation gen only.
__device__ __forceinline__ void mark_exhausted(const CtlStatic &cs, int s, unsigned long long gen) {
  const uint32_t g = slot_flag_gen(gen);
  atomicCAS(&cs.slot_flags[s], g, g | kSlotExhausted);
}

// Thread 0: take up the descriptor of slot s (coherent loads: the host
// rewrites it between codes); no pass is cached for it yet.
__device__ __forceinline__ void refresh_desc(ClaimCache &cc, const SlotDesc *slots, int s) {
  cc.sd = load_cg(&slots[s]);
  cc.gen = cc.sd.seq & kGenMask;
  cc.P = -1;
}

// Serving: a claim enters the slot before it reads the finished flag and
// leaves it after its task's last write.  With the full fences on both
// sides (here and in conclude), either the claim sees the code finished or
// the concluding CTA sees the claim in flight and waits for it: no task of
// a code writes into a slot after the code's completion is posted, so the
// host may hand the slot to the next code at once.
__device__ __forceinline__ void slot_enter(const CtlStatic &cs, int s) {
  if (cs.inflight) {
    atomicAdd(&cs.inflight[s * kInflightStride], 1u);
    __threadfence();
  }
}
__device__ __forceinline__ void slot_leave(const CtlStatic &cs, int s) {
  if (cs.inflight) atomicSub(&cs.inflight[s * kInflightStride], 1u);
}

// Thread 0: fill in the claim of task t (global index, already located in
// cc.P) of slot s.  A task the skip rule drops needs no work; every later
// task of the pass is then droppable too, so the rest of the pass is taken
// in the same claim by compare-and-swap on the code's own generation.
template <class SC>
__device__ __forceinline__ void take(SlotState *st, const KParams &kp, bool serve, int s, unsigned long long w,
                                    uint64_t key, Claim *o, ClaimCache &cc, SC &sc, const fpenum::BinomCols &B) {
  const unsigned long long t = w & kTaskMask;  // a slice of a pass numbers its tasks from task_off
  // the bound: the best recorded weight, else n - k + 2 (the skip rule uses
  // this one: it needs a recorded key); the g = 1 passes' least weight
  // (known before the search) caps the bound the task filters against, so
  // the tasks that start at once filter against it.  No key stands behind
  // the cap until the g = 1 passes record it.
  const int Ukey = key == kNoKey ? cc.sd.n - cc.sd.k + 2 : (int)key_weight(key);
  const int U = cc.sd.seed_u > 0 ? min(Ukey, cc.sd.seed_u) : Ukey;
  const int mid = kp.mid_pass < 0 ? cc.sd.mid_pass_exit : kp.mid_pass;
  o->task = t - cc.pd.task_base + cc.pd.task_off;
  o->lsplit = 0;
  if (cc.pd.g > 1 && cc.pd.nseg > 0) {
    // pair-leaf pass: its segments from the CTA's copy of the whole list,
    // else copied for this pass (eight loads in flight at a time)
    const PairSeg *segs = sc.seg;
    if (sc.slot == s && sc.gen == cc.gen && sc.pass == -2) {
      segs += cc.pd.seg_off;
    } else if (sc.slot != s || sc.gen != cc.gen || sc.pass != cc.P) {
      const uint2 *src = reinterpret_cast<const uint2 *>(cc.sd.passes + cc.sd.npasses) + cc.pd.seg_off;
      const int n = min((int)cc.pd.nseg, kSegPass);
      for (int i0 = 0; i0 < n; i0 += 8) {
        uint2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (i0 + u < n) v[u] = __ldcg(src + i0 + u);
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (i0 + u < n) reinterpret_cast<uint2 *>(sc.seg)[i0 + u] = v[u];
      }
      sc.slot = s;
      sc.gen = cc.gen;
      sc.pass = cc.P;
    }
    int ls = 0, spg = 1;
    pair_task(cc.pd, segs, cc.sd.k, B, o->task, &o->ulo, &o->uhi, &ls, &spg);
    o->lsplit = ls | (spg << 4);
  } else if (cc.pd.g > 1) {
    task_range(cc.pd, o->task, &o->ulo, &o->uhi);
  } else {
    o->ulo = o->task;
    o->uhi = o->task + 1;
  }
  o->slot = s;
  o->pass = cc.P;
  o->U = U;
  // Early exit inside a pass: sound only if the best codeword comes from
  // this pass or an earlier one (passes run ahead of the termination test).
  o->skip = (mid && key != kNoKey && (int)key_pass(key) <= cc.P && Ukey <= cc.pd.L_before) ? 1 : 0;
  o->ndone = 1;
  if (o->skip && !serve && !cc.sd.per_round_check && (int)key_pass(key) < cc.P) {
    // With a test after every pass, a best codeword from a pass before P
    // with U <= L_before(P) = L_after(P - 1) means the test after pass P - 1
    // certifies the code, so no pass from P on is ever tested: the rest of
    // the sequence is dropped, uncounted, by setting a bit above every task
    // index (32-bit; the counter's field has 40 bits).  A one-shot launch
    // never reuses the slot, so the bit cannot reach another code's counter.
    atomicOr(&st->word, 1ull << 32);
    o->ndone = 0;
  } else if (o->skip) {
    const unsigned long long end = (unsigned long long)cc.pd.task_base + cc.pd.ntasks;
    unsigned long long cur = w + 1;
    for (int tries = 0; tries < 4; ++tries) {
      if ((cur >> kGenShift) != cc.gen || (cur & kTaskMask) >= end) break;
      const unsigned long long want = cur - (cur & kTaskMask) + end;
      const unsigned long long prev = atomicCAS(&st->word, cur, want);
      if (prev == cur) {
        o->ndone += (unsigned int)(end - (cur & kTaskMask));
        break;
      }
      cur = prev;
    }
  }
}

// Thread 0: claim the next task of any live code.
template <class SC>
__device__ __forceinline__ int claim(const SlotDesc *slots, SlotState *states, const CtlStatic &cs,
                                     const KParams &kp, CtlDyn *cd, int &rr, unsigned long long &wait_t0,
                                     unsigned long long t_start, Claim *o, ClaimCache &cc, SC &sc,
                                     const PassDesc *pc, int npc, const fpenum::BinomCols &B) {
  const int nslots = cs.nslots;
  unsigned long long now = globaltimer();
  if (kp.timeout_ns && now - t_start > kp.timeout_ns) {
    atomicExch(&cd->err, 2);
    return kCmdExit;
  }
  // serving: once one CTA has decided the kernel retires, all leave at their
  // next claim, so that no code that arrives meanwhile runs on a shrinking
  // grid (the host launches the kernel again for it)
  if (cs.serve && ld_vol(&cd->leaving)) return kCmdExit;
  // Fast path: the slot served last, descriptors cached.  The task counter,
  // the finished flag and the best key are read in one round trip.  A task
  // taken from a code that has finished is dropped (nothing is left to
  // count for it); one taken from a newer code in the slot is run.  Both
  // paths end in the one call of take() below.
  int got = -1;  // the slot of the task taken
  unsigned long long w = 0;
  uint64_t key = kNoKey;
  if (kp.lookahead && cc.slot >= 0 && cc.P >= 0) {
    const int s = cc.slot;
    SlotState *st = &states[s];
    w = atomicAdd(&st->word, 1ull);
    slot_enter(cs, s);
    int fin = ld_vol(&st->finished);
    key = best_key(st);
    if ((w >> kGenShift) != cc.gen) {
      __threadfence();  // the descriptor was written before the state was reset
      refresh_desc(cc, slots, s);
      fin = ld_vol(&st->finished);
      key = best_key(st);
    }
    if ((w >> kGenShift) == cc.gen && cc.sd.npasses > 0 && fin != fin_tag(cc.gen)) {
      if (locate(cc, pc, npc, w & kTaskMask)) got = s;
      else mark_exhausted(cs, s, cc.gen);
    }
    if (got < 0) slot_leave(cs, s);
  }
  bool live = false;
  // four slot flags per load, from the group of the slot served last
  const int ngroups = (nslots + 3) >> 2;
  int q = rr >> 2;
  for (int qi = 0; qi < ngroups && got < 0; ++qi, ++q) {
    if (q >= ngroups) q = 0;
    const uint4 f4 = __ldcg(reinterpret_cast<const uint4 *>(cs.slot_flags) + q);
#pragma unroll 1
    for (int b = 0; b < 4; ++b) {
      const int s = 4 * q + b;
      if (s >= nslots) break;
      const uint32_t fl = b == 0 ? f4.x : b == 1 ? f4.y : b == 2 ? f4.z : f4.w;
      if (fl & (kSlotFinished | kSlotExhausted)) continue;
      SlotState *st = &states[s];
      if (ld_vol(&st->finished)) continue;
      w = ld_vol(&st->word);
      const unsigned long long wgen = w >> kGenShift;
      if (cc.slot != s || cc.gen != wgen) {
        __threadfence();  // the descriptor was written before the state was reset
        cc.slot = s;
        refresh_desc(cc, slots, s);
      }
      if (cc.sd.npasses <= 0) continue;
      live = true;
      if (wgen != cc.gen) continue;  // slot in transition between two codes
      if (!locate(cc, pc, cc.slot == 0 ? npc : 0, w & kTaskMask)) {  // every task handed out
        mark_exhausted(cs, s, wgen);
        continue;
      }
      if (!kp.lookahead && cc.P > ld_vol(&st->frontier)) continue;  // one pass at a time
      w = atomicAdd(&st->word, 1ull);
      slot_enter(cs, s);
      if ((w >> kGenShift) != cc.gen) {
        // the slot now holds a newer code; its descriptor was written before
        // its state, so re-reading it gives the code this task belongs to
        __threadfence();
        refresh_desc(cc, slots, s);
        if (cc.gen != (w >> kGenShift)) {
          slot_leave(cs, s);
          continue;
        }
      }
      if (!locate(cc, pc, cc.slot == 0 ? npc : 0, w & kTaskMask)) {
        mark_exhausted(cs, s, cc.gen);
        slot_leave(cs, s);
        continue;
      }
      if (ld_vol(&st->finished) == fin_tag(cc.gen)) {  // concluded since the check above: nothing to do
        slot_leave(cs, s);
        continue;
      }
      key = best_key(st);
      got = s;
      break;
    }
  }
  if (got >= 0) {
    take(&states[got], kp, cs.serve != 0, got, w, key, o, cc, sc, B);
    rr = got;
    wait_t0 = 0;
    cc.sleep_ns = 128;
    return kCmdRun;
  }
  if (!live && !cs.serve) return kCmdExit;
  if (ld_vol(&cd->err)) return kCmdExit;
  if (wait_t0 == 0) {
    wait_t0 = now;
  } else if (live) {
    if (now - wait_t0 > kp.wait_limit_ns) {
      atomicExch(&cd->err, 1);
      return kCmdExit;
    }
  } else {
    // serving, nothing to do: the kernel leaves once no CTA has found work
    // for the idle limit, all CTAs together (a CTA leaving on its own idle
    // time would shrink the kernel while a few CTAs keep taking the small
    // codes, and a large code arriving then ran on those few)
    const unsigned long long busy = ld_vol(&cd->last_busy);
    const unsigned long long since = busy > wait_t0 ? busy : wait_t0;
    if (now > since && now - since > kp.idle_limit_ns) {
      atomicExch(&cd->leaving, 1);
      return kCmdExit;
    }
  }
  __nanosleep(cc.sleep_ns);  // back off: idle probes must not crowd the state's cache lines
  if (cc.sleep_ns < 4096) cc.sleep_ns <<= 1;
  return kCmdWait;
}

constexpr int kFrontierDone = 1 << 30;  // frontier value once the code is concluded

// Finish the code: certified at pass sp, or out of passes.
__device__ __forceinline__ void conclude(const CtlStatic &cs, const KParams &kp, CtlDyn *cd, const SlotDesc &sd,
                                        SlotState *st, SlotAux *ax, int slot, int sp, bool certified) {
  int status = (certified || sd.complete) ? 0 : 4 /* FPCODE_EBUDGET */;
  unsigned long long entered = 0;
  for (int P = 0; P <= sp; ++P) entered += atomicAdd(&ax->pass_count[P], 0ull);
  const uint64_t key = ~(uint64_t)atomicOr(&st->best_key, 0ull);
  st->entered = entered;
  st->stop_pass = sp;
  st->status = kDoneFlag | status;
  fence_acq_rel();  // release: the outcome before the flag
  atomicExch(&st->finished, fin_tag(sd.seq));
  atomicOr(&cs.slot_flags[slot], kSlotFinished);
  if (cs.inflight) {
    // serving: wait until no other claim of this slot is in flight (this
    // CTA's own is the one left).  Tasks that ran ahead stop within 16 Gray
    // steps of reading the flag; claims made from now on see it and leave
    // without a write.  Only then is the outcome posted, and the host may
    // hand the slot to the next code.  Bounded: past the wait limit the
    // code reports a timeout and the host keeps the slot until the kernel
    // has exited.
    __threadfence();
    const unsigned long long t0 = globaltimer();
    while (*(volatile const uint32_t *)&cs.inflight[slot * kInflightStride] > 1u) {
      if (globaltimer() - t0 > kp.wait_limit_ns) {
        status = 5;  // FPCODE_ETIMEOUT
        atomicExch(&cd->err, 1);
        break;
      }
      __nanosleep(256);
    }
  }
  if (cs.done_host) {  // serving: post the outcome; the host may reuse the slot after seq
    Completion *c = cs.done_host + slot;
    c->best_key = key;
    c->enumerated = entered;
    c->status = status;
    c->stop_pass = sp;
    __threadfence_system();
    *(volatile unsigned long long *)&c->seq = sd.seq;
  }
}

// Thread 0 counts a finished task of pass P off.  Passes complete in any
// order; whoever sees the frontier pass complete applies its termination
// test (Alg. 6) with the least weight recorded in it and the passes before
// it, and moves the frontier on.  Two CTAs may test the same pass: they
// read the same final values and write the same results, and the
// compare-and-swap on the frontier lets exactly one move it.
//
// The count-off itself: a release add, so that the task's records and
// counts (made before it, by this thread or, through the CTA barrier, by
// the others) are seen by whoever finds the pass complete.  Returns the
// tasks of pass P done with this one.
__device__ __forceinline__ unsigned int count_off(SlotAux *ax, int P, unsigned int ndone) {
  unsigned int old;
  asm volatile("atom.release.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(&ax->pass_done[P]), "r"(ndone) : "memory");
  return old + ndone;
}

// Termination tests from the frontier on, after a count-off that completed
// pass P (see finish_task).  Returns true when this call concluded the code.
//
// One round of the walk reads the counts of the next kWalk passes at once
// (and, after an acquire fence, their least weights), tests every complete
// pass of them in order, and moves the frontier past them with one
// compare-and-swap (a test per pass in its own round takes seven dependent
// round trips, and a CTA that finds several passes complete holds up its
// CTA for tens of microseconds).  Fences keep the two orders the protocol
// rests on:
// a count-off before the completer's read of the frontier, and a move of
// the frontier before the mover's next read of the counts (so that of two
// CTAs racing there, one sees the other's write).
constexpr int kWalk = 4;

__device__ __forceinline__ bool test_frontier(const CtlStatic &cs, const KParams &kp, CtlDyn *cd, const SlotDesc &sd,
                                              SlotState *st, SlotAux *ax, int slot, int P, const PassDesc &pd,
                                              const PassDesc *pc, int npc) {
  int f = -1;      // the frontier, once read or moved by this call
  int useq = 0;    // the bound after pass f - 1, once known
  for (;;) {
    __threadfence();  // store-then-load: the count-off (or the move) before the reads below
    int fin;
    if (f < 0) {
      f = ld_vol(&st->frontier);
      fin = ld_vol(&st->finished);
      fence_acq_rel();  // acquire: what the tester of pass f - 1 wrote before moving the frontier
    } else {
      fin = ld_vol(&st->finished);
    }
    if (f >= sd.npasses || fin) return false;
    const int n = min(kWalk, sd.npasses - f);
    uint32_t done[kWalk], nt[kWalk];
    int La[kWalk], re[kWalk];
#pragma unroll
    for (int i = 0; i < kWalk; ++i) {
      done[i] = 0;
      nt[i] = 1;
      La[i] = 0;
      re[i] = 0;
      if (i < n) {
        done[i] = (uint32_t)ld_vol(reinterpret_cast<const int32_t *>(&ax->pass_done[f + i]));
        if (f + i == P) {
          nt[i] = pd.ntasks;
          La[i] = pd.L_after;
          re[i] = pd.round_end;
        } else if (f + i < npc) {
          nt[i] = pc[f + i].ntasks;
          La[i] = pc[f + i].L_after;
          re[i] = pc[f + i].round_end;
        } else {
          nt[i] = __ldcg(&sd.passes[f + i].ntasks);
          La[i] = __ldcg(&sd.passes[f + i].L_after);
          re[i] = __ldcg(&sd.passes[f + i].round_end);
        }
      }
    }
    if (useq == 0) {
      const int u0 = f > 0 ? ld_vol(&ax->useq_after[f - 1]) : 0;
      useq = u0 ? u0 : sd.n - sd.k + 2;
    }
    if (done[0] != nt[0]) return false;  // the frontier pass is still running
    fence_acq_rel();  // acquire: the records of the passes seen complete
    int pm[kWalk];
#pragma unroll
    for (int i = 0; i < kWalk; ++i) pm[i] = i < n && done[i] == nt[i] ? ld_vol(&ax->pass_min[f + i]) : 0;
    int j = 0;
#pragma unroll
    for (int i = 0; i < kWalk; ++i) {
      if (i != j || i >= n || done[i] != nt[i]) continue;  // stop at the first pass still running
      if (pm[i]) useq = min(useq, 256 - pm[i]);
      if (sd.pass_times) sd.pass_times[f + i] = globaltimer();
      const bool check = !sd.per_round_check || re[i];
      const bool certified = check && La[i] >= useq;
      if (certified || f + i + 1 >= sd.npasses) {
        // the frontier jumps past every pass, so no later pass is ever tested
        if (atomicCAS(&st->frontier, f, kFrontierDone) != f) return false;
        conclude(cs, kp, cd, sd, st, ax, slot, f + i, certified);
        return true;
      }
      ax->useq_after[f + i] = useq;  // a second tester writes the same value here
      ++j;
    }
    fence_acq_rel();  // release: the bounds before the move
    if (atomicCAS(&st->frontier, f, f + j) != f) return false;  // another CTA moved it
    f += j;
  }
}

// Returns true when this count-off concluded the code.
__device__ __forceinline__ bool finish_task(const CtlStatic &cs, const KParams &kp, CtlDyn *cd, const SlotDesc &sd,
                                            SlotState *st, SlotAux *ax, int slot, int P, const PassDesc &pd,
                                            unsigned int ndone, const PassDesc *pc, int npc) {
  return count_off(ax, P, ndone) == pd.ntasks && test_frontier(cs, kp, cd, sd, st, ax, slot, P, pd, pc, npc);
}


#ifndef FPK_MIN_BLOCKS
#define FPK_MIN_BLOCKS 4  // CTAs per SM the register allocation is capped for
#endif

template <class V>
__global__ void __launch_bounds__(kThreads, FPK_MIN_BLOCKS) bz_kernel(const SlotDesc *__restrict__ slots, SlotState *states,
                                                      const CtlStatic *__restrict__ ctl, CtlDyn *cdyn,
                                                      KParams kp) {
  extern __shared__ uint4 smem_raw[];
  uint64_t *bcols = reinterpret_cast<uint64_t *>(smem_raw);  // binomial columns t < kBinomCols
  uint4 *tab4 = smem_raw + kBinomBytes / 16;
  uint32_t *tab = reinterpret_cast<uint32_t *>(tab4);
  __shared__ Claim s_cl;
  __shared__ ClaimCache s_cc;
  __shared__ SegCache<V::kSegCache> s_sc;
  __shared__ __align__(16) PassDesc s_pc[V::kPassCache];  // copied in 16-byte pieces
  __shared__ int s_npc;
  __shared__ int s_cmd, s_stage;
  __shared__ int s_over;  // one-code launch: this CTA concluded the code, so it leaves without a claim
  __shared__ unsigned long long s_count, s_staged_seq;
  __shared__ int s_staged_slot, s_staged_j;

  const CtlStatic cs = *ctl;
  const int tid = threadIdx.x;
  int rr = (int)(blockIdx.x % (unsigned)(cs.nslots > 0 ? cs.nslots : 1));
  unsigned long long wait_t0 = 0;
  const unsigned long long t_start = globaltimer();
  if (tid == 0) {
    s_staged_slot = -1;
    s_staged_j = -1;
    s_staged_seq = 0;
    s_cc.slot = -1;
    s_cc.P = -1;
    s_cc.gen = 0;
    s_cc.sleep_ns = 128;
    s_cc.busy_note = 0;
    s_sc.slot = -1;
    s_sc.pass = -1;
    s_sc.gen = 0;
    s_npc = 0;
    s_over = 0;
  }
  {
    static_assert(kBinomBytes == sizeof(cs.binom->cols), "staged binomial columns");
    const uint4 *bsrc = reinterpret_cast<const uint4 *>(cs.binom->cols);
    for (int i = tid; i < kBinomBytes / 16; i += kThreads) smem_raw[i] = __ldg(bsrc + i);
  }
  const fpenum::BinomCols binom{bcols};
  if (blockIdx.x == 0 && tid == 0 && cs.nslots == 1) {
    const SlotDesc sd0 = load_cg(&slots[0]);
    if (sd0.pass_times) sd0.pass_times[kMaxPasses] = t_start;  // launch start
  }
  if (cs.nslots == 1 && !cs.serve) {
    // One code: its descriptor, its pass descriptors (when they fit) and
    // its pair-leaf segments are staged once, so the first claim already
    // takes the fast path and locates its pass in shared memory.  Nothing
    // in the launch writes them, so they are read through L1, and the slot
    // descriptor by one thread: every CTA reads the same bytes at once, and
    // an L2 load per warp of the grid queues thousands of requests on one
    // line (several microseconds before the first claim).
    if (tid == 0) s_cc.sd = load_nc(&slots[0]);
    __syncthreads();
    const int np = s_cc.sd.npasses, nsegs = s_cc.sd.nsegs;
    const PassDesc *passes = s_cc.sd.passes;
    const unsigned long long gen = s_cc.sd.seq & kGenMask;
    const int npc = np < V::kPassCache ? np : V::kPassCache;  // the first passes: where every CTA starts
    {
      const uint4 *src = reinterpret_cast<const uint4 *>(passes);
      for (int i = tid; i < npc * (int)(sizeof(PassDesc) / 16); i += kThreads)
        reinterpret_cast<uint4 *>(s_pc)[i] = __ldg(src + i);
    }
    if constexpr (V::kSegCache > kSegPass) {
      if (nsegs > 0 && nsegs <= V::kSegCache) {
        const uint2 *src = reinterpret_cast<const uint2 *>(passes + np);
        for (int i = tid; i < nsegs; i += kThreads) reinterpret_cast<uint2 *>(s_sc.seg)[i] = __ldg(src + i);
        if (tid == 0) {
          s_sc.slot = 0;
          s_sc.gen = gen;
          s_sc.pass = -2;
        }
      }
    }
    __syncthreads();
    if (tid == 0) {
      s_cc.slot = 0;
      s_cc.gen = gen;
      s_cc.P = -1;
      s_npc = npc;
      if (np > 0) {
        s_cc.pd = npc ? s_pc[0] : load_nc(&passes[0]);
        s_cc.P = 0;
      }
    }
  }
  __syncthreads();
  for (;;) {
    if (tid == 0) {
      const int cmd =
          s_over ? kCmdExit : claim(slots, states, cs, kp, cdyn, rr, wait_t0, t_start, &s_cl, s_cc, s_sc, s_pc, s_npc, binom);
      s_cmd = cmd;
      if (cmd == kCmdRun && cs.serve) {  // keep the serving kernel whole (at most one note per 0.5 ms)
        const unsigned long long now = globaltimer();
        if (now - s_cc.busy_note > 500000ull) {
          atomicMax(&cdyn->last_busy, now);
          s_cc.busy_note = now;
        }
      }
      if (cmd == kCmdRun) {
        s_stage = (!s_cl.skip && (s_cl.slot != s_staged_slot || s_cc.pd.j != s_staged_j ||
                                  s_cc.sd.seq != s_staged_seq)) ? 1 : 0;
        if (s_stage) {
          s_staged_slot = s_cl.slot;
          s_staged_j = s_cc.pd.j;
          s_staged_seq = s_cc.sd.seq;
        }
      }
      s_count = 0;
    }
    __syncthreads();
    const int cmd = s_cmd;
    if (cmd == kCmdExit) break;
    if (cmd == kCmdWait) {
      __syncthreads();
      continue;
    }
    const int slot = s_cl.slot;
    if (s_stage) {
      // eight loads in flight per thread before their stores: one L2 round
      // trip per 32 KiB instead of one per 4 KiB
      const int words = table_words(s_cc.sd);
      const int nv = words / 4;
      const uint4 *src = reinterpret_cast<const uint4 *>(s_cc.sd.table + (size_t)s_cc.pd.j * (size_t)words);
      for (int i0 = tid; i0 < nv; i0 += 8 * kThreads) {
        uint4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (i0 + u * kThreads < nv) v[u] = __ldcg(src + i0 + u * kThreads);
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (i0 + u * kThreads < nv) tab4[i0 + u * kThreads] = v[u];
      }
      __syncthreads();
      if (s_cc.sd.pair_sigp > 0) {
        V::stage_pairs(tab, s_cc.sd);
        __syncthreads();
      }
    }
    unsigned long long count = 0;
    SlotAux *ax = cs.aux + slot;
    if (!s_cl.skip)
      V::run(s_cc.sd, s_cc.pd, s_cl.pass, tab, binom, s_cl.ulo, s_cl.uhi, s_cl.lsplit, s_cl.U, &states[slot], ax, count);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) count += __shfl_xor_sync(0xffffffffu, count, o);
    if ((tid & 31) == 0 && count) atomicAdd(&s_count, count);
    __syncthreads();
    if (tid == 0) {
      if (s_count) {
        atomicAdd(&states[slot].enumerated, s_count);
        atomicAdd(&ax->pass_count[s_cl.pass], s_count);
      }
      if (finish_task(cs, kp, cdyn, s_cc.sd, &states[slot], ax, slot, s_cl.pass, s_cc.pd, s_cl.ndone, s_pc, s_npc) &&
          cs.nslots == 1 && !cs.serve)
        s_over = 1;
      if (cs.inflight) {
        __threadfence();  // the task's writes before it leaves the slot
        slot_leave(cs, slot);
      }
    }
  }
  if (cs.outcome) {
    // One-code launch: the last CTA to leave copies the final state (the
    // outcome and the count of every CTA's codewords) to host-mapped memory
    // and zeroes the dynamic state, so the next search of the code needs no
    // reset and its result no copy of its own.
    __shared__ int s_last;
    if (tid == 0) {
      fence_acq_rel();  // release: this CTA's writes before its count
      s_last = atomicAdd(&cdyn->exited, 1u) == gridDim.x - 1 ? 1 : 0;
      if (s_last) fence_acq_rel();  // acquire: every CTA's writes
    }
    __syncthreads();
    if (s_last) {
      const uint4 *src = reinterpret_cast<const uint4 *>(states);
      uint4 *dst = reinterpret_cast<uint4 *>(cs.outcome);
      for (int i = tid; i < (int)(cs.dyn_bytes / 16); i += kThreads) dst[i] = __ldcg(src + i);
      __syncthreads();
      uint4 *z = reinterpret_cast<uint4 *>(states);
      for (int i = tid; i < (int)(cs.clean_bytes / 16); i += kThreads) z[i] = make_uint4(0u, 0u, 0u, 0u);
    }
  }
}

}  // namespace fpk
