// fp_enum.cuh -- enumeration order of one Brouwer-Zimmermann pass.
//
// A pass (g, j) visits every codeword sum_{t in T} c_t Gamma_j[t] with
// |T| = g and every c_t in [1, p), normalised projectively (Sec. 4.2): of
// the p-1 nonzero multiples of a codeword only one is visited.  Here the
// normalised coefficient is that of the SECOND largest row of T (any fixed
// row works, since scalar multiples have equal weight).
//
// For g >= 2 the rows of T split into
//   leaf   x = max T                      coefficient c_x in [1, p)
//   prefix P = T \ {x}, with max m < x    coefficient of m fixed to 1
//          Q = P \ {m}, |Q| = g - 2       coefficients in [1, p)
// The GPU keeps the exact bit-sliced sum S of the prefix in registers and
// evaluates every leaf (x, c_x) against it without forming the sum (the
// isometric last addition of Sec. 4.3).
//
// Prefixes of a pass are numbered I = 0 .. C(k-1, g-1)(p-1)^(g-2) - 1 in
// this order: by m ascending; within m by the revolving-door rank of Q among
// the (g-2)-subsets of {0..m-1}; within Q by the reflected (p-1)-ary Gray
// code of the coefficient vector.  Walking I -> I+1 changes one coefficient
// by +-1 (one exact row add) except where Q or m changes.
//
// Revolving-door order of t-subsets of {0..n-1} (Nijenhuis-Wilf; Kreher-
// Stinson): R(n,t) = R(n-1,t) followed by the reverse of R(n-1,t-1) with
// n-1 added to each subset.  Successive subsets differ by exchanging one
// element.  All functions are __host__ __device__.
#pragma once
#include <stdint.h>

#ifndef FP_HD
#if defined(__CUDACC__)
#define FP_HD __host__ __device__ __forceinline__
#else
#define FP_HD inline
#endif
#endif

namespace fpenum {

constexpr int kMaxK = 64;

// Columns t < kBinomCols of the table are all the enumeration needs on the
// GPU (t <= g - 2 and g is capped well below 26).
constexpr int kBinomCols = 24;

// Binomial table C(n, t), 0 <= t <= n <= 64 (C(64,32) < 2^63).  The
// enumeration functions take any accessor B with B(n, t) = C(n, t).  The
// first kBinomCols columns are stored a second time, t-major, so that a
// CTA copies them into shared memory with plain coalesced 16-byte loads.
struct Binom {
  uint64_t cols[kBinomCols][kMaxK + 1];  // cols[t][n] = C(n, t); 12480 bytes, a multiple of 16
  uint64_t c[kMaxK + 1][kMaxK + 1];
  FP_HD uint64_t operator()(int n, int t) const { return c[n][t]; }
};

// Columns t < T of the table, stored t-major (shared memory on the GPU).
struct BinomCols {
  const uint64_t *p;  // p[t * (kMaxK + 1) + n]
  FP_HD uint64_t operator()(int n, int t) const { return p[t * (kMaxK + 1) + n]; }
};

inline void fill_binom(Binom *b) {
  for (int n = 0; n <= kMaxK; ++n)
    for (int t = 0; t <= kMaxK; ++t) b->c[n][t] = 0;
  for (int n = 0; n <= kMaxK; ++n) {
    b->c[n][0] = 1;
    for (int t = 1; t <= n; ++t) b->c[n][t] = b->c[n - 1][t - 1] + (t <= n - 1 ? b->c[n - 1][t] : 0);
  }
  for (int t = 0; t < kBinomCols; ++t)
    for (int n = 0; n <= kMaxK; ++n) b->cols[t][n] = b->c[n][t];
}

FP_HD int ctz64(uint64_t x) {
#if defined(__CUDA_ARCH__)
  return __ffsll((long long)x) - 1;
#else
  return __builtin_ctzll(x);
#endif
}

FP_HD int ctz32(uint32_t x) {
#if defined(__CUDA_ARCH__)
  return __ffs((int)x) - 1;
#else
  return __builtin_ctz(x);
#endif
}

FP_HD int popc64(uint64_t x) {
#if defined(__CUDA_ARCH__)
  return __popcll(x);
#else
  return __builtin_popcountll(x);
#endif
}

FP_HD uint64_t low_mask(int n) { return n >= 64 ? ~0ull : ((1ull << n) - 1ull); }

// Subset of rank r in R(n, t), as a bit mask over {0..n-1}.  Top down, a
// level n whose element n-1 is not a member keeps the rank (the subset lies
// in the first half, R(n-1, t)); the largest member is therefore the largest
// x with C(x, t) <= r, found by bisection (C(x, t) grows with x, and
// C(t-1, t) = 0), and the rest is the subset of rank C(x+1, t) - 1 - r in
// R(x, t-1) (the reflected second half).
template <class BT>
FP_HD uint64_t rd_unrank(const BT &B, uint64_t r, int n, int t) {
  uint64_t mask = 0;
  while (t > 0) {
    int lo = t - 1, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (B(mid, t) <= r) lo = mid;
      else hi = mid - 1;
    }
    mask |= 1ull << lo;
    r = B(lo + 1, t) - 1 - r;
    n = lo;
    --t;
  }
  return mask;
}

// Rank of subset T (|T| = t) in R(n, t).
template <class BT>
FP_HD uint64_t rd_rank(const BT &B, uint64_t T, int n, int t) {
  // Walk from the top; each member n-1 reflects the rank of the rest.
  int flip = 0;  // parity of reflections so far
  uint64_t off = 0;
  // r(T, n, t) = n-1 in T ? C(n,t) - 1 - r(T', n-1, t-1) : r(T, n-1, t)
  // unrolled as an affine map r = off + (flip ? -1 : 1) * r_rest
  while (t > 0 && t < n) {
    if (T >> (n - 1) & 1ull) {
      uint64_t base = B(n, t) - 1;
      // r = base - r_rest, composed with the current map
      if (!flip) off = off + base; else off = off - base;
      flip ^= 1;
      --t;
    }
    --n;
  }
  return off;  // the innermost rank (base case) is 0
}

// Successor of T in R(n, t).  Returns false if T is the last subset.  On
// success *out gets the next subset, *removed / *added the exchanged rows.
//
// Derivation: following the recursive definition from the top element
// down, the successor is decided at the deepest level n' whose call can
// fall back to the other half of its list.  Level n' (element j = n'-1) can
// fall back iff the number of members of T in [j, n-1] is even, and levels
// are explored only above the base level b (the first level where the
// remaining subset is empty or full).  At that level, with t' members of T
// below n', the exchange is
//   j not in T:  remove (t' >= 2 ? t'-2 : n'-2), add j
//   j in T:      remove j, add (t' >= 2 ? t'-2 : n'-2).
FP_HD bool rd_next(uint64_t T, int n, int t, uint64_t *out, int *removed, int *added) {
  if (t <= 0 || t >= n) return false;
  int z = ctz64(~T);  // length of the initial run 0..z-1 inside T
  int mn = ctz64(T);  // smallest member
  int b = z > mn ? z : mn;
  uint64_t X = T;  // bit j of X = parity of the members >= j
  X ^= X >> 1;
  X ^= X >> 2;
  X ^= X >> 4;
  X ^= X >> 8;
  X ^= X >> 16;
  X ^= X >> 32;
  uint64_t cand = ~X & low_mask(n) & ~low_mask(b);
  if (!cand) return false;
  int j = ctz64(cand);
  int np = j + 1;
  int tp = popc64(T & low_mask(np));
  int other = tp >= 2 ? tp - 2 : np - 2;
  if (T >> j & 1ull) {
    *removed = j;
    *added = other;
  } else {
    *removed = other;
    *added = j;
  }
  *out = (T & ~(1ull << *removed)) | (1ull << *added);
  return true;
}

// ---------------------------------------------------------------------------
// Reflected b-ary Gray code (b = p - 1, even for odd p) on L digits.  The
// counter i has base-b digits d_s (s = 0 least significant); the Gray digit
// is e_s = d_s if d_{s+1} is even, else b-1-d_s (d_L = 0).  For even b only
// the digit above matters.  Stepping i -> i+1 changes exactly Gray digit s =
// the lowest counter digit below b-1, by +1 if d_{s+1} is even, else -1.
// Digits are packed DB bits each in a uint64_t.
// ---------------------------------------------------------------------------
template <int DB>
FP_HD int digit(uint64_t d, int s) {
  return (int)((d >> (s * DB)) & ((1ull << DB) - 1));
}

template <int DB>
FP_HD uint64_t counter_digits(uint64_t ci, int b, int L) {
  uint64_t d = 0;
  for (int s = 0; s < L; ++s) {
    d |= (uint64_t)(ci % (uint64_t)b) << (s * DB);
    ci /= (uint64_t)b;
  }
  return d;
}

// Gray digit s (coefficient of slot s minus one).
template <int DB>
FP_HD int gray_digit(uint64_t d, int s, int b, int L) {
  int ds = digit<DB>(d, s);
  int up = s + 1 < L ? digit<DB>(d, s + 1) : 0;
  return (up & 1) ? b - 1 - ds : ds;
}

// Advance the counter; returns the changed slot s and *dir = +1 / -1.
// Precondition: the counter is not at its last value.
template <int DB>
FP_HD int gray_step(uint64_t *d, int b, int L, int *dir) {
  if constexpr (DB == 1) {
    // b = 2: the counter is a binary number; its lowest 0 bit is the digit
    // that moves, and the 1 bits below it wrap to 0.  The schedule keeps
    // L = g - 2 below the staged binomial columns, so the counter fits 32
    // bits.
    const uint32_t d32 = (uint32_t)*d;
    const int s = ctz32(~d32);
    const uint32_t n32 = d32 + 1u;
    *d = n32;
    *dir = (s + 1 < L && ((n32 >> (s + 1)) & 1u)) ? -1 : 1;
    return s;
  } else if constexpr (DB == 4) {
    // nibble digits: the lowest digit below b - 1 moves; those below it
    // (all b - 1) wrap to 0
    const uint64_t x = *d ^ (0x1111111111111111ull * (uint64_t)(b - 1));  // zero nibble: digit b - 1
    const uint64_t nz = (x | (x >> 1) | (x >> 2) | (x >> 3)) & 0x1111111111111111ull;
    const int s = ctz64(nz) >> 2;
    const uint64_t low = s == 0 ? 0ull : ((1ull << (4 * s)) - 1);
    *d = (*d & ~low) + (1ull << (4 * s));
    *dir = (s + 1 < L && ((*d >> (4 * (s + 1))) & 1ull)) ? -1 : 1;
    return s;
  }
  int s = 0;
  while (digit<DB>(*d, s) == b - 1) ++s;
  uint64_t keep = (s + 1) * DB >= 64 ? 0ull : (*d >> ((s + 1) * DB)) << ((s + 1) * DB);
  int v = digit<DB>(*d, s) + 1;
  *d = keep | ((uint64_t)v << (s * DB));
  int up = s + 1 < L ? digit<DB>(*d, s + 1) : 0;
  *dir = (up & 1) ? -1 : 1;
  return s;
}

// ---------------------------------------------------------------------------
// Prefix index I <-> (m, Q, coefficient counter) within pass g >= 2.
// ---------------------------------------------------------------------------
FP_HD uint64_t ipow(uint64_t b, int e) {
  uint64_t r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// Number of prefixes of pass g >= 2 whose largest row is below m:
// sum_{m' < m} C(m', g-2) NC = C(m, g-1) NC, NC = (p-1)^(g-2).
template <class BT>
FP_HD uint64_t prefixes_below(const BT &B, int m, int g, uint64_t NC) { return B(m, g - 1) * NC; }

struct Prefix {
  int m;        // largest row of the prefix (coefficient 1)
  uint64_t qi;  // revolving-door rank of Q among (g-2)-subsets of {0..m-1}
  uint64_t Q;   // mask of Q
  uint64_t d;   // counter digits of the coefficient vector of Q (slot order)
};

template <int DB, class BT>
FP_HD Prefix prefix_unrank(const BT &B, uint64_t I, int k, int g, int b) {
  const int L = g - 2;
  const uint64_t NC = ipow((uint64_t)b, L);
  // largest m in [g-2, k-2] with C(m, g-1) NC <= I (binary search)
  int lo = g - 2, hi = k - 2;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (prefixes_below(B, mid, g, NC) <= I) lo = mid; else hi = mid - 1;
  }
  Prefix P;
  P.m = lo;
  uint64_t rem = I - prefixes_below(B, lo, g, NC);
  uint64_t ci;
  if constexpr (DB == 1) {  // b = 2: NC = 2^L
    P.qi = rem >> L;
    ci = rem & (NC - 1);
  } else {
    P.qi = rem / NC;
    ci = rem - P.qi * NC;
  }
  P.Q = rd_unrank(B, P.qi, P.m, L);
  P.d = counter_digits<DB>(ci, b, L);
  return P;
}

// Step a prefix from index I to I + 1 (precondition: I + 1 is still a
// prefix of the pass).  ci is the coefficient counter value, nq the number
// of subsets C(m, g-2).  Returns the slot whose coefficient changed (by
// *dir = +1 or -1), or -1 if Q or m changed and the prefix sum must be
// rebuilt (all coefficients back to 1).
template <int DB, class BT>
FP_HD int prefix_advance(const BT &B, Prefix &pf, uint64_t &ci, uint64_t &nq, uint64_t NC, int b, int L,
                         int *dir) {
  if constexpr (DB == 1) {
    // b = 2: the packed digits are the counter itself (ci is not kept)
    if (pf.d + 1 < NC) return gray_step<DB>(&pf.d, b, L, dir);
  } else {
    if (ci + 1 < NC) {
      int s = gray_step<DB>(&pf.d, b, L, dir);
      ++ci;
      return s;
    }
  }
  ci = 0;
  pf.d = 0;
  if (pf.qi + 1 < nq) {
    uint64_t nQ = pf.Q;
    int rm = 0, ad = 0;
    rd_next(pf.Q, pf.m, L, &nQ, &rm, &ad);
    pf.Q = nQ;
    ++pf.qi;
  } else {
    ++pf.m;
    pf.qi = 0;
    pf.Q = low_mask(L);
    nq = B(pf.m, L);
  }
  return -1;
}

// Row of slot s of Q (the s-th smallest member).
FP_HD int nth_member(uint64_t Q, int s) {
  for (int i = 0; i < s; ++i) Q &= Q - 1;
  return ctz64(Q);
}

}  // namespace fpenum
