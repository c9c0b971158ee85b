// fp_bitslice.cuh -- F_p arithmetic on bit-sliced words (natural binary
// encoding, sliced-bit storage).
//
// A vector of 32 symbols of F_p is held as r = floor(log2 p) + 1 words
// ("slices"): bit q of slice i is bit i of the natural binary expansion of
// symbol q (Sec. 2, storage example (2,0,1) -> ((0,0,1),(1,0,0))).  Every
// operation below is lane-wise over the 32 bit positions, so the same code
// serves 32 symbols at once.  Inputs must be canonical (each symbol in
// [0, p)); outputs are canonical.
//
// Functions are __host__ __device__ so that the host can check them
// exhaustively against (a + b) mod p and the GPU kernels can inline them.
#pragma once
#include <stdint.h>

#ifndef FP_HD
#if defined(__CUDACC__)
#define FP_HD __host__ __device__ __forceinline__
#else
#define FP_HD inline
#endif
#endif

namespace fpbs {

// Bits per symbol: r = floor(log2 p) + 1 (Sec. 2).
FP_HD int bits_for(int p) {
  int r = 0;
  while ((1 << r) <= p) ++r;
  return r;
}

// ---------------------------------------------------------------------------
// Exact addition, p = 3 (r = 2): Alg. 3, with its sixth line read as
// s0 = s0 xor carry_1 (the printed "and" gives wrong sums on 5 of the 9
// input pairs; xor gives all 9 right and keeps the paper's count of nine
// operations).  Natural encoding 0 = (0,0), 1 = (1,0), 2 = (0,1).
// ---------------------------------------------------------------------------
FP_HD void add_p3(uint32_t a0, uint32_t a1, uint32_t b0, uint32_t b1, uint32_t &s0, uint32_t &s1) {
  uint32_t x0 = a0 ^ b0;
  uint32_t c0 = a0 & b0;
  uint32_t x1 = a1 ^ b1 ^ c0;
  uint32_t c1 = a1 & b1;
  x0 = x0 ^ c1;
  uint32_t t = x0 & x1;  // (1,1) encodes 3 = 0 mod 3
  s0 = x0 ^ t;
  s1 = x1 ^ t;
}

// ---------------------------------------------------------------------------
// Exact addition, p = 7 (r = 3): Alg. 4 -- ripple add with the carry out of
// bit 2 added back at bit 0 (2^3 = 1 mod 7), then (1,1,1) -> (0,0,0).
// ---------------------------------------------------------------------------
FP_HD void add_p7(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t b0, uint32_t b1, uint32_t b2, uint32_t &s0,
                  uint32_t &s1, uint32_t &s2) {
  uint32_t x0 = a0 ^ b0;
  uint32_t c0 = a0 & b0;
  uint32_t x1 = a1 ^ b1 ^ c0;
  uint32_t c1 = (a1 & b1) | (a1 & c0) | (b1 & c0);
  uint32_t x2 = a2 ^ b2 ^ c1;
  uint32_t c2 = (a2 & b2) | (a2 & c1) | (b2 & c1);
  c0 = x0 & c2;  // end-around carry
  x0 = x0 ^ c2;
  c1 = x1 & c0;
  x1 = x1 ^ c0;
  x2 = x2 ^ c1;
  uint32_t t = x0 & x1 & x2;
  s0 = x0 ^ t;
  s1 = x1 ^ t;
  s2 = x2 ^ t;
}

// ---------------------------------------------------------------------------
// Exact addition for any odd prime p < 2^R: ripple-carry add to R+1 bits,
// subtract p, and keep the difference where it did not borrow.  This is the
// build's own form for p != 2^r - 1: Alg. 5 as printed leaves results in
// [p+1, 2^r) unreduced (e.g. 3 + 3 -> 6 for p = 5), so it is not used.
// a, b, s: R slices each.
// ---------------------------------------------------------------------------
template <int R>
FP_HD void add_generic(const uint32_t *a, const uint32_t *b, uint32_t *s, int p) {
  uint32_t sum[R + 1];
  uint32_t carry = 0;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    uint32_t x = a[i] ^ b[i];
    sum[i] = x ^ carry;
    carry = (a[i] & b[i]) | (x & carry);
  }
  sum[R] = carry;
  uint32_t diff[R + 1];
  uint32_t borrow = 0;
#pragma unroll
  for (int i = 0; i <= R; ++i) {
    uint32_t pb = ((p >> i) & 1) ? 0xFFFFFFFFu : 0u;  // bit i of p, splat
    uint32_t x = sum[i] ^ pb;
    diff[i] = x ^ borrow;
    borrow = (~sum[i] & pb) | (~x & borrow);
  }
  // borrow set: sum < p, keep sum; else keep sum - p
#pragma unroll
  for (int i = 0; i < R; ++i) s[i] = (borrow & sum[i]) | (~borrow & diff[i]);
}

// ---------------------------------------------------------------------------
// Exact addition for a Mersenne prime p = 2^R - 1 (p = 31, 127): the
// end-around-carry form (Alg. 1's reduction unrolled over the R slices, as
// Alg. 4 is for R = 3).  The R-bit ripple sum x of a and b leaves a carry c
// out of bit R - 1; 2^R = 1 mod p, so c is added back at bit 0.  That second
// ripple cannot carry out: c = 1 means a + b >= 2^R, so x = a + b - 2^R <=
// 2^R - 4.  Last, x = 2^R - 1 (all ones, only when a + b = p) is 0 mod p.
// ---------------------------------------------------------------------------
template <int R>
FP_HD void add_mersenne(const uint32_t *a, const uint32_t *b, uint32_t *s) {
  uint32_t x[R];
  uint32_t c = 0;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const uint32_t t = a[i] ^ b[i];
    x[i] = t ^ c;
    c = (a[i] & b[i]) | (t & c);
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {  // + the end-around carry
    const uint32_t t = x[i] & c;
    x[i] ^= c;
    c = t;
  }
  uint32_t ones = x[0];
#pragma unroll
  for (int i = 1; i < R; ++i) ones &= x[i];
#pragma unroll
  for (int i = 0; i < R; ++i) s[i] = x[i] ^ ones;
}

// Dispatch on a compile-time prime P (3 and 7 use Alg. 3 / Alg. 4, the
// Mersenne primes 31 and 127 the end-around-carry form).
template <int P, int R>
FP_HD void add_exact(const uint32_t *a, const uint32_t *b, uint32_t *s, int p) {
  if (P == 3) {
    add_p3(a[0], a[1], b[0], b[1], s[0], s[1]);
  } else if (P == 7) {
    add_p7(a[0], a[1], a[2], b[0], b[1], b[2], s[0], s[1], s[2]);
  } else if (P > 7 && P == (1 << R) - 1) {
    add_mersenne<R>(a, b, s);
  } else {
    add_generic<R>(a, b, s, P ? P : p);
  }
}

// ---------------------------------------------------------------------------
// Isometric subtraction (Sec. 4.3): a - b != 0 exactly where some slice
// differs, so the nonzero mask of a - b is OR_i (a_i xor b_i).  Valid for
// every p when both operands are canonical.
// ---------------------------------------------------------------------------
template <int R>
FP_HD uint32_t nz_sub(const uint32_t *a, const uint32_t *b) {
  uint32_t m = 0;
#pragma unroll
  for (int i = 0; i < R; ++i) m |= a[i] ^ b[i];
  return m;
}

// Isometric addition, p = 3 (Sec. 4.3): c = a or b, nonzero mask c0 xor c1.
FP_HD uint32_t nz_add_p3(uint32_t a0, uint32_t a1, uint32_t b0, uint32_t b1) {
  return (a0 | b0) ^ (a1 | b1);
}

// Isometric addition, p = 2^r - 1 (Sec. 4.3): a + b != 0 iff some slice of
// a xnor b is set and some slice of a or b is set.
template <int R>
FP_HD uint32_t nz_add_mersenne(const uint32_t *a, const uint32_t *b) {
  uint32_t x = 0, o = 0;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    x |= ~(a[i] ^ b[i]);
    o |= a[i] | b[i];
  }
  return x & o;
}

// Nonzero mask of one bit-sliced vector: OR of its slices.
template <int R>
FP_HD uint32_t nz(const uint32_t *a) {
  uint32_t m = 0;
#pragma unroll
  for (int i = 0; i < R; ++i) m |= a[i];
  return m;
}

// Negation for p = 2^r - 1: -a is the bitwise complement (2^r - 1 - a),
// kept zero where a is zero.
template <int R>
FP_HD void neg_mersenne(const uint32_t *a, uint32_t *s) {
  uint32_t m = nz<R>(a);
#pragma unroll
  for (int i = 0; i < R; ++i) s[i] = ~a[i] & m;
}

// Multiplication by 2^t for p = 2^r - 1: circular shift of the slice index
// (Sec. 4.2: 3 * 2 = (0,1,1), 3 * 4 = (1,0,1) in F_7).
template <int R>
FP_HD void mul_pow2_mersenne(const uint32_t *a, uint32_t *s, int t) {
#pragma unroll
  for (int i = 0; i < R; ++i) s[(i + t) % R] = a[i];
}

}  // namespace fpbs
