/*
 * fpcode_testing.h -- introspection and unit hooks of libfpcode, used by
 * the test-suite to check host logic and the bit-sliced F_p arithmetic on
 * their own.  Not needed to compute distances.
 */
#ifndef FPCODE_TESTING_H
#define FPCODE_TESTING_H

#include <stdint.h>

#include "fpcode.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Bit-sliced operations (lane-wise over 32 symbols; r = floor(log2 p) + 1
 * slices per operand, slice i = bit i of the natural binary expansion,
 * Sec. 2):
 *   0 FPCODE_OP_ADD       exact a + b (Alg. 3 for p = 3, Alg. 4 for p = 7,
 *                         ripple add + conditional subtract otherwise)
 *   1 FPCODE_OP_NZ_SUB    mask of a - b != 0 (isometric subtraction, Sec. 4.3)
 *   2 FPCODE_OP_NZ_ADD    mask of a + b != 0 (isometric addition, Sec. 4.3;
 *                         p = 3 or p = 2^r - 1 only)
 *   3 FPCODE_OP_NEG       -a (p = 2^r - 1 only: complement where nonzero)
 *   4 FPCODE_OP_MUL2      2a (p = 2^r - 1 only: slice rotation, Sec. 4.2)
 * a, b, out: r words each (out: 1 word for the masks).  Host evaluation. */
enum { FPCODE_OP_ADD = 0, FPCODE_OP_NZ_SUB = 1, FPCODE_OP_NZ_ADD = 2, FPCODE_OP_NEG = 3, FPCODE_OP_MUL2 = 4 };
int fpcode_test_bitslice_host(int op, int p, const uint32_t *a, const uint32_t *b, uint32_t *out);

/* The same operations in a GPU kernel over `count` independent operand
 * sets laid out back to back (a, b: count * r words; out: count * r words,
 * or count words for the masks).  Host pointers; copies in and out. */
int fpcode_test_bitslice_device(int op, int p, int count, const uint32_t *a, const uint32_t *b, uint32_t *out);

/* Revolving-door order of t-subsets of {0..n-1}, subsets as bit masks. */
uint64_t fpcode_test_rd_unrank(uint64_t rank, int n, int t);
uint64_t fpcode_test_rd_rank(uint64_t subset, int n, int t);
/* 1 and *next = successor, or 0 if `subset` is the last one. */
int fpcode_test_rd_next(uint64_t subset, int n, int t, uint64_t *next);

/* Prefix index I of pass g (k rows, prime p) -> largest row m, subset mask
 * Q and the coefficients of Q's members in increasing row order (coefs:
 * g - 2 ints). */
int fpcode_test_prefix_unrank(uint64_t I, int k, int g, int p, int *m, uint64_t *Q, int *coefs);
/* The walk the kernel takes from prefix I to I + 1, on the host: same
 * outputs for I + 1. */
int fpcode_test_prefix_walk(uint64_t I, uint64_t steps, int k, int g, int p, int *m, uint64_t *Q, int *coefs);

/* Introspection of a prepared object. */
typedef struct fpcode_pass_info {
  int g, j, L_before, L_after, round_end;
  int ntasks;  /* CTA tasks of the pass under the plan of the code's upload (0 before it) */
  uint64_t size;
  uint64_t nprefix;
} fpcode_pass_info;
int fpcode_prepared_shape(const fpcode_prepared *prep, int *m, int *kj, int *npasses, int *complete);
/* Gamma_j (k x n) and its pivot columns (k). */
int fpcode_prepared_gamma(const fpcode_prepared *prep, int j, uint8_t *gamma, int *pivots);
int fpcode_prepared_passes(const fpcode_prepared *prep, fpcode_pass_info *passes, int max);
/* Stored bit-sliced multiple v * A_j[t] of the non-pivot part of row t of
 * Gamma_j (v in 1..p-1): r * W words into `slices`, word w and slice i at
 * [w * r + i]; and, when `sig` is given and p is 3 or 7, the row's pair
 * signature words.  Returns the number of signature words (0: none), or a
 * negative status. */
int fpcode_test_prepared_row(const fpcode_prepared *prep, int j, int t, int v, uint32_t *slices, uint32_t *sig);
/* The CTA task ranges [lo, hi), in prefixes (pair-leaf passes: stems), of pass `pass` when planned
 * for `ctas` CTAs (fixed_pl > 0: fixed tasks of 256 * fixed_pl prefixes; 0:
 * guided, with fixed tasks of at least min_steps prefixes per lane for a pass
 * too small to give every lane of the grid that many; with min_steps <= 8,
 * as for one code, a pass under one prefix unit per lane of the grid gets one
 * unit per lane).  Returns the number of tasks (at most max written). */
int fpcode_test_task_ranges(fpcode_prepared *prep, int pass, int ctas, int fixed_pl, int min_steps, uint64_t *lo,
                            uint64_t *hi, int max);
/* Pair leaves (fpcode_opts.pair_leaves): words per pair-table entry of the
 * prepared code (0: one-row leaves).  With `pass` >= 0 and a stem J of that
 * pass, *entries receives the pair entries the stem is evaluated against,
 * (p-1) C(k-1-q, 2) with q the stem's largest row (g = 2: all pairs).
 * Returns the words per entry, or a negative status. */
/* The prefixes [lo, hi) every lane of every task of one-row pass `pass`
 * (g >= 2) walks under the plan for `ctas` CTAs, task-major, lane-minor:
 * the task's contiguous range of units split evenly over its lanes, as the
 * kernel splits it.  Returns tasks x threads per CTA (entries past max not
 * written), or -1. */
int fpcode_test_lane_ranges(fpcode_prepared *prep, int pass, int ctas, int fixed_pl, int min_steps, uint64_t *lo,
                            uint64_t *hi, int max);
int fpcode_test_pair_mode(const fpcode_prepared *prep, int pass, uint64_t J, uint32_t *entries);
/* Pair-table entry e of Gamma_j (pair leaves), computed on the host from
 * the prepared multiples: its pair_sigp words (the signature words of
 * B = A_j[y] + c A_j[x], word w's r - 1 words at [w * (r - 1)], then
 * zeros), followed by slice 0 of B (W words).  `sig` holds up to 12 words.
 * Returns the number of words, or a negative status. */
int fpcode_test_pair_entry(const fpcode_prepared *prep, int j, uint32_t e, uint32_t *sig);
/* The pair table of Gamma_j as the kernels build it in shared memory
 * (Sec. 4.3 with pair leaves): one CTA stages the set's multiples, runs the
 * builder and copies the table out: all entries' pair_sigp signature words
 * (padded to 16 bytes), then all entries' slice 0 (W words each).  `out`
 * holds max_words u32 (host memory); runs on the current device,
 * synchronously.  Returns the table's words, or a negative status. */
int fpcode_test_pair_table_device(const fpcode_prepared *prep, int j, uint32_t *out, int max_words);
/* The coordinate search of fpcode_autotune_batch over a synthetic cost
 * table: ndim settings with sizes[i] values each, cost[] in row-major order
 * (the last setting fastest), starting at index vector `start`.  best
 * receives the chosen index vector, *evals the points evaluated.  Returns
 * 0, or a negative status. */
int fpcode_test_tune_search(int ndim, const int *sizes, const int *start, const double *cost, int *best, int *evals);
/* Coefficients (k ints, 0 for rows outside the codeword) of the codeword of
 * Gamma_j that packed key `key` stands for, as the witness is rebuilt; *g
 * and *j receive its level and information set.  Returns 0, or -1 if the
 * key names no codeword of the schedule. */
int fpcode_test_key_coefficients(const fpcode_prepared *prep, uint64_t key, int *g, int *j, int *coef);
/* Microseconds from the start of the last search on `prep` to the end of
 * each of its passes (-1: not reached), for up to max passes.  Returns the
 * number of passes written, or -1. */
int fpcode_test_pass_times(fpcode_prepared *prep, void *stream, double *us, int max);

/* Single-pass probe (kernel efficiency on a pass of fixed, closed-form size,
 * Sec. 3.1 Alg. 6 with its termination test switched off): *out is a new
 * prepared code whose schedule is pass `pass` of `src` alone, with lower
 * bounds 0 so that every task runs and nothing is certified.  u_init > 0
 * starts the search with the upper bound U = u_init (the record threshold a
 * real search has by that level); 0 starts from the Singleton bound.  Run it
 * with fpcode_search_enqueue / fpcode_search_finish: the status is
 * FPCODE_EBUDGET, counts[g] is the pass size, U the least weight found in
 * the pass (or u_init if none is lower), and a witness is returned only for
 * a codeword of the pass.  Owned by the caller (fpcode_prepared_free).
 * FPCODE_EINVAL: no such pass, or u_init outside 0..255. */
int fpcode_prepared_single_pass(const fpcode_prepared *src, int pass, int u_init, fpcode_prepared **out);

/* Additions benchmark (Sec. 5.1: two sets of vectors over F_p added
 * pairwise, repeated): a and b are nvec x nsym symbols in [0, p) (host,
 * row-major, caller-owned); the device computes out = a + reps * b (mod p)
 * as a dependent chain of `reps` additions c <- c + b, in the bit-sliced
 * natural encoding (sliced = 1: p = 3 or 7, 32 symbols per word and slice)
 * or one symbol per byte with per-byte SIMD operations (sliced = 0: any
 * odd prime p < 128).  *ms is the kernel time (CUDA events on `stream`).
 * Allocates and frees its own device buffers.  FPCODE_EINVAL on bad
 * arguments or a symbol >= p, FPCODE_ECUDA on a CUDA error. */
int fpcode_bench_additions(int p, int sliced, int nvec, int nsym, int reps, const uint8_t *a, const uint8_t *b,
                           uint8_t *out, void *stream, double *ms);
/* Bytes one fpcode_min_distance call on this code moves: host-to-device
 * (tables, schedule, descriptors, the first state and the zeroed per-pass
 * bookkeeping, in one copy) and device-to-host (final state). */
int fpcode_prepared_bytes(const fpcode_prepared *prep, uint64_t *h2d, uint64_t *d2h);

#ifdef __cplusplus
}
#endif
#endif /* FPCODE_TESTING_H */
