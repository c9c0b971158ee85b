/*
 * fpcode.h -- C ABI of libfpcode: certified minimum Hamming distance of a
 * linear [n,k] code over a prime field F_p on one NVIDIA GB300 (sm_103a).
 *
 * The method is the Brouwer-Zimmermann search of arXiv 2603.29942
 * (Sec. 3.1, Alg. 6): for each systematic generator matrix Gamma_j of the
 * code on disjoint information sets, every codeword that is a combination
 * of exactly g rows with nonzero coefficients is enumerated; g grows until
 * the lower bound L meets the best weight U found.  Codewords are held in
 * the paper's bit-sliced natural encoding (Sec. 2, Sec. 4.1), so F_p
 * addition is a boolean formula over 32-bit words (Alg. 3 for p = 3,
 * Alg. 4 for p = 7 and its end-around-carry form for p = 31 and 127, a
 * ripple add with a conditional subtraction of p otherwise) and a weight is
 * the popcount of the OR of the slices (Sec. 4.3).
 *
 * Conventions for every call:
 *   - Returns an fpcode status (FPCODE_OK = 0).  Outputs are written only on
 *     FPCODE_OK, except that FPCODE_EBUDGET / FPCODE_ETIMEOUT still fill the
 *     certified interval [L, U] and the counts of an fpcode_result.
 *   - Matrices are row-major uint8 arrays in host memory with entries in
 *     [0, p); they are copied, never retained.
 *   - `stream` is a cudaStream_t (NULL: the legacy default stream).  Calls
 *     that return results synchronise that stream before returning.
 *   - Device memory belongs to the library (per-device workspace, or the
 *     prepared object / server that asked for it).
 *   - Limits: p an odd prime < 256; 1 <= k <= 64; k <= n <= 255;
 *     n - k <= 128; a code whose bit-sliced row multiples of one
 *     information set exceed 96 KiB is rejected (FPCODE_EINVAL).
 *     Passes beyond 255 per code or beyond 2^34 prefixes are not entered
 *     (FPCODE_EBUDGET with [L, U]).
 *   - Thread safety: calls on different prepared objects / servers may run
 *     concurrently; calls that use the shared per-device workspace
 *     (fpcode_min_distance, fpcode_min_distance_batch) serialise on it.
 */
#ifndef FPCODE_H
#define FPCODE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FPCODE_MAX_K 64
#define FPCODE_MAX_N 255
#define FPCODE_MAX_M 255

enum fpcode_status {
  FPCODE_OK = 0,
  FPCODE_EINVAL = 1,   /* bad argument: p not an odd prime < 256, k, n out of range,
                          an entry >= p, rank(G) < k, a table too large */
  FPCODE_ENOMEM = 2,   /* host or device allocation failed */
  FPCODE_ECUDA = 3,    /* a CUDA call failed (message: fpcode_last_error) */
  FPCODE_EBUDGET = 4,  /* not certified within the budget: L < U returned */
  FPCODE_ETIMEOUT = 5, /* time limit, or a bounded device wait gave up */
  FPCODE_EBUSY = 6,    /* serving: no free slot */
  FPCODE_ENOTREADY = 7 /* serving: the ticket is still running */
};

/* Search options.  fpcode_opts_default() fills the defaults shown. */
typedef struct fpcode_opts {
  int per_round_check; /* 0: test L >= U after every pass (default);
                          1: only after each full round g (Alg. 6) */
  int defer;           /* 1 (default): a rank-deficient Gamma_j is first
                          enumerated in round g = k - k_j (it cannot raise L
                          earlier), catching up its levels 1..g */
  int mid_pass_exit;   /* 1 (default): stop a pass as soon as U <= L held
                          before it (early termination, Sec. 4.4); d and the
                          per-level counts are unchanged, `enumerated` and
                          the choice among equal-weight witnesses may vary */
  int ctas_per_sm;     /* 0: from the occupancy calculator */
  int prefixes_per_lane; /* one-row leaves: 0: the task plan (guided
                          tasks, min_steps for small passes); else fixed
                          tasks of this many prefixes per lane (1..64) */
  int lookahead;       /* 1 (default): CTAs take tasks of the next passes as
                          soon as the current pass has none left, instead of
                          waiting for its last tasks; the termination test
                          still runs pass by pass in order, so d, L and the
                          passes entered are the same; 0: one pass at a time */
  uint64_t budget;     /* 0: unlimited; else a pass is not entered if it
                          would take the per-level count total above it */
  double timeout_s;    /* 0: none; else time limit of one device search */
  double wait_limit_s; /* bound on one device wait at a pass hand-off
                          (default 10 s); past it the kernel exits with
                          FPCODE_ETIMEOUT instead of spinning */
  int pair_leaves;     /* 1: a single code with p = 3 or 7 whose pair
                          table fits (40 KiB per information set)
                          enumerates each codeword of a pass g >= 2 as a
                          stem of g - 2 rows held exactly plus a pair of
                          rows (y, x) from a table of A[y] + c A[x], and
                          bounds S + B and S - B with one popcount (the
                          isometric last addition of Sec. 4.3 carried to
                          the last two rows); 0: one-row leaves; 2
                          (default): pair leaves when the search is
                          expected to take 10^8 codewords or more (d from
                          the Gilbert-Varshamov bound), since the pair
                          table pays off on large passes and small
                          searches are bound by latency.  Batches and
                          servers use one-row leaves.  d, L, U and the
                          per-level counts do not depend on it. */
  int min_steps;       /* one-row leaves: prefixes per lane given to a pass
                          too small to fill the grid (0: 8 for one code,
                          32 for a batch, 1 when serving) */
  int task_work;       /* pair leaves: least work of a task per lane, in
                          pair entries (0: 192) */
  int task_share;      /* pair leaves: a task takes 1 / (task_share * C) of
                          its pass's remaining work, C the CTAs of the
                          grid, until task_work (0: 1 for a pass with more
                          passes after it in the launch, 2 for the last) */
  int batch_words;     /* batches: words per slice up to which a code with
                          p in {3, 5, 7} goes to the narrow batched kernel
                          (0 or 2: n - k <= 64, the others in a second,
                          wide launch; 4: every such code in one wide
                          launch); 1: one launch per kernel variant (prime
                          class and words per slice) of the single-code
                          kernels, where codes of p = 3, 7 may take pair
                          leaves (pair_leaves) */
} fpcode_opts;

typedef struct fpcode_result {
  int status;          /* FPCODE_OK: d certified */
  int d;               /* minimum distance (FPCODE_OK), else -1 */
  int L;               /* lower bound when the search stopped */
  int U;               /* best weight found (upper bound) */
  int m;               /* number of information sets */
  int npasses;         /* passes entered (last pass index + 1) */
  int launch;          /* fpcode_min_distance_batch: index of the kernel
                          launch that searched this code (codes are grouped
                          by kernel); t_kernel_ms is that launch's time */
  int reserved1;
  uint64_t enumerated; /* codewords the GPU evaluated in the passes entered
                          (work taken ahead past the certifying pass is not
                          counted) */
  uint64_t counts[FPCODE_MAX_K + 1]; /* per level g: codewords of the passes
                          entered, C(k,g)(p-1)^(g-1) each (equals the
                          enumeration when mid_pass_exit = 0) */
  int kj[FPCODE_MAX_M]; /* fresh pivot columns of each Gamma_j */
  int reserved2;
  double t_prepare_ms; /* host elimination and bit-slicing */
  double t_h2d_ms;     /* upload */
  double t_kernel_ms;  /* device search (CUDA events) */
  double t_d2h_ms;     /* result read-back */
  double t_total_ms;   /* whole call, host clock */
  uint64_t best_key;   /* packed key of the best codeword found (all ones:
                          none); fpcode_prepared_codeword rebuilds it */
} fpcode_result;

typedef struct fpcode_prepared fpcode_prepared; /* opaque, library-owned */

/* Fill *o with the defaults. */
void fpcode_opts_default(fpcode_opts *o);

/* Text of the last error on this thread (never NULL). */
const char *fpcode_last_error(void);

/* Host preparation (not on the hot path): Gaussian elimination mod p of G
 * into Gamma_1..Gamma_m on disjoint information sets (Sec. 3.1; the paper
 * leaves the choice open -- Gamma_1 pivots on the leftmost independent
 * columns, each later Gamma_j greedily on the leftmost columns unused so
 * far, completed with used ones if rank-deficient), the p-1 multiples of
 * every row restricted to the non-pivot columns, bit-sliced into
 * ceil((n-k)/32) words per slice (Sec. 2, Sec. 4.1), and the pass
 * schedule.  G: k x n, row-major, entries in [0, p), copied.  opts may be
 * NULL.  On success *out owns host memory; free with fpcode_prepared_free.
 * Errors: FPCODE_EINVAL, FPCODE_ENOMEM. */
int fpcode_prepare(int p, int n, int k, const uint8_t *G, const fpcode_opts *opts, fpcode_prepared **out);

/* Release a prepared object and its device copy (if any).  NULL is a no-op. */
void fpcode_prepared_free(fpcode_prepared *prep);

/* Copy the prepared tables into device memory owned by `prep` (once; later
 * calls are no-ops), enqueued on `stream`, synchronised before return.
 * Errors: FPCODE_ENOMEM, FPCODE_ECUDA. */
int fpcode_prepared_upload(fpcode_prepared *prep, void *stream);

/* Enqueue one device search on the uploaded `prep` without synchronising:
 * the persistent kernel, whose last CTA copies the final state into
 * host-mapped memory of `prep` and zeroes the device state for the next
 * search.  The first search after fpcode_prepared_upload is preceded by a
 * state reset; where the memory cannot be mapped, every search is, and its
 * state is copied back after the kernel.  Pair with fpcode_search_finish on the same stream; one search
 * of a prepared object at a time.  Errors: FPCODE_EINVAL (not uploaded),
 * FPCODE_ECUDA. */
int fpcode_search_enqueue(fpcode_prepared *prep, void *stream, const fpcode_opts *opts);

/* Synchronise `stream` and decode the last enqueued search into *res and,
 * if witness != NULL, a minimum-weight codeword (n bytes, caller-owned),
 * rebuilt exactly from its Gamma_j rows and checked to have weight d. */
int fpcode_search_finish(fpcode_prepared *prep, void *stream, fpcode_result *res, uint8_t *witness);

/* Checkpoint of a search that stopped at its budget without certifying
 * (status FPCODE_EBUDGET): the state of Sec. 3.1 Alg. 6 between two passes,
 * i.e. how many passes of the schedule are complete and the best codeword
 * found.  A later search of the same code, prepared with the same
 * per_round_check and defer and a larger budget (its schedule starts with
 * the same passes), continues from it with fpcode_search_resume instead of
 * starting over.  The result equals that of one search with the larger
 * budget, except that `enumerated` counts the codewords of the resumed run
 * only.  The paper has no counterpart: it budgets nothing. */
typedef struct fpcode_checkpoint {
  int p, n, k;
  int passes_done;     /* passes 0 .. passes_done - 1 of the schedule are complete */
  uint64_t best_key;   /* packed key of the best codeword found (all ones: none) */
  uint64_t code_hash;  /* 64-bit hash of (p, n, k, per_round_check, defer,
                          pair leaves taken) and G: the schedule and key layout */
} fpcode_checkpoint;

/* After fpcode_search_finish returned FPCODE_EBUDGET: the checkpoint of that
 * search.  FPCODE_EINVAL if the last search certified, timed out or never
 * ran. */
int fpcode_search_checkpoint(const fpcode_prepared *prep, fpcode_checkpoint *out);

/* Like fpcode_search_enqueue, but the search starts after the checkpoint's
 * passes with its best codeword as the bound; pair with
 * fpcode_search_finish.  FPCODE_EINVAL if the checkpoint is of another code
 * or other schedule options, if `prep`'s schedule has no pass after it, or
 * if `prep` is not uploaded. */
int fpcode_search_resume(fpcode_prepared *prep, const fpcode_checkpoint *ck, void *stream, const fpcode_opts *opts);

/* One search split over several GPUs (one process per GPU): the paper's
 * parallel search (Sec. 5.2, Table 4) carried to GPUs.  Every rank prepares
 * and uploads the same code (the same GPU type gives every rank the same
 * task plan: fpcode_pass_info.ntasks), then for each pass of the schedule in
 * order searches its own contiguous range of the pass's tasks, starting
 * from the best weight found so far; the ranks then take the minimum of
 * their packed keys (an allreduce of 8 bytes) and all apply the same
 * termination test L >= U (Alg. 6) to it.  paper_2603_29942_gb300/shard.py
 * drives this over torch.distributed.
 *
 * fpcode_prepared_pass_slice: *out (to free with fpcode_prepared_free) is
 * tasks [task_lo, task_hi) of pass `pass` of the uploaded `src`, alone, its
 * termination test off, with u_init (> 0) as its first bound: search it
 * with fpcode_min_distance_ex; the result's best_key (all ones: nothing at
 * or under the bound) carries pass field 0, the slice's one pass.
 * Errors: FPCODE_EINVAL (no such pass, an empty range). */
int fpcode_prepared_pass_slice(const fpcode_prepared *src, int pass, uint64_t task_lo, uint64_t task_hi, int u_init,
                               fpcode_prepared **out);

/* The first bound of the next searches of a slice made by
 * fpcode_prepared_pass_slice (0: none), so that one uploaded slice serves
 * every search of the split: the bound changes, the tables stay.  Errors:
 * FPCODE_EINVAL (not a slice, or u_init outside 0..255). */
int fpcode_prepared_set_bound(fpcode_prepared *slice, int u_init);
/* The codeword (n bytes, caller-owned) a packed key of `prep`'s schedule
 * stands for, rebuilt exactly from its Gamma_j rows, and its weight.
 * Errors: FPCODE_EINVAL (the key names no codeword). */
int fpcode_prepared_codeword(const fpcode_prepared *prep, uint64_t key, uint8_t *codeword, int *weight);

/* Upload (if needed) + enqueue + finish. */
int fpcode_min_distance_ex(fpcode_prepared *prep, void *stream, const fpcode_opts *opts, fpcode_result *res,
                           uint8_t *witness);

/* One call from a host matrix to a certified distance (Sec. 3.1, Alg. 6):
 * prepare, upload, search, read back.  *d receives the minimum distance;
 * witness (n bytes, may be NULL) a codeword of weight d.  Uses the shared
 * per-device workspace.  Errors: as above; FPCODE_EBUDGET cannot occur
 * (no budget). */
int fpcode_min_distance(int p, int n, int k, const uint8_t *G, void *stream, int *d, uint8_t *witness);

/* fpcode_min_distance without any allocation, for callers that cannot call
 * cudaMalloc (code running where the CUDA allocator is off limits, such as
 * a host callback or a component whose device memory is fixed at start-up).
 * The paper has no counterpart: this is a deployment variant of
 * fpcode_min_distance.  It allocates no device memory and no pinned host
 * memory (no cudaMalloc, cudaMallocHost, cudaFree or allocating library
 * routine); host-side preparation uses the ordinary C++ heap.  All device
 * state lives in one fixed 512 KiB array inside the library that every GPU
 * loading the library keeps until exit; a code whose tables, schedule and
 * state need more than that is rejected with FPCODE_EINVAL (message in
 * fpcode_last_error) -- use fpcode_min_distance for it.  The first call on
 * a device looks up the array's device address and writes a table into it
 * (make it before any stream capture; a cudaDeviceReset after it is not
 * supported).  Calls share the array: calls that overlap on the GPU race, and
 * calls from this process are serialised on the host.  Same arguments and
 * results as fpcode_min_distance. */
int fpcode_min_distance_noalloc(int p, int n, int k, const uint8_t *G, void *stream, int *d, uint8_t *witness);

/* One code of a batch or a served request. */
typedef struct fpcode_desc {
  int p, n, k;
  int reserved;
  const uint8_t *G;  /* k x n, row-major, host memory, copied */
  uint64_t budget;   /* per-code budget (0: opts->budget) */
} fpcode_desc;

/* Many codes of uneven (p, n, k) in one persistent launch: every code keeps
 * its own pass sequence and bound; CTAs steal tasks across codes.  Codes
 * with p outside {3, 5, 7} run in further launches.  results: num entries;
 * witnesses: sum of n_i bytes (code i at the sum of the earlier n), may be
 * NULL.  Returns FPCODE_OK if every code was processed (each result has
 * its own status) or the first global error. */
int fpcode_min_distance_batch(int num, const fpcode_desc *codes, void *stream, const fpcode_opts *opts,
                              fpcode_result *results, uint8_t *witnesses);

/* Launch settings of fpcode_min_distance_batch chosen by measurement on
 * this GPU (the paper tunes its word width and isometry per configuration
 * by hand, Sec. 4.1, Table 3).  The settings searched: CTAs per SM (0: the
 * occupancy limit, 3, 2: fewer, longer-lived warps per code), min_steps
 * (8, 16, 32, 64, 128 prefixes per lane in the small passes: the chunk
 * size) and batch_words (2: narrow and wide batched launches by words per
 * slice; 4: one wide batched launch; 1: one launch per kernel variant,
 * with pair leaves for the codes that take them).  A coordinate search
 * starts at the defaults, measures every value of one setting with the
 * others held (each point once, `reps` timed batches after a warm-up, end
 * to end from the host matrices), moves to the best, and stops when a round
 * over all settings finds nothing better.  The choice is cached per GPU
 * (name and SM count) and workload class (the primes present, the largest
 * words per slice and k, the number of codes and the budget, in powers of
 * two and ten): a later call for the same class returns it with
 * evaluated = 0. */
typedef struct fpcode_tuning {
  int ctas_per_sm;        /* chosen CTAs per SM (0: the occupancy limit) */
  int min_steps;          /* chosen prefixes per lane of small passes */
  int batch_words;        /* chosen grouping: 2, 4 or 1 */
  int evaluated;          /* settings measured by this call (0: from the cache) */
  double ms;              /* one batch with the chosen settings */
  double ms_default;      /* one batch with the default settings */
  char workload_class[96];
} fpcode_tuning;

/* Choose the batch launch settings for `codes` by measurement (above);
 * base: options the settings are added to (NULL: defaults; its budget
 * applies to codes whose own budget is 0).  *out receives the choice;
 * apply it with fpcode_tuning_apply.  Errors: as fpcode_min_distance_batch. */
int fpcode_autotune_batch(int num, const fpcode_desc *codes, void *stream, const fpcode_opts *base, int reps,
                          fpcode_tuning *out);
/* Copy a tuning's settings into *opts. */
void fpcode_tuning_apply(const fpcode_tuning *t, fpcode_opts *opts);

/* Serving: a request loop over the same persistent kernel.  Requests are
 * admitted into free slots as device memory allows, kept resident with
 * their bounds, and interleaved on the GPU with the codes already running;
 * results are polled without blocking. */
typedef struct fpcode_serve_opts {
  int slots;              /* concurrent codes on the device (default 64) */
  int ctas_per_sm;        /* 0: occupancy calculator */
  size_t device_bytes;    /* device memory for code tables (default 64 MiB) */
  double idle_exit_s;     /* persistent kernel exits after this long idle
                             (default 0.02 s); it is relaunched on demand */
  int max_words;          /* 32-bit words per slice a served code may need:
                             2 (default: n - k <= 64, the faster kernel) or
                             4 (n - k <= 128); a code above it is rejected
                             with FPCODE_EINVAL */
  int reserved;
  fpcode_opts search;     /* per-code search options */
} fpcode_serve_opts;

typedef struct fpcode_server fpcode_server;

void fpcode_serve_opts_default(fpcode_serve_opts *o);
int fpcode_serve_create(const fpcode_serve_opts *o, void *stream, fpcode_server **out);
/* Prepare and admit one code; *ticket identifies it.  FPCODE_EBUSY: no slot
 * or memory free right now (retry after polling). */
int fpcode_serve_submit(fpcode_server *s, const fpcode_desc *code, uint64_t *ticket);
/* Collect up to `max` finished codes (non-blocking).  witnesses: max * 255
 * bytes (row i at i*255), may be NULL. */
int fpcode_serve_poll(fpcode_server *s, fpcode_result *out, uint64_t *tickets, uint8_t *witnesses, int max,
                      int *n_out);
/* Wait until every admitted code has finished (bounded by timeout_ms). */
int fpcode_serve_drain(fpcode_server *s, int timeout_ms);
/* Kernel launches the server has made so far (the persistent kernel exits
 * after its idle period and is launched again on demand). */
int fpcode_serve_launches(const fpcode_server *s, uint64_t *n);
void fpcode_serve_destroy(fpcode_server *s);

/* Measured integer issue rates of this GPU (LOP3, POPC, IADD lanes per
 * clock per SM and per second), from a microbenchmark with independent
 * instruction chains on every SM; the ceiling the enumeration kernel is
 * compared with.  rates: 6 doubles {lop3/clk/SM, popc/clk/SM,
 * iadd/clk/SM, lop3/s, popc/s, sm_clock_mhz}. */
int fpcode_int_peaks(void *stream, double *rates);

#ifdef __cplusplus
}
#endif
#endif /* FPCODE_H */
