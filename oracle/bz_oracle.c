/*
 * bz_oracle.c -- CPU reference oracle for the minimum Hamming distance of a
 * linear [n,k] code over a prime field F_p.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package's smoke check
 * and the benchmark's CPU-baseline leg may load or run this library.  The
 * product path (the CUDA library under paper_2603_29942_gb300/) shares no
 * code with it and never calls it.
 *
 * Everything here is deliberately plain: one F_p symbol per byte and
 * ordinary "(a + b) mod p" arithmetic -- the contiguous 8-bit storage that
 * the paper keeps as its reference implementation (Sec. 4.5, SC8) -- so that
 * a reader can check it against the paper by eye.
 *
 *   oracle_brute_force  definition of d (Sec. 3): minimum weight over all
 *                       nonzero codewords m*G, plus the full weight
 *                       distribution.  Pinned by textbook codes, MacWilliams
 *                       and hand-checkable tiny cases in the tests.
 *   oracle_info_sets    systematic generator matrices Gamma_1..Gamma_m on
 *                       disjoint information sets (Sec. 3.1).  The paper is
 *                       silent on how they are chosen; this follows the
 *                       leftmost-column greedy reading (see the function).
 *   oracle_bz           Brouwer-Zimmermann search (Sec. 3.1, Alg. 6) with the
 *                       projective normalisation of Sec. 4.2 (coefficient of
 *                       the first chosen row fixed to 1), saved partial sums
 *                       (Sec. 4.3) and early termination (Sec. 4.4).
 *
 * Readings of the paper taken here (the paper is silent or ambiguous):
 *   - Alg. 6 enumerates, per pass, c in F_2^k of weight g (carried over from the binary
 *     algorithm); over F_p this is every c in F_p^k with exactly g nonzero
 *     entries, normalised projectively, C(k,g)(p-1)^(g-1) codewords per pass.
 *   - Lower bound after any pass: L = sum_i max(0, e_i + 1 - (k - k_i)),
 *     e_i = highest level completed for Gamma_i.  After a full round with
 *     only Gamma_m rank-deficient this is the bound of Alg. 6.
 *   - Termination when L >= U (the test of Alg. 6); checked after every pass by
 *     default, or only after each full round (per_round_check = 1).
 *   - A rank-deficient Gamma_j cannot raise L before level k - k_j; with
 *     defer = 1 it is first enumerated in round g = k - k_j, catching up all
 *     of its levels 1..g.
 *   - U starts at the Singleton bound n-k+1 (the start of Alg. 6); a codeword of
 *     that weight is still recorded while no witness is held, so a witness
 *     always exists at the end.
 *   - Budget: a pass is not entered if it would take the number of
 *     enumerated codewords above the budget (status ORACLE_EBUDGET).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_MAX_N 256
#define ORACLE_MAX_K 64
#define ORACLE_MAX_M 256
#define ORACLE_MAX_PASSES 1024

enum {
  ORACLE_OK = 0,
  ORACLE_EINVAL = 1,
  ORACLE_ENOMEM = 2,
  ORACLE_EBUDGET = 3,
  ORACLE_ETOOBIG = 4
};

typedef struct {
  int per_round_check; /* 1: test L >= U only after a full round (Alg. 6) */
  int defer;           /* 1: defer rank-deficient Gamma_j to g >= k - k_j */
  int threads;         /* worker threads for one pass (<= 1: sequential)   */
  int reserved;
  uint64_t budget;     /* 0: unlimited; else cap on enumerated codewords   */
} oracle_opts;

typedef struct {
  int status;          /* ORACLE_OK: d certified; ORACLE_EBUDGET: [L, U]   */
  int d;               /* minimum distance (valid when status == OK)      */
  int L;               /* lower bound when the search stopped             */
  int U;               /* best weight found (upper bound)                 */
  int m;               /* number of information sets                      */
  int npasses;         /* passes entered                                  */
  int exhausted;       /* 1: every level of Gamma_1 was enumerated        */
  int reserved;
  uint64_t evaluated;  /* codewords enumerated (sum of pass sizes)        */
  uint64_t counts[ORACLE_MAX_K + 1]; /* codewords enumerated per level g   */
  int kj[ORACLE_MAX_M];              /* fresh pivots of each Gamma_j       */
  int pass_g[ORACLE_MAX_PASSES];     /* level of each pass entered         */
  int pass_j[ORACLE_MAX_PASSES];     /* information set of each pass       */
  int pass_best[ORACLE_MAX_PASSES];  /* min weight seen in the pass        */
  int pass_L[ORACLE_MAX_PASSES];     /* lower bound after the pass         */
} oracle_result;

/* ------------------------------------------------------------------ */
/* F_p helpers: one symbol per byte, values in [0, p).                 */
/* ------------------------------------------------------------------ */

static int is_odd_prime(int p) {
  if (p < 3 || p > 255 || (p % 2) == 0) return 0;
  for (int q = 3; q * q <= p; q += 2)
    if (p % q == 0) return 0;
  return 1;
}

/* Multiplicative inverse by search: the x in [1, p) with a*x = 1 mod p. */
static int inv_mod(int a, int p) {
  for (int x = 1; x < p; ++x)
    if ((a * x) % p == 1) return x;
  return 0;
}

/* dst[i] = (dst[i] + c * src[i]) mod p for i < n. */
static void axpy_mod(uint8_t *dst, const uint8_t *src, int c, int p, int n) {
  for (int i = 0; i < n; ++i) dst[i] = (uint8_t)((dst[i] + c * src[i]) % p);
}

/* Hamming weight: number of nonzero symbols. */
static int weight(const uint8_t *v, int n) {
  int w = 0;
  for (int i = 0; i < n; ++i) w += (v[i] != 0);
  return w;
}

static int valid_matrix(int p, int n, int k, const uint8_t *G) {
  if (!is_odd_prime(p) || k < 1 || n < k || n > ORACLE_MAX_N || k > ORACLE_MAX_K || !G)
    return 0;
  for (int i = 0; i < k * n; ++i)
    if (G[i] >= p) return 0;
  return 1;
}

/* ------------------------------------------------------------------ */
/* Brute force: the definition of the minimum distance (Sec. 3).       */
/* ------------------------------------------------------------------ */

/* Walks every message m in F_p^k as a base-p odometer and keeps the
 * codeword c = m * G up to date: when digit i steps from v to v+1 (or wraps
 * from p-1 to 0) the codeword changes by +G_i (mod p) either way.
 * dist[w] counts all p^k codewords of weight w (dist[0] = 1).
 * Refuses p^k > 2^32 (ORACLE_ETOOBIG). */
int oracle_brute_force(int p, int n, int k, const uint8_t *G, int *d_out, uint64_t *dist,
                       uint8_t *witness) {
  if (!valid_matrix(p, n, k, G) || !d_out || !dist) return ORACLE_EINVAL;
  double space = 1.0;
  for (int i = 0; i < k; ++i) space *= p;
  if (space > 4294967296.0) return ORACLE_ETOOBIG;

  uint8_t msg[ORACLE_MAX_K];
  uint8_t cw[ORACLE_MAX_N];
  memset(msg, 0, sizeof(msg));
  memset(cw, 0, sizeof(cw));
  for (int w = 0; w <= n; ++w) dist[w] = 0;
  dist[0] = 1; /* the zero codeword */
  int best = n + 1;
  for (;;) {
    int i = 0;
    while (i < k && msg[i] == p - 1) { /* wrap p-1 -> 0: codeword += G_i */
      msg[i] = 0;
      axpy_mod(cw, G + (size_t)i * n, 1, p, n);
      ++i;
    }
    if (i == k) break; /* back at the zero message: every message seen */
    msg[i] += 1;
    axpy_mod(cw, G + (size_t)i * n, 1, p, n);
    int w = weight(cw, n);
    dist[w] += 1;
    if (w < best) {
      best = w;
      if (witness) memcpy(witness, cw, (size_t)n);
    }
  }
  *d_out = best; /* nonzero codewords exist because rank(G) >= 1 is not checked here */
  return ORACLE_OK;
}

/* ------------------------------------------------------------------ */
/* Information sets (Sec. 3.1).                                         */
/* ------------------------------------------------------------------ */

/* Make column c a unit column with its 1 in row r (row r scaled, column c
 * eliminated from every other row), all mod p. */
static void pivot(uint8_t *M, int k, int n, int p, int r, int c) {
  uint8_t *row = M + (size_t)r * n;
  int s = inv_mod(row[c], p);
  for (int i = 0; i < n; ++i) row[i] = (uint8_t)((row[i] * s) % p);
  for (int q = 0; q < k; ++q) {
    if (q == r) continue;
    int f = M[(size_t)q * n + c];
    if (f) axpy_mod(M + (size_t)q * n, row, p - f, p, n);
  }
}

/* Greedy reading of "systematic generator matrices on disjoint information
 * sets": Gamma_1 is the reduced row-echelon form of G (pivots on the
 * leftmost independent columns).  Each later Gamma_j scans the columns not
 * used by any earlier information set in increasing order and pivots on
 * every column that is independent of the ones already taken in this round;
 * k_j counts these fresh pivots.  If k_j < k the basis is completed with the
 * leftmost independent previously-used columns.  Rows of Gamma_j are stored
 * in increasing order of their pivot column, so Gamma_j restricted to its
 * pivot columns is the identity.  Stops when every column is used or a round
 * finds no fresh pivot.
 *
 * gam: m * k * n bytes; piv: m * k pivot columns; kj: m counts.
 * Returns ORACLE_EINVAL if rank(G) < k. */
int oracle_info_sets(int p, int n, int k, const uint8_t *G, int max_m, int *m_out, int *kj,
                     uint8_t *gam, int *piv) {
  if (!valid_matrix(p, n, k, G) || !m_out || !kj || !gam || !piv || max_m < 1) return ORACLE_EINVAL;
  uint8_t *M = (uint8_t *)malloc((size_t)k * n);
  if (!M) return ORACLE_ENOMEM;
  memcpy(M, G, (size_t)k * n);
  uint8_t used[ORACLE_MAX_N];
  memset(used, 0, sizeof(used));
  int m = 0;
  for (;;) {
    int rowpiv[ORACLE_MAX_K];
    for (int r = 0; r < k; ++r) rowpiv[r] = -1;
    int fresh = 0;
    for (int c = 0; c < n && fresh < k; ++c) {
      if (used[c]) continue;
      int r = -1;
      for (int q = 0; q < k; ++q)
        if (rowpiv[q] < 0 && M[(size_t)q * n + c]) { r = q; break; }
      if (r < 0) continue; /* column c depends on the pivots taken so far */
      pivot(M, k, n, p, r, c);
      rowpiv[r] = c;
      ++fresh;
    }
    if (m == 0 && fresh < k) { free(M); return ORACLE_EINVAL; } /* rank(G) < k */
    if (fresh == 0) break;
    int done = fresh;
    for (int c = 0; c < n && done < k; ++c) { /* complete with used columns */
      if (!used[c]) continue;
      int r = -1;
      for (int q = 0; q < k; ++q)
        if (rowpiv[q] < 0 && M[(size_t)q * n + c]) { r = q; break; }
      if (r < 0) continue;
      pivot(M, k, n, p, r, c);
      rowpiv[r] = c;
      ++done;
    }
    if (done < k) { free(M); return ORACLE_EINVAL; }
    if (m >= max_m) { free(M); return ORACLE_ETOOBIG; }
    /* store rows in increasing pivot-column order */
    int order[ORACLE_MAX_K];
    for (int r = 0; r < k; ++r) order[r] = r;
    for (int a = 1; a < k; ++a) { /* insertion sort by pivot column */
      int x = order[a], b = a - 1;
      while (b >= 0 && rowpiv[order[b]] > rowpiv[x]) { order[b + 1] = order[b]; --b; }
      order[b + 1] = x;
    }
    for (int r = 0; r < k; ++r) {
      memcpy(gam + ((size_t)m * k + r) * n, M + (size_t)order[r] * n, (size_t)n);
      piv[m * k + r] = rowpiv[order[r]];
    }
    kj[m] = fresh;
    for (int r = 0; r < k; ++r) /* only the fresh pivots join the used set */
      used[rowpiv[r]] = 1;
    ++m;
    int any_unused = 0;
    for (int c = 0; c < n; ++c) any_unused |= !used[c];
    if (!any_unused) break;
  }
  free(M);
  *m_out = m;
  return ORACLE_OK;
}

/* ------------------------------------------------------------------ */
/* One pass (g, j) of Alg. 6: every codeword of weight-g combinations. */
/* ------------------------------------------------------------------ */

/* Every g-subset T of the rows of Gamma_j in lexicographic order, with
 * every coefficient vector whose first (smallest-row) coefficient is 1
 * (Sec. 4.2) and the others in [1, p).  The codeword sum_t c_t Gamma_j[t]
 * is formed over all n columns; partial sums of the first rows are kept per
 * depth and reused (Sec. 4.3).  Work is split into items, one per first row
 * t1 (g == 1) or per pair of first rows (t1, t2); the best codeword of a
 * pass is the lowest-weight one that comes first in this order, whatever
 * the number of threads. */
typedef struct {
  int p, n, k, g;
  const uint8_t *gam; /* k x n, Gamma_j */
  int nitems;
  int item_t1[ORACLE_MAX_K * ORACLE_MAX_K];
  int item_t2[ORACLE_MAX_K * ORACLE_MAX_K];
  volatile int next_item;
  /* per-item best: weight and codeword */
  int *item_best;
  uint8_t *item_wit;
  uint64_t *item_count;
} pass_ctx;

typedef struct {
  int best;
  uint8_t wit[ORACLE_MAX_N];
  uint64_t count;
} dfs_state;

static void dfs(const pass_ctx *cx, int depth, int start, uint8_t part[][ORACLE_MAX_N],
                dfs_state *st) {
  /* part[depth] holds the sum of the `depth` rows chosen so far */
  const int p = cx->p, n = cx->n, k = cx->k, g = cx->g;
  for (int t = start; t <= k - (g - depth); ++t) {
    for (int c = 1; c < p; ++c) {
      memcpy(part[depth + 1], part[depth], (size_t)n);
      axpy_mod(part[depth + 1], cx->gam + (size_t)t * n, c, p, n);
      if (depth + 1 == g) {
        int w = weight(part[depth + 1], n);
        st->count += 1;
        if (w < st->best) {
          st->best = w;
          memcpy(st->wit, part[depth + 1], (size_t)n);
        }
      } else {
        dfs(cx, depth + 1, t + 1, part, st);
      }
    }
  }
}

static void run_item(const pass_ctx *cx, int it, dfs_state *st) {
  uint8_t part[ORACLE_MAX_K + 1][ORACLE_MAX_N];
  const int n = cx->n, p = cx->p;
  st->best = ORACLE_MAX_N + 1;
  st->count = 0;
  memset(part[0], 0, (size_t)n);
  int t1 = cx->item_t1[it];
  /* first row: coefficient fixed to 1 (projective normalisation, Sec. 4.2) */
  memcpy(part[1], part[0], (size_t)n);
  axpy_mod(part[1], cx->gam + (size_t)t1 * n, 1, p, n);
  if (cx->g == 1) {
    int w = weight(part[1], n);
    st->count = 1;
    st->best = w;
    memcpy(st->wit, part[1], (size_t)n);
    return;
  }
  int t2 = cx->item_t2[it];
  for (int c = 1; c < p; ++c) {
    memcpy(part[2], part[1], (size_t)n);
    axpy_mod(part[2], cx->gam + (size_t)t2 * n, c, p, n);
    if (cx->g == 2) {
      int w = weight(part[2], n);
      st->count += 1;
      if (w < st->best) {
        st->best = w;
        memcpy(st->wit, part[2], (size_t)n);
      }
    } else {
      dfs(cx, 2, t2 + 1, part, st);
    }
  }
}

static void *worker(void *arg) {
  pass_ctx *cx = (pass_ctx *)arg;
  dfs_state *st = (dfs_state *)malloc(sizeof(dfs_state));
  if (!st) return NULL;
  for (;;) {
    int it = __sync_fetch_and_add(&cx->next_item, 1);
    if (it >= cx->nitems) break;
    run_item(cx, it, st);
    cx->item_best[it] = st->best;
    memcpy(cx->item_wit + (size_t)it * cx->n, st->wit, (size_t)cx->n);
    cx->item_count[it] = st->count;
  }
  free(st);
  return NULL;
}

/* Runs pass (g, Gamma) and returns its best weight; *wit gets the codeword,
 * *count the number of codewords enumerated.  Returns -1 on allocation
 * failure. */
static int run_pass(int p, int n, int k, int g, const uint8_t *gam, int threads, uint8_t *wit,
                    uint64_t *count) {
  pass_ctx *cx = (pass_ctx *)calloc(1, sizeof(pass_ctx));
  if (!cx) return -1;
  cx->p = p; cx->n = n; cx->k = k; cx->g = g; cx->gam = gam;
  int ni = 0;
  if (g == 1) {
    for (int t1 = 0; t1 < k; ++t1) { cx->item_t1[ni] = t1; cx->item_t2[ni] = -1; ++ni; }
  } else {
    for (int t1 = 0; t1 <= k - g; ++t1)
      for (int t2 = t1 + 1; t2 <= k - g + 1; ++t2) {
        cx->item_t1[ni] = t1; cx->item_t2[ni] = t2; ++ni;
      }
  }
  cx->nitems = ni;
  cx->next_item = 0;
  cx->item_best = (int *)malloc(sizeof(int) * (size_t)ni);
  cx->item_wit = (uint8_t *)malloc((size_t)ni * n);
  cx->item_count = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)ni);
  if (!cx->item_best || !cx->item_wit || !cx->item_count) {
    free(cx->item_best); free(cx->item_wit); free(cx->item_count); free(cx);
    return -1;
  }
  if (threads < 1) threads = 1;
  if (threads > 256) threads = 256;
  if (threads == 1 || ni == 1) {
    worker(cx);
  } else {
    pthread_t tid[256];
    int started = 0;
    for (int i = 0; i < threads; ++i)
      if (pthread_create(&tid[i], NULL, worker, cx) == 0) ++started;
    if (started == 0) worker(cx);
    for (int i = 0; i < started; ++i) pthread_join(tid[i], NULL);
  }
  int best = ORACLE_MAX_N + 1, bi = -1;
  uint64_t total = 0;
  for (int i = 0; i < ni; ++i) { /* first item with the lowest weight */
    total += cx->item_count[i];
    if (cx->item_best[i] < best) { best = cx->item_best[i]; bi = i; }
  }
  if (bi >= 0) memcpy(wit, cx->item_wit + (size_t)bi * n, (size_t)n);
  *count = total;
  free(cx->item_best); free(cx->item_wit); free(cx->item_count); free(cx);
  return best;
}

/* ------------------------------------------------------------------ */
/* Brouwer-Zimmermann (Sec. 3.1, Alg. 6).                               */
/* ------------------------------------------------------------------ */

static uint64_t sat_mul(uint64_t a, uint64_t b) {
  if (a == 0 || b == 0) return 0;
  if (a > UINT64_MAX / b) return UINT64_MAX;
  return a * b;
}

/* Size of a pass: C(k, g) (p-1)^(g-1), saturating at 2^64-1. */
uint64_t oracle_pass_size(int p, int k, int g) {
  if (g < 1 || g > k) return 0;
  uint64_t c = 1;
  for (int i = 1; i <= g; ++i) { /* C(k, i) = C(k, i-1) (k-i+1) / i, exact */
    unsigned __int128 t = (unsigned __int128)c * (uint64_t)(k - i + 1);
    t /= (uint64_t)i;
    c = t > UINT64_MAX ? UINT64_MAX : (uint64_t)t;
  }
  for (int i = 1; i < g; ++i) c = sat_mul(c, (uint64_t)(p - 1));
  return c;
}

/* Lower bound from the levels completed so far (reading of the bound in Alg. 6). */
static int lower_bound(int m, const int *e, const int *kj, int k) {
  int L = 0;
  for (int i = 0; i < m; ++i) {
    int v = e[i] + 1 - (k - kj[i]);
    if (v > 0) L += v;
  }
  return L;
}

int oracle_bz(int p, int n, int k, const uint8_t *G, const oracle_opts *opts, oracle_result *res,
              uint8_t *witness) {
  if (!res) return ORACLE_EINVAL;
  memset(res, 0, sizeof(*res));
  if (!valid_matrix(p, n, k, G)) { res->status = ORACLE_EINVAL; return ORACLE_EINVAL; }
  oracle_opts o = {0, 1, 1, 0, 0};
  if (opts) o = *opts;

  uint8_t *gam = (uint8_t *)malloc((size_t)ORACLE_MAX_M * k * n);
  int *piv = (int *)malloc(sizeof(int) * (size_t)ORACLE_MAX_M * k);
  if (!gam || !piv) { free(gam); free(piv); res->status = ORACLE_ENOMEM; return ORACLE_ENOMEM; }
  int m = 0;
  int st = oracle_info_sets(p, n, k, G, ORACLE_MAX_M, &m, res->kj, gam, piv);
  if (st != ORACLE_OK) { free(gam); free(piv); res->status = st; return st; }
  res->m = m;

  int e[ORACLE_MAX_M];
  for (int j = 0; j < m; ++j) e[j] = 0;
  int U = n - k + 2; /* sentinel: Singleton bound n-k+1, no witness held yet */
  uint8_t best_cw[ORACLE_MAX_N], cw[ORACLE_MAX_N];
  memset(best_cw, 0, sizeof(best_cw));
  int L = lower_bound(m, e, res->kj, k);
  int status = ORACLE_OK, stop = 0;

  for (int g = 1; g <= k && !stop; ++g) {
    for (int j = 0; j < m && !stop; ++j) {
      if (o.defer && res->kj[j] < k && g < k - res->kj[j]) continue;
      for (int h = e[j] + 1; h <= g && !stop; ++h) {
        uint64_t size = oracle_pass_size(p, k, h);
        if (o.budget && (size > o.budget || res->evaluated > o.budget - size)) {
          status = ORACLE_EBUDGET;
          stop = 1;
          break;
        }
        if (res->npasses >= ORACLE_MAX_PASSES) { status = ORACLE_EBUDGET; stop = 1; break; }
        uint64_t cnt = 0;
        int best = run_pass(p, n, k, h, gam + (size_t)j * k * n, o.threads, cw, &cnt);
        if (best < 0) { free(gam); free(piv); res->status = ORACLE_ENOMEM; return ORACLE_ENOMEM; }
        res->evaluated += cnt;
        res->counts[h] += cnt;
        if (best < U) { U = best; memcpy(best_cw, cw, (size_t)n); }
        e[j] = h;
        int P = res->npasses++;
        res->pass_g[P] = h;
        res->pass_j[P] = j;
        res->pass_best[P] = best;
        if (!o.per_round_check) {
          L = lower_bound(m, e, res->kj, k);
          if (L >= U) stop = 1;
        }
        res->pass_L[P] = lower_bound(m, e, res->kj, k);
      }
    }
    if (!stop && o.per_round_check) {
      L = lower_bound(m, e, res->kj, k);
      if (L >= U) stop = 1;
    }
  }
  if (status == ORACLE_OK && !stop) res->exhausted = 1; /* every level of Gamma_1 done */
  L = lower_bound(m, e, res->kj, k);
  res->L = L;
  res->U = U > n - k + 1 ? n - k + 1 : U;
  res->status = status;
  res->d = status == ORACLE_OK ? U : -1;
  if (witness && U <= n - k + 1) memcpy(witness, best_cw, (size_t)n);
  free(gam);
  free(piv);
  return status;
}
