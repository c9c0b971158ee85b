// fp_host.cpp -- host side of libfpcode (not on the hot path): Gaussian
// elimination mod p into systematic generator matrices on disjoint
// information sets, bit-sliced row multiples, the pass schedule of the
// Brouwer-Zimmermann search (Sec. 3.1, Alg. 6) and the exact rebuild of a
// witness codeword from its packed key.  Plain C++17, no CUDA.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstring>
#include <unordered_map>
#include <string>
#include <vector>

#include "../../include/fpcode_testing.h"
#include "fp_bitslice.cuh"
#include "fp_internal.h"

namespace fph {

static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }
const char *last_error() { return g_err.c_str(); }

const fpenum::Binom &binom() {
  static const fpenum::Binom b = [] {
    fpenum::Binom x;
    fpenum::fill_binom(&x);
    return x;
  }();
  return b;
}

bool is_odd_prime(int p) {
  if (p < 3 || p > 255 || p % 2 == 0) return false;
  for (int q = 3; q * q <= p; q += 2)
    if (p % q == 0) return false;
  return true;
}

namespace {

// Multiplicative inverses of F_p by exponentiation a^(p-2).
std::vector<int> inverses(int p) {
  std::vector<int> inv(p, 0);
  for (int a = 1; a < p; ++a) {
    int r = 1, base = a, e = p - 2;
    while (e) {
      if (e & 1) r = r * base % p;
      base = base * base % p;
      e >>= 1;
    }
    inv[a] = r;
  }
  return inv;
}

// Column-selection elimination on a k x n working matrix of bytes.
// `owner[r]` is the pivot column of row r in the current round (-1: free).
// Each pivot makes its row's entry 1 and clears the column in every other
// row.  The multiples v * row of the pivot row as found (v = 1 .. p-1) are
// formed once by repeated addition; the pivot row scaled to a leading 1 is
// the multiple inv(a) * row (a its entry), and subtracting f times it from
// another row adds the multiple (p - f) inv(a) * row.  Every row operation
// is an add and a conditional subtract of p per byte (vectorisable), with
// no table lookup and no division.
struct Eliminator {
  int p, n, k;
  std::vector<uint8_t> M;    // row-major, values in [0, p)
  std::vector<int> inv;
  std::vector<int> owner;
  std::vector<uint8_t> mrow;  // (p-1) x n: v * row for v = 1 .. p-1 of the current pivot row

  Eliminator(int p_, int n_, int k_, const uint8_t *G)
      : p(p_), n(n_), k(k_), M(G, G + (size_t)k_ * n_), mrow((size_t)(p_ - 1) * n_) {
    inv = inverses(p);
  }
  void new_round() { owner.assign(k, -1); }
  // o = (o + y) mod p on n bytes, o, y in [0, p), separate arrays
  static void add_mod(uint8_t *__restrict__ o, const uint8_t *__restrict__ y, int n, int p) {
    if (p < 128) {
      // byte lanes: t = o + y < 2p <= 255; t - p wraps above t exactly when
      // t < p, so the smaller of the two is t mod p (vectorises)
      const uint8_t p8 = (uint8_t)p;
      for (int i = 0; i < n; ++i) {
        const uint8_t t = (uint8_t)(o[i] + y[i]);
        const uint8_t u = (uint8_t)(t - p8);
        o[i] = t < u ? t : u;
      }
    } else {
      for (int i = 0; i < n; ++i) {
        const uint16_t t = (uint16_t)(o[i] + y[i]);
        o[i] = (uint8_t)(t >= (uint16_t)p ? t - (uint16_t)p : t);
      }
    }
  }
  // Take column c as a pivot if a free row has a nonzero entry there.
  bool take(int c) {
    // locals: the byte stores below may alias any member as far as the
    // compiler knows, which would keep it from counting (and vectorising)
    // the loops
    const int n = this->n, k = this->k, p = this->p;
    int r = -1;
    for (int q = 0; q < k; ++q)
      if (owner[q] < 0 && M[(size_t)q * n + c] != 0) {
        r = q;
        break;
      }
    if (r < 0) return false;
    uint8_t *row = &M[(size_t)r * n];
    const int a = row[c];
    uint8_t *mv = mrow.data();
    std::memcpy(mv, row, (size_t)n);  // 1 * row
    for (int v = 2; v < p; ++v) {    // v * row = (v - 1) * row + row
      std::memcpy(mv + (size_t)(v - 1) * n, mv + (size_t)(v - 2) * n, (size_t)n);
      add_mod(mv + (size_t)(v - 1) * n, row, n, p);
    }
    const int ia = inv[a];
    // the pivot row scaled to a leading 1: inv(a) * row
    if (ia != 1) std::memcpy(row, mv + (size_t)(ia - 1) * n, (size_t)n);
    // o - f * (inv(a) * row) = o + ((p - f) inv(a)) * row: the multiple of
    // row to add for each entry f, once per pivot (a division per row was
    // most of the elimination's time)
    int vf[256];
    for (int f = 1; f < p; ++f) vf[f] = (p - f) * ia % p;
    for (int q = 0; q < k; ++q) {
      if (q == r) continue;
      uint8_t *o = &M[(size_t)q * n];
      const int f = o[c];
      if (!f) continue;
      add_mod(o, mv + (size_t)(vf[f] - 1) * n, n, p);
    }
    owner[r] = c;
    return true;
  }
};

int ceil_div(int a, int b) { return (a + b - 1) / b; }

// s = a + b mod p on W words of r slices each (word-major: slice i of word w
// at [w * r + i]), by the exact bit-sliced add.
template <int RR>
void add_words_r(const uint32_t *a, const uint32_t *b, uint32_t *s, int W, int p) {
  for (int w = 0; w < W; ++w) fpbs::add_generic<RR>(a + w * RR, b + w * RR, s + w * RR, p);
}
void add_sliced_words(int r, const uint32_t *a, const uint32_t *b, uint32_t *s, int W, int p) {
  switch (r) {
    case 2: add_words_r<2>(a, b, s, W, p); break;
    case 3: add_words_r<3>(a, b, s, W, p); break;
    case 4: add_words_r<4>(a, b, s, W, p); break;
    case 5: add_words_r<5>(a, b, s, W, p); break;
    case 6: add_words_r<6>(a, b, s, W, p); break;
    case 7: add_words_r<7>(a, b, s, W, p); break;
    default: add_words_r<8>(a, b, s, W, p); break;
  }
}

// Entry e of an information set's pair table (pair leaves, p = 3 or 7),
// as the kernel builds it in shared memory: entries run over y from k - 2
// down to 0, x from y + 1 up, c from 1 to p - 1; entry (y, x, c) holds the
// signature words B_i xor B_{i+1} of B = A[y] + c A[x] (the exact add of
// Alg. 3 / Alg. 4), zero-padded to sp words, then B's slice 0 (W words).
// rows: the set's multiples, rwpad words each.
template <int P, int R>
void pair_entry(const uint32_t *rows, int k, int rwpad, int W, int sp, uint32_t e, uint32_t *out) {
  constexpr int b = P - 1;
  int y = 0, x = 0, c = 0;
  fpk::pair_entry_rows(k, b, e, &y, &x, &c);
  const uint32_t *ay = rows + (size_t)y * b * rwpad;
  const uint32_t *ax = rows + ((size_t)x * b + (c - 1)) * rwpad;
  for (int q = 0; q < sp; ++q) out[q] = 0;
  for (int w = 0; w < W; ++w) {
    uint32_t sum[R];
    fpbs::add_exact<P, R>(ay + w * R, ax + w * R, sum, P);
    for (int i = 0; i + 1 < R; ++i) out[w * (R - 1) + i] = sum[i] ^ sum[i + 1];
    out[sp + w] = sum[0];
  }
}

uint64_t sat_mul(uint64_t a, uint64_t b) {
  if (a == 0 || b == 0) return 0;
  if (a > ~0ull / b) return ~0ull;
  return a * b;
}

// C(k, g) (p-1)^(g-1), saturating.
uint64_t pass_size(int p, int k, int g) {
  uint64_t c = binom().c[k][g];
  for (int i = 1; i < g; ++i) c = sat_mul(c, (uint64_t)(p - 1));
  return c;
}

}  // namespace

int digit_bits_of(int p) { return p == 3 ? 1 : (p == 5 || p == 7) ? 4 : 8; }

namespace {

int lower_bound(const std::vector<int> &e, const std::vector<int> &kj, int k) {
  int L = 0;
  for (size_t i = 0; i < e.size(); ++i) L += std::max(0, e[i] + 1 - (k - kj[i]));
  return L;
}

int digit_bits(int p) { return digit_bits_of(p); }

// Codewords a search of a random [n, k] code over F_p is expected to take:
// d estimated by the Gilbert-Varshamov bound (the least d with
// sum_{i<d} C(n,i)(p-1)^i >= p^(n-k), in logarithms), the information sets
// taken as m = floor(n/k) full ones, and the passes of each round g summed
// until the bound after the round, m (g + 1), reaches d.  Only a guide for
// choosing the leaf form: the search itself certifies the true d.
double expected_work_of(int p, int n, int k) {
  const double lq = std::log((double)p);
  double lsum = -1e300;
  int d = 1;
  for (int i = 0; i <= n; ++i) {
    const double lt = std::lgamma(n + 1.0) - std::lgamma(i + 1.0) - std::lgamma(n - i + 1.0) + i * std::log(p - 1.0);
    lsum = lsum > lt ? lsum + std::log1p(std::exp(lt - lsum)) : lt + std::log1p(std::exp(lsum - lt));
    if (lsum >= (n - k) * lq) {
      d = i + 1;
      break;
    }
  }
  const int m = std::max(1, n / k);
  double work = 0;
  for (int g = 1; g <= k; ++g) {
    work += m * std::exp(std::lgamma(k + 1.0) - std::lgamma(g + 1.0) - std::lgamma(k - g + 1.0) + (g - 1) * std::log(p - 1.0));
    if (m * (g + 1) >= d) break;
  }
  return work;
}
// The same, remembered per (p, n, k) by each thread (about fifty lgamma and
// exp calls; a stream of codes of a few shapes asks for it once per shape).
double expected_work(int p, int n, int k) {
  thread_local std::unordered_map<uint32_t, double> memo;
  const uint32_t key = (uint32_t)p << 16 | (uint32_t)n << 8 | (uint32_t)k;
  auto it = memo.find(key);
  if (it != memo.end()) return it->second;
  const double w = expected_work_of(p, n, k);
  if (memo.size() < 4096) memo.emplace(key, w);
  return w;
}
constexpr double kPairWork = 1e8;  // pair_leaves 2: pair leaves from this much expected work on

}  // namespace

int prepare(int p, int n, int k, const uint8_t *G, const fpcode_opts &opts, Prepared *P) {
  auto t0 = std::chrono::steady_clock::now();
  if (!is_odd_prime(p)) {
    set_error("p must be an odd prime below 256");
    return FPCODE_EINVAL;
  }
  if (k < 1 || k > FPCODE_MAX_K || n < k || n > FPCODE_MAX_N || n - k > 128 || !G) {
    set_error("need 1 <= k <= 64, k <= n <= 255, n - k <= 128 and a matrix");
    return FPCODE_EINVAL;
  }
  for (size_t i = 0; i < (size_t)k * n; ++i)
    if (G[i] >= p) {
      set_error("matrix entry >= p");
      return FPCODE_EINVAL;
    }
  P->p = p;
  P->n = n;
  P->k = k;
  P->opts = opts;
  P->r = fpbs::bits_for(p);
  P->W = std::max(1, ceil_div(n - k, 32));
  P->rwpad = (P->r * P->W + 3) & ~3;
  P->variant = fpk::variant_id(p, P->r, P->W);
  // pair leaves: p = 3, 7 (pair signatures of the natural encoding), a
  // stem below the pair (k >= 3), and a pair table that fits
  P->pair = false;
  P->pair_sigp = 0;
  if (opts.pair_leaves && (p == 3 || p == 7) && k >= 3 && (opts.pair_leaves == 1 || expected_work(p, n, k) >= kPairWork)) {
    const int sigw = P->W * (P->r - 1);
    P->pair = true;
    P->pair_sigp = sigw <= 1 ? 1 : sigw <= 2 ? 2 : sigw <= 4 ? 4 : 8;
    if (P->pair_words_per_set() * 4 > kPairTableMaxBytes) {
      P->pair = false;
      P->pair_sigp = 0;
    }
  }
  {  // identity of the code and of the options that shape its schedule and keys:
     // eight bytes of G per multiply (a byte at a time was a serial chain of
     // k n multiplies, about 4 us for a 40 x 80 matrix)
    uint64_t h = 1469598103934665603ull;
    auto mix = [&h](uint64_t w) {
      h = (h ^ w) * 0x9E3779B97F4A7C15ull;
      h ^= h >> 32;
    };
    mix((uint64_t)p | (uint64_t)n << 16 | (uint64_t)k << 32);
    mix((uint64_t)opts.per_round_check | (uint64_t)opts.defer << 8 | (uint64_t)(P->pair ? 1 : 0) << 16);
    const size_t nb = (size_t)k * n;
    size_t i = 0;
    for (; i + 8 <= nb; i += 8) {
      uint64_t w;
      std::memcpy(&w, G + i, 8);  // byte order decides the value; it is only compared on one machine
      mix(w);
    }
    uint64_t tail = (uint64_t)nb << 56;
    for (int b = 0; i < nb; ++i, ++b) tail |= (uint64_t)G[i] << (8 * b);
    mix(tail);
    P->code_hash = h;
  }
  if (P->smem_bytes_per_set() > 96 * 1024) {
    set_error("bit-sliced multiples of one information set exceed 96 KiB (k (p-1) r W too large)");
    return FPCODE_EINVAL;
  }

  // --- information sets: greedy leftmost columns, disjoint fresh pivots ---
  Eliminator E(p, n, k, G);
  std::vector<char> used(n, 0);
  P->kj.clear();
  P->gam.clear();
  P->piv.clear();
  P->red.clear();
  for (;;) {
    E.new_round();
    std::vector<int> fresh;
    for (int c = 0; c < n && (int)fresh.size() < k; ++c)
      if (!used[c] && E.take(c)) fresh.push_back(c);
    if (P->kj.empty() && (int)fresh.size() < k) {
      set_error("rank(G) < k");
      return FPCODE_EINVAL;
    }
    if (fresh.empty()) break;
    int have = (int)fresh.size();
    for (int c = 0; c < n && have < k; ++c)
      if (used[c] && E.take(c)) ++have;
    if (have < k) {
      set_error("internal: information set could not be completed");
      return FPCODE_EINVAL;
    }
    if ((int)P->kj.size() >= FPCODE_MAX_M) break;
    std::vector<int> rows(k);
    for (int r = 0; r < k; ++r) rows[r] = r;
    std::sort(rows.begin(), rows.end(), [&](int a, int b) { return E.owner[a] < E.owner[b]; });
    std::vector<char> is_piv(n, 0);
    const size_t g0 = P->gam.size();
    P->gam.resize(g0 + (size_t)k * n);
    for (int q = 0; q < k; ++q) {
      const int r = rows[q];
      std::memcpy(&P->gam[g0 + (size_t)q * n], &E.M[(size_t)r * n], (size_t)n);
      P->piv.push_back(E.owner[r]);
      is_piv[E.owner[r]] = 1;
    }
    for (int c = 0; c < n; ++c)
      if (!is_piv[c]) P->red.push_back(c);
    P->kj.push_back((int)fresh.size());
    for (int c : fresh) used[c] = 1;
    if (std::find(used.begin(), used.end(), 0) == used.end()) break;
  }
  P->m = (int)P->kj.size();

  // --- bit-sliced multiples v * A_j[t] of the non-pivot part, then the
  //     pair signatures (Mersenne p) ---
  const int m = P->m, nk = n - k, R = P->r, RWP = P->rwpad, W = P->W;
  const int SIG = P->pair ? 0 : fpk::sig_words(p, R, W);
  const size_t set_words = P->table_words_per_set();
  P->table.assign((size_t)m * set_words, 0u);
  const int nk32 = W * 32;  // values padded with zeros to whole words
  std::vector<uint8_t> a(nk32, 0);
  // slice words of the values y[0..nk): word w, slice i at e[w * stride + i].
  // Eight symbols at a time: bit i of each byte, masked to the bytes' low
  // bits, times 0x0102040810204080 lands byte b's bit at bit 56 + b with no
  // carries (each product bit below 56 has one source), so the top byte is
  // the eight bits in order.
  auto slice = [&](const std::vector<uint8_t> &vals, uint32_t *e, int nbits, int stride) {
    for (int w = 0; w < W; ++w)
      for (int i = 0; i < nbits; ++i) {
        uint32_t word = 0;
        for (int g8 = 0; g8 < 4; ++g8) {
          uint64_t x;
          std::memcpy(&x, &vals[(size_t)w * 32 + 8 * g8], 8);  // little-endian: symbol b in byte b
          word |= (uint32_t)((((x >> i) & 0x0101010101010101ull) * 0x0102040810204080ull) >> 56) << (8 * g8);
        }
        e[w * stride + i] = word;
      }
  };
  // Row t's multiples: v = 1 sliced from the symbols, then v A = (v-1) A + A
  // by the exact bit-sliced add; a pair signature word i is slice i xor
  // slice i+1 of the representative's multiple.
  for (int j = 0; j < m; ++j)
    for (int t = 0; t < k; ++t) {
      const uint8_t *row = &P->gam[((size_t)j * k + t) * n];
      const int *red = &P->red[(size_t)j * nk];
      for (int q = 0; q < nk; ++q) a[q] = row[red[q]];
      uint32_t *e0 = &P->table[(size_t)j * set_words + (size_t)t * (p - 1) * RWP];
      slice(a, e0, R, R);
      for (int v = 2; v < p; ++v) add_sliced_words(R, e0 + (size_t)(v - 2) * RWP, e0, e0 + (size_t)(v - 1) * RWP, W, p);
      if (SIG) {
        uint32_t *sg = &P->table[(size_t)j * set_words + (size_t)k * (p - 1) * RWP + (size_t)t * SIG];
        const int npair = (p - 1) / 2;
        for (int pq = 0; pq < npair; ++pq) {
          const uint32_t *ec = e0 + (size_t)(fpk::pair_rep(p, pq) - 1) * RWP;
          for (int w = 0; w < W; ++w)
            for (int i = 0; i + 1 < R; ++i)
              sg[(size_t)pq * W * (R - 1) + (size_t)w * (R - 1) + i] = ec[w * R + i] ^ ec[w * R + i + 1];
        }
      }
    }

  // Pair leaves: the kernel builds each set's pair table from the staged
  // multiples (fp_kernel.cuh, build_pairs); only its threshold rule is
  // set here.
  if (P->pair) {
    // The one-popcount bound ORs the words of a pair mask before counting,
    // so a bit of it covers one position per word.  A position is set in a
    // pair mask with chance rho (p = 3: 4/9, p = 7: 36/49, for random
    // symbols); take the one-popcount bound only for thresholds 3.5
    // standard deviations under its mean, where a warp's vote rarely fires.
    const double rho = p == 3 ? 4.0 / 9.0 : 36.0 / 49.0;
    double mean = 0, var = 0;
    for (int bit = 0; bit < 32; ++bit) {
      int cnt = 0;
      for (int w = 0; w < W; ++w) cnt += 32 * w + bit < nk;
      const double q = 1.0 - std::pow(1.0 - rho, cnt);
      mean += q;
      var += q * (1.0 - q);
    }
    P->pair_quick_max = W > 1 ? std::max(0, (int)std::floor(mean - 3.5 * std::sqrt(var) + 0.5)) : 255;
  }

  // --- pass schedule ---
  P->passes.clear();
  std::vector<int> e(m, 0);
  P->L0 = lower_bound(e, P->kj, k);
  const int DB = digit_bits(p);
  const int gmax_digits = 2 + 64 / DB;
  uint64_t total = 0;
  bool truncated = false;
  for (int g = 1; g <= k && !truncated; ++g) {
    const size_t round_start = P->passes.size();
    for (int j = 0; j < m && !truncated; ++j) {
      if (opts.defer && P->kj[j] < k && g < k - P->kj[j]) continue;
      for (int h = e[j] + 1; h <= g; ++h) {
        const uint64_t size = pass_size(p, k, h);
        uint64_t nprefix = (uint64_t)k;
        uint64_t NC = 1;
        uint64_t limit = fpk::kMaxPrefix;
        if (h >= 2 && P->pair) {
          // stems: one (the empty stem) for g = 2; else (p-1)/2 * C(k-2, g-2) (p-1)^(g-3)
          limit = fpk::kMaxPrefix >> 1;  // the stem index fits 33 bits of the key
          nprefix = 1;
          if (h >= 3) {
            for (int i = 0; i < h - 3; ++i) NC = sat_mul(NC, (uint64_t)(p - 1));
            nprefix = sat_mul(sat_mul(binom().c[k - 2][h - 2], NC), (uint64_t)((p - 1) / 2));
          }
        } else if (h >= 2) {
          for (int i = 0; i < h - 2; ++i) NC = sat_mul(NC, (uint64_t)(p - 1));
          nprefix = sat_mul(binom().c[k - 1][h - 1], NC);
        }
        const bool over_budget = opts.budget && (size > opts.budget || total > opts.budget - size);
        // a level the kernels cannot take ends the schedule (status EBUDGET
        // if the search gets there): prefix indices must fit the key, the
        // coefficient counter 64 bits, the binomials of an unrank the staged
        // columns t < kBinomCols, the pass index 8 bits
        if (over_budget || size == ~0ull || nprefix >= limit || h > gmax_digits ||
            h > fpenum::kBinomCols || (int)P->passes.size() >= fpk::kMaxPasses) {
          truncated = true;
          break;
        }
        fpk::PassDesc d{};
        d.g = h;
        d.j = j;
        d.L_before = lower_bound(e, P->kj, k);
        e[j] = h;
        d.L_after = lower_bound(e, P->kj, k);
        d.size = size;
        d.nprefix = nprefix;
        d.NC = NC;
        d.pl = 1;
        d.ntasks = 1;
        P->passes.push_back(d);
        total += size;
      }
    }
    if (P->passes.size() > round_start && !truncated) P->passes.back().round_end = 1;
  }
  P->complete = truncated ? 0 : 1;
  // The g = 1 passes are the rows of the Gamma_j themselves: their least
  // weight is known now.  A search starts with it as its bound (the claims
  // cap U with it; no key stands behind it), so the tasks that start at once
  // (every early pass) filter their leaves against it instead of against
  // n - k + 2.  The outcome is unchanged: the g = 1 passes still run, record
  // that weight with its key, and the termination tests see only records.
  P->seed_u = 0;
  for (size_t q = 0; q < P->passes.size(); ++q) {
    if (P->passes[q].g != 1) continue;
    const int j = P->passes[q].j;
    for (int x = 0; x < k; ++x) {
      const uint8_t *row = &P->gam[((size_t)j * k + x) * n];
      const int *red = &P->red[(size_t)j * nk];
      int w = 1;
      for (int c = 0; c < nk; ++c) w += row[red[c]] != 0;
      if (P->seed_u == 0 || w < P->seed_u) P->seed_u = w;
    }
  }
  P->t_prepare_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return FPCODE_OK;
}

namespace {

// Task plan of pair-leaf pass d (g >= 2) for a grid of C CTAs, appended to
// P->segs.  Stems come in blocks (h, q) -- h outer, q = the stem's largest
// row ascending -- whose stems all have E(q) = (p-1) C(k-1-q, 2) entries.
// A lane's work for one stem is its share of the entries plus the stem
// step.  Tasks are guided by work: a block's tasks aim at a per-lane load
// of 1 / task_share of the pass's remaining work spread over every lane of
// the grid (at least task_work).  A stem whose entries alone exceed that target,
// or a block with too few stems to give every group one, splits its
// entries over 2^lsplit lanes (interleaved entry chunks, so a warp's loads
// stay broadcasts or consecutive words).  Each block is a segment of its
// own, so the groups of a task have equal work.
constexpr uint64_t kStemCost = 8;      // a stem step, in entry evaluations
constexpr uint64_t kMinTaskLane = 192;  // least per-lane work of a task, in entry evaluations (task_work 0)
// Guided share (task_share 0): a task takes 1 / (share C) of its pass's
// remaining work.  A pass with more passes after it in the launch takes
// share 1: CTAs that run out of its tasks move on to the next pass (run
// ahead), so its larger tasks cost no idle lanes at its end, and there are
// fewer claims.  The launch's last pass (a pass run alone: a probe, a
// slice of a split search) takes share 2, so that its tail is short.
constexpr uint64_t kTaskShareMid = 1;
constexpr uint64_t kTaskShareLast = 2;

}  // namespace

int task_share_of(const fpcode_opts &o, bool last) {
  return o.task_share > 0 ? o.task_share : (int)(last ? kTaskShareLast : kTaskShareMid);
}

namespace {
constexpr uint64_t kSpreadLane = 4;    // a pass of at most this much work per lane of the grid is spread wide

// Quotients of the task plans: 64-bit division only where 32 bits do not
// hold the operands.
inline uint64_t div_floor(uint64_t a, uint64_t b) {
  return (a | b) >> 32 ? a / b : (uint64_t)((uint32_t)a / (uint32_t)b);
}
inline uint64_t div_up(uint64_t a, uint64_t b) { return div_floor(a + b - 1, b); }
// floor(a / b) from a reciprocal of b, corrected to the exact quotient
inline uint64_t div_floor_rcp(uint64_t a, uint64_t b, double binv) {
  uint64_t q = (uint64_t)((double)a * binv);
  while (q > 0 && q * b > a) --q;
  while ((q + 1) * b <= a) ++q;
  return q;
}

void plan_pair_pass(Prepared *P, fpk::PassDesc &d, uint64_t C, bool last) {
  const int k = P->k, b = P->p - 1, g = d.g;
  const int H = g == 2 ? 1 : b / 2;
  const uint64_t lanes = (uint64_t)fpk::kThreads;
  struct Blk {
    int h, q;
    uint64_t n;  // stems
    uint64_t E;  // entries per stem
  };
  std::vector<Blk> blks;
  blks.reserve(g == 2 ? 1 : (size_t)H * (size_t)(k - g + 1));
  if (g == 2) {
    blks.push_back({1, -1, 1, (uint64_t)fpk::pair_entries_above(k, -1, b)});
  } else {
    for (int h = 1; h <= H; ++h)
      for (int q = g - 3; q <= k - 3; ++q)
        blks.push_back({h, q, binom().c[q][g - 3] * d.NC, (uint64_t)fpk::pair_entries_above(k, q, b)});
  }
  // work in entries plus the stems' cost: below 2^33 stems x 2^14 entries per block, so exact in 64 bits
  uint64_t rem = 0;
  for (auto &x : blks) rem += x.n * (x.E + kStemCost);
  // A small pass (the first passes of a search, which run before records
  // exist and send most entries down the exact path) is spread as wide as
  // the grid allows: one stem per group, a stem's entries over as many
  // lanes as keeps two loads per lane.
  const bool spread = rem <= C * lanes * kSpreadLane;
  const uint64_t Tmin = P->opts.task_work > 0 ? (uint64_t)P->opts.task_work : kMinTaskLane;
  const uint64_t share = (uint64_t)task_share_of(P->opts, last);
  const uint64_t T_spread = std::max<uint64_t>(2, rem / (C * lanes) + 1);
  // Stems of one group start on the same phase of the coefficient counter
  // (units of (p-1)^t stems, t <= g - 3), so the lanes of a warp take the
  // same Gray steps and rebuild their sums at the same stem.
  const int L = g >= 3 ? g - 3 : 0;
  d.seg_off = (uint32_t)P->segs.size();
  uint32_t tasks = 0;
  int cur_l = -1, cur_spg = -1;  // shape of the open segment
  uint64_t cur_n = 0;            // its stems so far
  auto close = [&]() {
    if (cur_l < 0) return;
    const uint64_t per = (lanes >> cur_l) * (uint64_t)cur_spg;
    tasks += (uint32_t)div_up(cur_n, per);
    P->segs.back().task_end = tasks;
  };
  // the per-block quotients below are the plan's cost (a pass has up to
  // (p-1)/2 (k-2) blocks, a schedule a few hundred): the pass's divisor
  // goes through a reciprocal (then corrected to the exact quotient), the
  // others through 32 bits where they fit
  const uint64_t Dg = share * C * lanes;
  const double Dinv = 1.0 / (double)Dg;
  const int lanes_log = __builtin_ctzll(lanes);  // kThreads is a power of two
  for (auto &x : blks) {
    const uint64_t T = spread ? T_spread : std::max<uint64_t>(Tmin, div_floor_rcp(rem, Dg, Dinv));
    int l = 0;
    // split a stem's entries while one lane's share exceeds the target, or
    // while the block cannot give every group a stem (at least two entry
    // pairs per lane per stem)
    while (l < 8 && x.E >> (l + 1) >= 4 &&
           (((x.E + (1ull << l) - 1) >> l) + kStemCost > T || (lanes >> l) > x.n))
      ++l;
    const uint64_t per_stem = ((x.E + (1ull << l) - 1) >> l) + kStemCost;
    uint64_t want = spread ? 1 : std::max<uint64_t>(1, div_floor(T + per_stem / 2, per_stem));
    // no more stems per group than spreads the block over every group
    want = std::min<uint64_t>(want, (x.n + (lanes >> l) - 1) >> (lanes_log - l));
    // at most 65535 stems per group (the segment's field), in whole units
    // of the coefficient counter, and at least one unit (a unit chosen
    // before the cap could exceed it and leave zero stems per group)
    want = std::min<uint64_t>(want, 65535);
    uint64_t unit = 1;
    for (int t = 0; t < L && unit * (uint64_t)b <= want; ++t) unit *= (uint64_t)b;
    want = unit == 1 ? want : (uint32_t)want / (uint32_t)unit * unit;
    const int spg = (int)want;
    {  // one segment per block: every stem of a task has the same entries, so its groups finish together
      close();
      fpk::PairSeg s{};
      s.task_end = 0;
      s.spg = (uint16_t)spg;
      s.q = x.q < 0 ? (uint8_t)255 : (uint8_t)x.q;
      s.hsplit = (uint8_t)(((x.h - 1) << 4) | l);
      P->segs.push_back(s);
      cur_l = l;
      cur_spg = spg;
      cur_n = 0;
    }
    cur_n += x.n;
    rem -= x.n * (x.E + kStemCost);
  }
  close();
  d.nseg = (uint32_t)P->segs.size() - d.seg_off;
  d.ntasks = tasks;
  d.pl = 0;
  d.phases = 0;
  d.unit = 1;
}

}  // namespace

void plan_tasks(Prepared *P, int ctas, int fixed_pl, int min_steps, bool spread_tiny) {
  const uint64_t lanes = (uint64_t)fpk::kThreads;
  const uint64_t C = (uint64_t)std::max(1, ctas);
  const uint64_t b = (uint64_t)(P->p - 1);
  P->segs.clear();
  for (auto &d : P->passes) {
    d.phases = 0;
    d.plan_ctas = (uint32_t)C;
    d.unit = 1;
    d.seg_off = 0;
    d.nseg = 0;
    if (d.g == 1) {
      d.pl = 1;
      d.ntasks = 1;
      continue;
    }
    if (P->pair) {
      plan_pair_pass(P, d, C, &d == &P->passes.back());
      continue;
    }
    if (fixed_pl > 0) {
      d.pl = std::min(fixed_pl, 64);
      const uint64_t per_task = lanes * (uint64_t)d.pl;
      d.ntasks = (uint32_t)((d.nprefix + per_task - 1) / per_task);
      continue;
    }
    d.pl = 0;
    // unit b^t: as many whole low digits as keep two units per lane of the grid
    uint64_t unit = 1;
    for (int t = 0; t < d.g - 2; ++t) {
      if (unit * b > 256 || d.nprefix / (unit * b) < 2 * lanes * C) break;
      unit *= b;
    }
    d.unit = (uint32_t)unit;
    const uint64_t N = d.nprefix / unit;
    // small pass (fewer than min_steps prefixes per lane of the grid): fixed
    // tasks of min_steps prefixes per lane on part of the grid, which takes
    // up the following passes meanwhile; a lane's setup (unranking its first
    // prefix, summing its rows) then serves several prefixes
    const uint64_t umin = ((uint64_t)std::max(1, min_steps) + unit - 1) / unit;
    if (spread_tiny && N <= lanes * C) {  // under one unit per lane of the grid: spread it wide
      d.ntasks = (uint32_t)((N + lanes - 1) / lanes);
      continue;
    }
    if (N < lanes * C * umin) {
      d.pl = (int32_t)umin;
      d.ntasks = (uint32_t)((N + lanes * umin - 1) / (lanes * umin));
      continue;
    }
    if (N <= 2 * lanes * C) {  // small pass: one unit per lane
      d.ntasks = (uint32_t)((N + lanes - 1) / lanes);
      continue;
    }
    // guided rows (task_range): tasks shrink as the pass drains, down to one
    // unit per lane
    uint32_t H = 0;
    d.ntasks = (uint32_t)fpk::guided_phases((N + lanes - 1) / lanes, C, [&](uint64_t, uint64_t) {
      ++H;
      return false;
    });
    d.phases = H;
  }
  // one task sequence over all passes
  uint64_t base = 0;
  for (auto &d : P->passes) {
    d.task_base = (uint32_t)base;
    base += d.ntasks;
  }
}

// Coefficients (length k) of the codeword a key stands for.
bool key_coefficients(const Prepared &P, uint64_t key, int *g_out, int *j_out, std::vector<int> &coef) {
  const int pass = (int)fpk::key_pass(key);
  if (pass >= (int)P.passes.size()) return false;
  const fpk::PassDesc &d = P.passes[pass];
  coef.assign(P.k, 0);
  if (P.pair && d.g >= 2) {
    // stem J: h and the prefix over rows 0..k-2 at level g - 1; entry e:
    // (y, x, c); sign 1: the codeword S - B, i.e. y and x negated
    const int b = P.p - 1, g = d.g;
    const uint64_t J = fpk::pair_key_stem(key);
    const uint32_t e = fpk::pair_key_entry(key);
    const int sign = (int)fpk::pair_key_sign(key);
    if (J >= d.nprefix || e >= (uint32_t)b * (uint32_t)(P.k * (P.k - 1) / 2) || (g == 2 && sign)) return false;
    int y, x, c;
    fpk::pair_entry_rows(P.k, b, e, &y, &x, &c);
    int q = -1;
    if (g >= 3) {
      const int L = g - 3;
      const uint64_t N1 = binom().c[P.k - 2][g - 2] * d.NC;
      const int h = (int)(J / N1) + 1;
      const uint64_t I1 = J % N1;
      const int DB = digit_bits(P.p);
      fpenum::Prefix pf = DB == 1 ? fpenum::prefix_unrank<1>(binom(), I1, P.k - 1, g - 1, b)
                                  : fpenum::prefix_unrank<4>(binom(), I1, P.k - 1, g - 1, b);
      q = pf.m;
      coef[q] = h;
      uint64_t Q = pf.Q;
      for (int s = 0; s < L; ++s) {
        const int r = fpenum::ctz64(Q);
        Q &= Q - 1;
        coef[r] = (DB == 1 ? fpenum::gray_digit<1>(pf.d, s, b, L) : fpenum::gray_digit<4>(pf.d, s, b, L)) + 1;
      }
    }
    if (y <= q) return false;  // entries of this stem have y > q
    coef[y] = sign ? P.p - 1 : 1;
    coef[x] = sign ? P.p - c : c;
    *g_out = g;
    *j_out = d.j;
    return true;
  }
  const int x = (int)fpk::key_leaf(key);
  const int c = (int)fpk::key_coef(key);
  if (x >= P.k || c < 1 || c >= P.p) return false;
  if (d.g == 1) {
    coef[x] = 1;
  } else {
    const uint64_t I = fpk::key_prefix(key);
    if (I >= d.nprefix) return false;
    const int L = d.g - 2, b = P.p - 1;
    const int DB = digit_bits(P.p);
    fpenum::Prefix pf = DB == 1   ? fpenum::prefix_unrank<1>(binom(), I, P.k, d.g, b)
                        : DB == 4 ? fpenum::prefix_unrank<4>(binom(), I, P.k, d.g, b)
                                  : fpenum::prefix_unrank<8>(binom(), I, P.k, d.g, b);
    if (pf.m >= x) return false;
    coef[pf.m] = 1;
    uint64_t Q = pf.Q;
    for (int s = 0; s < L; ++s) {
      const int q = fpenum::ctz64(Q);
      Q &= Q - 1;
      coef[q] = (DB == 1   ? fpenum::gray_digit<1>(pf.d, s, b, L)
                 : DB == 4 ? fpenum::gray_digit<4>(pf.d, s, b, L)
                           : fpenum::gray_digit<8>(pf.d, s, b, L)) + 1;
    }
    coef[x] = c;
  }
  *g_out = d.g;
  *j_out = d.j;
  return true;
}

int decode_result(const Prepared &P, const DeviceOutcome &o, fpcode_result *res, uint8_t *witness) {
  std::memset(res, 0, sizeof(*res));
  res->m = P.m;
  for (int j = 0; j < P.m && j < FPCODE_MAX_M; ++j) res->kj[j] = P.kj[j];
  res->enumerated = o.enumerated;
  res->t_prepare_ms = P.t_prepare_ms;
  const int singleton = P.n - P.k + 1;
  res->npasses = o.stop_pass + 1;
  for (int i = 0; i <= o.stop_pass && i < (int)P.passes.size(); ++i) res->counts[P.passes[i].g] += P.passes[i].size;
  res->L = o.stop_pass >= 0 ? P.passes[o.stop_pass].L_after : P.L0;
  // a key whose pass is outside the schedule is a seeded bound, not a codeword
  const bool seeded = o.best_key != fpk::kNoKey && fpk::key_pass(o.best_key) >= P.passes.size();
  const bool have = o.best_key != fpk::kNoKey && !seeded;
  res->U = o.best_key != fpk::kNoKey ? std::min<int>((int)fpk::key_weight(o.best_key), singleton) : singleton;
  res->best_key = have ? o.best_key : fpk::kNoKey;
  res->status = o.status < 0 ? FPCODE_ETIMEOUT : o.status;
  res->d = -1;
  if (res->status == FPCODE_OK) {
    if (!have) {
      set_error("internal: certified without a witness");
      res->status = FPCODE_ECUDA;
      return res->status;
    }
    res->d = (int)fpk::key_weight(o.best_key);
  }
  if (have && (witness || res->status == FPCODE_OK)) {
    int g, j;
    std::vector<int> coef;
    if (!key_coefficients(P, o.best_key, &g, &j, coef)) {
      set_error("internal: witness key does not decode");
      res->status = FPCODE_ECUDA;
      return res->status;
    }
    std::vector<uint8_t> cw(P.n, 0);
    int nnz = 0;
    for (int t = 0; t < P.k; ++t)
      if (coef[t]) {
        ++nnz;
        const uint8_t *row = &P.gam[((size_t)j * P.k + t) * P.n];
        for (int c = 0; c < P.n; ++c) cw[c] = (uint8_t)((cw[c] + coef[t] * row[c]) % P.p);
      }
    int wt = 0;
    for (int c = 0; c < P.n; ++c) wt += cw[c] != 0;
    if (nnz != g || wt != (int)fpk::key_weight(o.best_key)) {
      set_error("internal: rebuilt witness has the wrong weight");
      res->status = FPCODE_ECUDA;
      return res->status;
    }
    if (witness) std::memcpy(witness, cw.data(), (size_t)P.n);
  }
  return res->status;
}

}  // namespace fph

// ---------------------------------------------------------------------------
// Host-side hooks declared in fpcode_testing.h.
// ---------------------------------------------------------------------------
extern "C" {

int fpcode_test_bitslice_host(int op, int p, const uint32_t *a, const uint32_t *b, uint32_t *out) {
  if (!fph::is_odd_prime(p) || !a || !out) return FPCODE_EINVAL;
  const int r = fpbs::bits_for(p);
  const bool mersenne = ((p + 1) & p) == 0;
  switch (op) {
    case FPCODE_OP_ADD:
      if (!b) return FPCODE_EINVAL;
      if (p == 3) fpbs::add_exact<3, 2>(a, b, out, p);
      else if (p == 7) fpbs::add_exact<7, 3>(a, b, out, p);
      else if (p == 31) fpbs::add_exact<31, 5>(a, b, out, p);
      else if (p == 127) fpbs::add_exact<127, 7>(a, b, out, p);
      else {
        switch (r) {
          case 3: fpbs::add_generic<3>(a, b, out, p); break;
          case 4: fpbs::add_generic<4>(a, b, out, p); break;
          case 5: fpbs::add_generic<5>(a, b, out, p); break;
          case 6: fpbs::add_generic<6>(a, b, out, p); break;
          case 7: fpbs::add_generic<7>(a, b, out, p); break;
          case 8: fpbs::add_generic<8>(a, b, out, p); break;
          default: return FPCODE_EINVAL;
        }
      }
      return FPCODE_OK;
    case FPCODE_OP_NZ_SUB: {
      if (!b) return FPCODE_EINVAL;
      uint32_t mask = 0;
      for (int i = 0; i < r; ++i) mask |= a[i] ^ b[i];
      out[0] = mask;
      return FPCODE_OK;
    }
    case FPCODE_OP_NZ_ADD:
      if (!b) return FPCODE_EINVAL;
      if (p == 3) out[0] = fpbs::nz_add_p3(a[0], a[1], b[0], b[1]);
      else if (p == 7) out[0] = fpbs::nz_add_mersenne<3>(a, b);
      else if (p == 31) out[0] = fpbs::nz_add_mersenne<5>(a, b);
      else if (p == 127) out[0] = fpbs::nz_add_mersenne<7>(a, b);
      else return FPCODE_EINVAL;
      return FPCODE_OK;
    case FPCODE_OP_NEG:
      if (!mersenne) return FPCODE_EINVAL;
      if (p == 3) fpbs::neg_mersenne<2>(a, out);
      else if (p == 7) fpbs::neg_mersenne<3>(a, out);
      else if (p == 31) fpbs::neg_mersenne<5>(a, out);
      else fpbs::neg_mersenne<7>(a, out);
      return FPCODE_OK;
    case FPCODE_OP_MUL2:
      if (!mersenne) return FPCODE_EINVAL;
      if (p == 3) fpbs::mul_pow2_mersenne<2>(a, out, 1);
      else if (p == 7) fpbs::mul_pow2_mersenne<3>(a, out, 1);
      else if (p == 31) fpbs::mul_pow2_mersenne<5>(a, out, 1);
      else fpbs::mul_pow2_mersenne<7>(a, out, 1);
      return FPCODE_OK;
    default:
      return FPCODE_EINVAL;
  }
}

uint64_t fpcode_test_rd_unrank(uint64_t rank, int n, int t) { return fpenum::rd_unrank(fph::binom(), rank, n, t); }
uint64_t fpcode_test_rd_rank(uint64_t subset, int n, int t) { return fpenum::rd_rank(fph::binom(), subset, n, t); }
int fpcode_test_rd_next(uint64_t subset, int n, int t, uint64_t *next) {
  int rm, ad;
  return fpenum::rd_next(subset, n, t, next, &rm, &ad) ? 1 : 0;
}

extern "C++" {
namespace {
template <int DB>
int prefix_out(const fpenum::Prefix &pf, int g, int p, int *m, uint64_t *Q, int *coefs) {
  *m = pf.m;
  *Q = pf.Q;
  const int L = g - 2, b = p - 1;
  for (int s = 0; s < L; ++s) coefs[s] = fpenum::gray_digit<DB>(pf.d, s, b, L) + 1;
  return FPCODE_OK;
}

template <int DB>
int prefix_walk(uint64_t I, uint64_t steps, int k, int g, int p, int *m, uint64_t *Q, int *coefs) {
  const fpenum::Binom &B = fph::binom();
  const int L = g - 2, b = p - 1;
  const uint64_t NC = fpenum::ipow((uint64_t)b, L);
  fpenum::Prefix pf = fpenum::prefix_unrank<DB>(B, I, k, g, b);
  uint64_t ci = (I - fpenum::prefixes_below(B, pf.m, g, NC)) - pf.qi * NC;
  uint64_t nq = B(pf.m, L);
  for (uint64_t s = 0; s < steps; ++s) {
    int dir;
    fpenum::prefix_advance<DB>(B, pf, ci, nq, NC, b, L, &dir);
  }
  return prefix_out<DB>(pf, g, p, m, Q, coefs);
}
}  // namespace
}  // extern "C++"

int fpcode_test_prefix_unrank(uint64_t I, int k, int g, int p, int *m, uint64_t *Q, int *coefs) {
  if (g < 2 || g > k || k > 64 || !fph::is_odd_prime(p)) return FPCODE_EINVAL;
  switch (fph::digit_bits_of(p)) {
    case 1: return prefix_out<1>(fpenum::prefix_unrank<1>(fph::binom(), I, k, g, p - 1), g, p, m, Q, coefs);
    case 4: return prefix_out<4>(fpenum::prefix_unrank<4>(fph::binom(), I, k, g, p - 1), g, p, m, Q, coefs);
    default: return prefix_out<8>(fpenum::prefix_unrank<8>(fph::binom(), I, k, g, p - 1), g, p, m, Q, coefs);
  }
}

int fpcode_test_prefix_walk(uint64_t I, uint64_t steps, int k, int g, int p, int *m, uint64_t *Q, int *coefs) {
  if (g < 2 || g > k || k > 64 || !fph::is_odd_prime(p)) return FPCODE_EINVAL;
  switch (fph::digit_bits_of(p)) {
    case 1: return prefix_walk<1>(I, steps, k, g, p, m, Q, coefs);
    case 4: return prefix_walk<4>(I, steps, k, g, p, m, Q, coefs);
    default: return prefix_walk<8>(I, steps, k, g, p, m, Q, coefs);
  }
}

int fpcode_test_task_ranges(fpcode_prepared *prep, int pass, int ctas, int fixed_pl, int min_steps, uint64_t *lo,
                            uint64_t *hi, int max) {
  if (!prep || pass < 0 || pass >= (int)prep->host.passes.size() || !lo || !hi) return -1;
  fph::plan_tasks(&prep->host, ctas, fixed_pl, min_steps, min_steps <= fph::kMinStepsSingle);
  const fpk::PassDesc &d = prep->host.passes[pass];
  const int n = (int)std::min<uint64_t>(d.ntasks, (uint64_t)max);
  for (int t = 0; t < n; ++t) {
    if (d.g == 1) {
      lo[t] = 0;
      hi[t] = d.nprefix;
    } else if (d.nseg > 0) {
      int ls = 0;
      fpk::pair_task(d, &prep->host.segs[d.seg_off], prep->host.k, fph::binom(), (uint64_t)t, &lo[t], &hi[t], &ls);
    } else {
      fpk::task_range(d, (uint64_t)t, &lo[t], &hi[t]);
      lo[t] *= d.unit;
      hi[t] *= d.unit;
      if (hi[t] > d.nprefix) hi[t] = d.nprefix;
    }
  }
  return (int)d.ntasks;
}

int fpcode_test_lane_ranges(fpcode_prepared *prep, int pass, int ctas, int fixed_pl, int min_steps, uint64_t *lo,
                            uint64_t *hi, int max) {
  if (!prep || pass < 0 || pass >= (int)prep->host.passes.size() || !lo || !hi || max < 0) return -1;
  fph::plan_tasks(&prep->host, ctas, fixed_pl, min_steps, min_steps <= fph::kMinStepsSingle);
  const fpk::PassDesc &d = prep->host.passes[pass];
  if (d.g < 2 || d.nseg > 0) return -1;  // one-row passes with g >= 2 only
  const uint64_t total = (uint64_t)d.ntasks * fpk::kThreads;
  int n = 0;
  for (uint64_t t = 0; t < d.ntasks && n < max; ++t)
    for (int lane = 0; lane < fpk::kThreads && n < max; ++lane, ++n) {
      // as the kernel splits a task's units over its lanes (task_prefixes)
      uint64_t ulo = 0, uhi = 0;
      fpk::task_range(d, t, &ulo, &uhi);
      const uint64_t pu = (uhi - ulo + fpk::kThreads - 1) / fpk::kThreads;
      const uint64_t a = (ulo + (uint64_t)lane * pu) * d.unit;
      const uint64_t e = std::min(uhi * d.unit, d.nprefix);
      lo[n] = std::min(a, e);
      hi[n] = std::min(a + pu * d.unit, e);
    }
  return (int)std::min<uint64_t>(total, (uint64_t)INT32_MAX);
}

int fpcode_test_pair_mode(const fpcode_prepared *prep, int pass, uint64_t J, uint32_t *entries) {
  if (!prep) return -FPCODE_EINVAL;
  const fph::Prepared &P = prep->host;
  if (pass >= 0) {
    if (pass >= (int)P.passes.size() || !entries || !P.pair) return -FPCODE_EINVAL;
    const fpk::PassDesc &d = P.passes[pass];
    if (d.g < 2 || J >= d.nprefix) return -FPCODE_EINVAL;
    int q = -1;
    if (d.g >= 3) {
      const uint64_t N1 = fph::binom().c[P.k - 2][d.g - 2] * d.NC;
      const int b = P.p - 1;
      q = fph::digit_bits_of(P.p) == 1 ? fpenum::prefix_unrank<1>(fph::binom(), J % N1, P.k - 1, d.g - 1, b).m
                                       : fpenum::prefix_unrank<4>(fph::binom(), J % N1, P.k - 1, d.g - 1, b).m;
    }
    *entries = fpk::pair_entries_above(P.k, q, P.p - 1);
  }
  return P.pair ? P.pair_sigp : 0;
}

int fpcode_test_key_coefficients(const fpcode_prepared *prep, uint64_t key, int *g, int *j, int *coef) {
  if (!prep || !g || !j || !coef) return -1;
  std::vector<int> c;
  if (!fph::key_coefficients(prep->host, key, g, j, c)) return -1;
  for (int t = 0; t < prep->host.k; ++t) coef[t] = c[t];
  return 0;
}

int fpcode_prepared_shape(const fpcode_prepared *prep, int *m, int *kj, int *npasses, int *complete) {
  const fph::Prepared *P = prep ? &prep->host : nullptr;
  if (!P) return FPCODE_EINVAL;
  if (m) *m = P->m;
  if (kj)
    for (int j = 0; j < P->m; ++j) kj[j] = P->kj[j];
  if (npasses) *npasses = (int)P->passes.size();
  if (complete) *complete = P->complete;
  return FPCODE_OK;
}

int fpcode_prepared_gamma(const fpcode_prepared *prep, int j, uint8_t *gamma, int *pivots) {
  const fph::Prepared *P = prep ? &prep->host : nullptr;
  if (!P || j < 0 || j >= P->m) return FPCODE_EINVAL;
  if (gamma) std::memcpy(gamma, &P->gam[(size_t)j * P->k * P->n], (size_t)P->k * P->n);
  if (pivots)
    for (int r = 0; r < P->k; ++r) pivots[r] = P->piv[(size_t)j * P->k + r];
  return FPCODE_OK;
}

int fpcode_test_prepared_row(const fpcode_prepared *prep, int j, int t, int v, uint32_t *slices, uint32_t *sig) {
  const fph::Prepared *P = prep ? &prep->host : nullptr;
  if (!P || j < 0 || j >= P->m || t < 0 || t >= P->k || v < 1 || v >= P->p || !slices) return FPCODE_EINVAL;
  const size_t set_words = P->table_words_per_set();
  const uint32_t *e = &P->table[(size_t)j * set_words + ((size_t)t * (P->p - 1) + (v - 1)) * P->rwpad];
  std::memcpy(slices, e, (size_t)P->r * P->W * sizeof(uint32_t));
  const int SIG = P->pair ? 0 : fpk::sig_words(P->p, P->r, P->W);  // pair leaves keep no row signatures
  if (sig && SIG) {
    const uint32_t *sg = &P->table[(size_t)j * set_words + (size_t)P->k * (P->p - 1) * P->rwpad + (size_t)t * SIG];
    std::memcpy(sig, sg, (size_t)SIG * sizeof(uint32_t));
  }
  return SIG;
}

int fpcode_test_pair_entry(const fpcode_prepared *prep, int j, uint32_t e, uint32_t *sig) {
  const fph::Prepared *P = prep ? &prep->host : nullptr;
  if (!P || !P->pair || j < 0 || j >= P->m || !sig) return -FPCODE_EINVAL;
  const uint32_t ne = (uint32_t)(P->p - 1) * (uint32_t)(P->k * (P->k - 1) / 2);
  if (e >= ne) return -FPCODE_EINVAL;
  const uint32_t *rows = &P->table[(size_t)j * P->table_words_per_set()];
  if (P->p == 3) fph::pair_entry<3, 2>(rows, P->k, P->rwpad, P->W, P->pair_sigp, e, sig);
  else fph::pair_entry<7, 3>(rows, P->k, P->rwpad, P->W, P->pair_sigp, e, sig);
  return P->pair_sigp + P->W;
}

int fpcode_prepared_codeword(const fpcode_prepared *prep, uint64_t key, uint8_t *codeword, int *weight) {
  if (!prep || !codeword) return FPCODE_EINVAL;
  const fph::Prepared &P = prep->host;
  int g = 0, j = 0;
  std::vector<int> coef;
  if (key == fpk::kNoKey || !fph::key_coefficients(P, key, &g, &j, coef)) {
    fph::set_error("fpcode_prepared_codeword: the key names no codeword of the schedule");
    return FPCODE_EINVAL;
  }
  std::vector<uint8_t> cw(P.n, 0);
  for (int t = 0; t < P.k; ++t)
    if (coef[t]) {
      const uint8_t *row = &P.gam[((size_t)j * P.k + t) * P.n];
      for (int c = 0; c < P.n; ++c) cw[c] = (uint8_t)((cw[c] + coef[t] * row[c]) % P.p);
    }
  int wt = 0;
  for (int c = 0; c < P.n; ++c) wt += cw[c] != 0;
  std::memcpy(codeword, cw.data(), (size_t)P.n);
  if (weight) *weight = wt;
  return FPCODE_OK;
}

int fpcode_prepared_passes(const fpcode_prepared *prep, fpcode_pass_info *passes, int max) {
  const fph::Prepared *P = prep ? &prep->host : nullptr;
  if (!P || !passes) return FPCODE_EINVAL;
  int n = std::min<int>(max, (int)P->passes.size());
  for (int i = 0; i < n; ++i) {
    const fpk::PassDesc &d = P->passes[i];
    passes[i].g = d.g;
    passes[i].j = d.j;
    passes[i].L_before = d.L_before;
    passes[i].L_after = d.L_after;
    passes[i].round_end = d.round_end;
    passes[i].ntasks = (int)d.ntasks;
    passes[i].size = d.size;
    passes[i].nprefix = d.nprefix;
  }
  return n;
}

}  // extern "C"
