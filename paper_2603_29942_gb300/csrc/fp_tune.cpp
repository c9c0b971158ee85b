// fp_tune.cpp -- measured choice of the batch launch settings
// (fpcode_autotune_batch): a coordinate search over CTAs per SM, the chunk
// size of small passes and the grouping by words per slice, each point
// timed end to end through fpcode_min_distance_batch, the choice cached per
// GPU and workload class.  Host C++ only: the CUDA work is the batch call.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fpcode.h"
#include "../../include/fpcode_testing.h"
#include "fp_internal.h"

namespace fph {

// Coordinate search on a grid: from `start`, for each dimension in turn
// evaluate every value with the others held, move to the cheapest; repeat
// until a whole round changes nothing.  Points are evaluated once (memo).
// cost(point) < 0 marks a point that cannot run.
std::vector<int> tune_coordinate(const std::vector<int> &sizes, std::vector<int> at,
                                 const std::function<double(const std::vector<int> &)> &cost, int *evals) {
  std::map<std::vector<int>, double> memo;
  auto eval = [&](const std::vector<int> &x) {
    auto it = memo.find(x);
    if (it != memo.end()) return it->second;
    const double c = cost(x);
    memo[x] = c;
    return c;
  };
  double best = eval(at);
  for (int round = 0; round < 8; ++round) {
    bool moved = false;
    for (size_t d = 0; d < sizes.size(); ++d) {
      std::vector<int> x = at;
      for (int v = 0; v < sizes[d]; ++v) {
        x[d] = v;
        const double c = eval(x);
        if (c >= 0 && (best < 0 || c < best)) {
          best = c;
          at = x;
          moved = true;
        }
      }
    }
    if (!moved) break;
  }
  if (evals) *evals = (int)memo.size();
  return at;
}

namespace {

const int kCtas[] = {0, 3, 2};
const int kSteps[] = {8, 16, 32, 64, 128};
const int kWords[] = {2, 4, 1};

std::mutex g_tune_mu;
std::map<std::string, fpcode_tuning> g_tune_cache;

// Workload class: primes present, largest words per slice and k, number of
// codes (power of two), budget (power of ten).
std::string workload_class(int num, const fpcode_desc *codes, uint64_t budget) {
  unsigned primes = 0;
  int wmax = 0, kmax = 0;
  uint64_t bmax = 0;
  for (int i = 0; i < num; ++i) {
    const int p = codes[i].p;
    primes |= p == 3 ? 1u : p == 5 ? 2u : p == 7 ? 4u : 8u;
    wmax = std::max(wmax, (codes[i].n - codes[i].k + 31) / 32);
    kmax = std::max(kmax, codes[i].k);
    bmax = std::max<uint64_t>(bmax, codes[i].budget ? codes[i].budget : budget);
  }
  char buf[96];
  std::snprintf(buf, sizeof buf, "p%s%s%s%s|W%d|k%d|n2^%d|B1e%d", primes & 1 ? "3" : "", primes & 2 ? "5" : "",
                primes & 4 ? "7" : "", primes & 8 ? "+" : "", wmax, kmax,
                num > 0 ? (int)std::ceil(std::log2((double)num)) : 0,
                bmax ? (int)std::lround(std::log10((double)bmax)) : -1);
  return buf;
}

}  // namespace
}  // namespace fph

extern "C" {

void fpcode_tuning_apply(const fpcode_tuning *t, fpcode_opts *opts) {
  if (!t || !opts) return;
  opts->ctas_per_sm = t->ctas_per_sm;
  opts->min_steps = t->min_steps;
  opts->batch_words = t->batch_words;
}

int fpcode_autotune_batch(int num, const fpcode_desc *codes, void *stream, const fpcode_opts *base, int reps,
                          fpcode_tuning *out) {
  if (num <= 0 || !codes || !out) return FPCODE_EINVAL;
  fpcode_opts o;
  fpcode_opts_default(&o);
  if (base) o = *base;
  reps = std::max(1, reps);
  char name[256] = {0};
  int sms = 0;
  if (fph::device_identity(&sms, name, sizeof name)) return FPCODE_ECUDA;  // the current GPU's name and SMs
  const std::string key = std::string(name) + "|sm" + std::to_string(sms) + "|" +
                          fph::workload_class(num, codes, o.budget);
  {
    std::lock_guard<std::mutex> lk(fph::g_tune_mu);
    auto it = fph::g_tune_cache.find(key);
    if (it != fph::g_tune_cache.end()) {
      *out = it->second;
      out->evaluated = 0;
      return FPCODE_OK;
    }
  }
  std::vector<fpcode_result> res(num);
  int err = FPCODE_OK;
  auto run = [&](const fpcode_opts &x) -> double {
    int s = fpcode_min_distance_batch(num, codes, stream, &x, res.data(), nullptr);  // warm-up
    if (s) {
      err = s;
      return -1.0;
    }
    const auto t0 = std::chrono::steady_clock::now();
    for (int r = 0; r < reps; ++r) {
      s = fpcode_min_distance_batch(num, codes, stream, &x, res.data(), nullptr);
      if (s) {
        err = s;
        return -1.0;
      }
    }
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count() / reps;
  };
  auto opts_at = [&](const std::vector<int> &x) {
    fpcode_opts y = o;
    y.ctas_per_sm = fph::kCtas[x[0]];
    y.min_steps = fph::kSteps[x[1]];
    y.batch_words = fph::kWords[x[2]];
    return y;
  };
  const std::vector<int> sizes = {3, 5, 3};
  const std::vector<int> start = {0, 2, 0};  // the defaults: occupancy limit, 32 prefixes per lane, two launches
  int evals = 0;
  const std::vector<int> best =
      fph::tune_coordinate(sizes, start, [&](const std::vector<int> &x) { return run(opts_at(x)); }, &evals);
  if (err) return err;
  fpcode_tuning t{};
  t.ctas_per_sm = fph::kCtas[best[0]];
  t.min_steps = fph::kSteps[best[1]];
  t.batch_words = fph::kWords[best[2]];
  t.evaluated = evals;
  t.ms = run(opts_at(best));
  t.ms_default = run(opts_at(start));
  if (err) return err;
  std::snprintf(t.workload_class, sizeof t.workload_class, "%s", fph::workload_class(num, codes, o.budget).c_str());
  {
    std::lock_guard<std::mutex> lk(fph::g_tune_mu);
    fph::g_tune_cache[key] = t;
  }
  *out = t;
  return FPCODE_OK;
}

int fpcode_test_tune_search(int ndim, const int *sizes, const int *start, const double *cost, int *best, int *evals) {
  if (ndim < 1 || ndim > 8 || !sizes || !start || !cost || !best) return -FPCODE_EINVAL;
  std::vector<int> sz(sizes, sizes + ndim), st(start, start + ndim);
  for (int d = 0; d < ndim; ++d)
    if (sz[d] < 1 || st[d] < 0 || st[d] >= sz[d]) return -FPCODE_EINVAL;
  auto at = [&](const std::vector<int> &x) {
    size_t idx = 0;
    for (int d = 0; d < ndim; ++d) idx = idx * (size_t)sz[d] + (size_t)x[d];
    return cost[idx];
  };
  const std::vector<int> b = fph::tune_coordinate(sz, st, at, evals);
  for (int d = 0; d < ndim; ++d) best[d] = b[d];
  return 0;
}

}  // extern "C"
