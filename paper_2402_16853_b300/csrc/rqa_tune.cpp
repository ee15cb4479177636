// rqa_tune.cpp -- the autotuner: times a whole run (copies, tile kernel,
// merges; the width changes the descriptor volume the merges read) for every
// CTA-strip width (1, 2, 4, 8 warps of 32 lanes x 4 columns) on one series and
// records the fastest for the series' class (kind, m, norm, precision,
// ceil(log2 n)), which choose_tile() then uses for every later run of that
// class in the process -- single, cross, batched or served.  Sect. 9 of the
// paper plans the automatic selection of the best-performing implementation
// at runtime; the strip width is the choice that matters here (parallelism
// against descriptor traffic and pipeline lag).  Every width gives the same,
// exact result, so tuning never changes an answer.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/rqa.h"
#include "rqa_engine.h"

namespace rqa {

namespace {

using TuneKey = std::tuple<int, int, int, int, int>;  // kind, m, norm, f64, bucket
std::mutex g_mu;
std::map<TuneKey, int> g_table;
thread_local int t_force = 0;
thread_local std::string t_tune_error;

int bucket_of(int64_t n) {
  int b = 0;
  while ((int64_t(1) << b) < n && b < 62) ++b;
  return b;
}

// SplitMix64: a fixed, published generator, so the synthetic series is the
// same on every machine.
uint64_t splitmix64(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// z-scored AR(1) series x_t = 0.95 x_{t-1} + N(0, 1) (Box-Muller normals).
std::vector<double> synthetic_series(int64_t N) {
  std::vector<double> s(static_cast<size_t>(N));
  uint64_t st = 12345;
  double x = 0.0, sum = 0.0;
  for (int64_t t = 0; t < N; ++t) {
    const double u1 = (static_cast<double>(splitmix64(st) >> 11) + 1.0) * 0x1p-53;
    const double u2 = static_cast<double>(splitmix64(st) >> 11) * 0x1p-53;
    const double g = std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    x = 0.95 * x + g;
    s[t] = x;
    sum += x;
  }
  const double mean = sum / static_cast<double>(N);
  double var = 0.0;
  for (double v : s) var += (v - mean) * (v - mean);
  const double sd = std::sqrt(var / static_cast<double>(N));
  for (double& v : s) v = sd > 0.0 ? (v - mean) / sd : 0.0;
  return s;
}

int tune_fail(int code, const std::string& m) {
  t_tune_error = m;
  return code;
}

}  // namespace

int tune_lookup(int kind, int m, int norm, bool f64, int64_t n) {
  std::lock_guard<std::mutex> g(g_mu);
  auto it = g_table.find(TuneKey{kind, m, norm, f64 ? 1 : 0, bucket_of(n)});
  return it == g_table.end() ? 0 : it->second;
}

void tune_record(int kind, int m, int norm, bool f64, int64_t n, int warps) {
  std::lock_guard<std::mutex> g(g_mu);
  g_table[TuneKey{kind, m, norm, f64 ? 1 : 0, bucket_of(n)}] = warps;
}

void tune_clear() {
  std::lock_guard<std::mutex> g(g_mu);
  g_table.clear();
}

void tune_force_warps(int warps) { t_force = warps; }
int tune_forced_warps() { return t_force; }

}  // namespace rqa

extern "C" const char* rqa_autotune_last_error(void) { return rqa::t_tune_error.c_str(); }

extern "C" void rqa_autotune_clear(void) { rqa::tune_clear(); }

extern "C" int rqa_autotune(const rqa_settings* settings, const double* host_series,
                            int64_t n_points, int32_t cross, int32_t* best_warps,
                            float* ms_per_width) {
  using namespace rqa;
  t_tune_error.clear();
  std::string msg;
  int rc = validate_settings(settings, &msg);
  if (rc != RQA_OK) return tune_fail(rc, msg);
  if (cross != 0 && cross != 1) return tune_fail(RQA_EINVAL, "cross must be 0 or 1");
  const int64_t n = n_points - static_cast<int64_t>(settings->m - 1) * settings->tau;
  if (n_points < 1 || n < 2) return tune_fail(RQA_ESHORT, "series too short to tune on");
  if (n > RQA_MAX_N) return tune_fail(RQA_ETOOBIG, "more than RQA_MAX_N embedded vectors");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return tune_fail(RQA_ENODEV, cudaGetErrorString(e));
  std::vector<double> synth;
  if (!host_series) {
    synth = synthetic_series(n_points);
    host_series = synth.data();
  }
  Engine eng(dev);
  std::vector<SeriesInput> in(1);
  in[0].st = *settings;
  in[0].host = host_series;
  in[0].N = n_points;
  if (cross) {
    in[0].cross = true;
    in[0].host2 = host_series;
    in[0].N2 = n_points;
  }
  static const int widths[4] = {1, 2, 4, 8};
  float best = INFINITY;
  int best_w = 0;
  std::vector<SeriesResult> res;
  for (int q = 0; q < 4; ++q) {
    tune_force_warps(widths[q]);
    float t = INFINITY;
    for (int rep = 0; rep < 3 && rc == RQA_OK; ++rep) {  // the first run warms up
      rc = eng.run(in, res, nullptr, false);
      if (rc == RQA_OK && rep > 0) t = std::fmin(t, eng.last_total_ms());
    }
    tune_force_warps(0);
    if (rc != RQA_OK) return tune_fail(rc, eng.error());
    if (ms_per_width) ms_per_width[q] = t;
    if (t < best) {
      best = t;
      best_w = widths[q];
    }
  }
  tune_record(cross ? 1 : 0, settings->m, settings->norm,
              settings->precision == RQA_PREC_FP64, n, best_w);
  if (best_warps) *best_warps = best_w;
  return RQA_OK;
}
