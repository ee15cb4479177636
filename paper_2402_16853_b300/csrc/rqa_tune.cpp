// rqa_tune.cpp -- the autotuner: times whole runs (copies, tile kernel,
// merges; the strip shape changes the descriptor volume the merges read) of
// one series for every tile shape -- CTA-strip width (1, 2, 4, 8 warps),
// columns per lane (4, and 2 for FP32 distances) and, where the series runs
// in row bands, the band height (the size rule's, half or double) -- and
// records the fastest for the series' class (kind, m, norm, precision,
// ceil(log2 n)), which choose_tile() then uses for every later run of that
// class in the process: single, cross, batched or served.  The table can be
// written to and read from a text file, so that tuning done once on a B300
// serves later processes.  Sect. 9 of the paper plans the automatic
// selection of the best-performing implementation at runtime; every shape
// gives the same, exact result, so tuning never changes an answer.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
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
std::map<TuneKey, TileConfig> g_table;
thread_local TileConfig t_force{0, 0, 2};
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

bool tune_lookup(int kind, int m, int norm, bool f64, int64_t n, TileConfig* out) {
  std::lock_guard<std::mutex> g(g_mu);
  auto it = g_table.find(TuneKey{kind, m, norm, f64 ? 1 : 0, bucket_of(n)});
  if (it == g_table.end()) return false;
  *out = it->second;
  return true;
}

void tune_record(int kind, int m, int norm, bool f64, int64_t n, const TileConfig& c) {
  std::lock_guard<std::mutex> g(g_mu);
  g_table[TuneKey{kind, m, norm, f64 ? 1 : 0, bucket_of(n)}] = c;
}

void tune_clear() {
  std::lock_guard<std::mutex> g(g_mu);
  g_table.clear();
}

void tune_force(int warps, int cols, int band_scale) {
  t_force = TileConfig{warps, cols, band_scale};
}
void tune_force_clear() { t_force = TileConfig{0, 0, 2}; }
void tune_apply_forced(TileConfig* c) {
  if (t_force.warps > 0) c->warps = t_force.warps;
  if (t_force.cols > 0) c->cols = t_force.cols;
  if (t_force.band_scale >= -1 && t_force.band_scale <= 1) c->band_scale = t_force.band_scale;
}

}  // namespace rqa

extern "C" const char* rqa_autotune_last_error(void) { return rqa::t_tune_error.c_str(); }

extern "C" void rqa_autotune_clear(void) { rqa::tune_clear(); }

namespace {

// Time one forced shape: the best of two runs after a warm-up (device time of
// the whole run); INFINITY if a run failed.
float time_shape(rqa::Engine& eng, const std::vector<rqa::SeriesInput>& in,
                 const rqa::TileConfig& c, int* rc, int64_t* band_rows) {
  std::vector<rqa::SeriesResult> res;
  rqa::tune_force(c.warps, c.cols, c.band_scale);
  float t = INFINITY;
  for (int rep = 0; rep < 3 && *rc == RQA_OK; ++rep) {
    *rc = eng.run(in, res, nullptr, rqa::Engine::kNoGraph);
    if (*rc == RQA_OK && rep > 0) t = std::fmin(t, eng.last_total_ms());
  }
  rqa::tune_force_clear();
  if (*rc == RQA_OK && band_rows) *band_rows = res.empty() ? 0 : res[0].stats.band_rows;
  return t;
}

// The search shared by rqa_autotune and rqa_autotune_shape: every width at
// four (and, for FP32, two) columns per lane, then, if the best runs in row
// bands, half and double the band height.  Records and returns the winner.
int tune_search(const rqa_settings* settings, const double* host_series, int64_t n_points,
                int32_t cross, rqa::TileConfig* best_out, float* best_ms, float* ms_per_width) {
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
  const bool f64 = settings->precision == RQA_PREC_FP64;
  static const int widths[4] = {1, 2, 4, 8};
  TileConfig best{0, 4, 0};
  float best_t = INFINITY;
  int64_t best_band = 0;
  for (int cols : {4, 2}) {
    if (cols == 2 && f64) continue;
    for (int q = 0; q < 4; ++q) {
      const TileConfig c{widths[q], cols, 0};
      int64_t band = 0;
      const float t = time_shape(eng, in, c, &rc, &band);
      if (rc != RQA_OK) return tune_fail(rc, eng.error());
      if (ms_per_width && cols == 4) ms_per_width[q] = t;
      if (t < best_t) {
        best_t = t;
        best = c;
        best_band = band;
      }
    }
  }
  if (best_band > 0) {  // the winner runs in row bands: try other heights
    for (int sc : {-1, 1}) {
      const TileConfig c{best.warps, best.cols, sc};
      const float t = time_shape(eng, in, c, &rc, nullptr);
      if (rc != RQA_OK) return tune_fail(rc, eng.error());
      if (t < best_t) {
        best_t = t;
        best = c;
      }
    }
  }
  tune_record(cross ? 1 : 0, settings->m, settings->norm, f64, n, best);
  if (best_out) *best_out = best;
  if (best_ms) *best_ms = best_t;
  return RQA_OK;
}

}  // namespace

extern "C" int rqa_autotune(const rqa_settings* settings, const double* host_series,
                            int64_t n_points, int32_t cross, int32_t* best_warps,
                            float* ms_per_width) {
  rqa::TileConfig best{};
  const int rc = tune_search(settings, host_series, n_points, cross, &best, nullptr, ms_per_width);
  if (rc == RQA_OK && best_warps) *best_warps = best.warps;
  return rc;
}

extern "C" int rqa_autotune_shape(const rqa_settings* settings, const double* host_series,
                                  int64_t n_points, int32_t cross, int32_t* best_warps,
                                  int32_t* best_cols, int32_t* best_band_scale, float* best_ms) {
  rqa::TileConfig best{};
  const int rc = tune_search(settings, host_series, n_points, cross, &best, best_ms, nullptr);
  if (rc == RQA_OK) {
    if (best_warps) *best_warps = best.warps;
    if (best_cols) *best_cols = best.cols;
    if (best_band_scale) *best_band_scale = best.band_scale;
  }
  return rc;
}

// Text form of the table: one class per line,
//   kind m norm f64 log2n warps cols band_scale
// lines starting with '#' are comments.
extern "C" int rqa_autotune_save(const char* path) {
  using namespace rqa;
  if (!path) return RQA_EINVAL;
  std::FILE* f = std::fopen(path, "w");
  if (!f) return tune_fail(RQA_EINVAL, std::string("cannot write ") + path);
  std::fprintf(f, "# kind m norm f64 log2n warps cols band_scale\n");
  {
    std::lock_guard<std::mutex> g(g_mu);
    for (const auto& kv : g_table) {
      const TuneKey& k = kv.first;
      const TileConfig& c = kv.second;
      std::fprintf(f, "%d %d %d %d %d %d %d %d\n", std::get<0>(k), std::get<1>(k),
                   std::get<2>(k), std::get<3>(k), std::get<4>(k), c.warps, c.cols,
                   c.band_scale);
    }
  }
  return std::fclose(f) == 0 ? RQA_OK : tune_fail(RQA_EINVAL, "write failed");
}

extern "C" int rqa_autotune_load(const char* path, int32_t* entries) {
  using namespace rqa;
  if (!path) return RQA_EINVAL;
  std::FILE* f = std::fopen(path, "r");
  if (!f) return tune_fail(RQA_EINVAL, std::string("cannot read ") + path);
  std::vector<std::pair<TuneKey, TileConfig>> got;
  char line[256];
  int lineno = 0;
  int rc = RQA_OK;
  while (std::fgets(line, sizeof line, f)) {
    ++lineno;
    if (line[0] == '#' || line[0] == '\n') continue;
    int v[8];
    if (std::sscanf(line, "%d %d %d %d %d %d %d %d", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5],
                    &v[6], &v[7]) != 8 ||
        v[0] < 0 || v[0] > 2 || v[1] < 1 || v[1] > RQA_MAX_M || v[2] < 0 || v[2] > 2 ||
        v[3] < 0 || v[3] > 1 || v[4] < 0 || v[4] > 62 ||
        !(v[5] == 1 || v[5] == 2 || v[5] == 4 || v[5] == 8) || !(v[6] == 2 || v[6] == 4) ||
        v[7] < -1 || v[7] > 1 || (v[6] == 2 && v[3] == 1)) {
      rc = tune_fail(RQA_EINVAL, std::string(path) + ": bad line " + std::to_string(lineno));
      break;
    }
    got.emplace_back(TuneKey{v[0], v[1], v[2], v[3], v[4]}, TileConfig{v[5], v[6], v[7]});
  }
  std::fclose(f);
  if (rc != RQA_OK) return rc;  // nothing recorded from a malformed file
  {
    std::lock_guard<std::mutex> g(g_mu);
    for (const auto& kv : got) g_table[kv.first] = kv.second;
  }
  if (entries) *entries = static_cast<int32_t>(got.size());
  return RQA_OK;
}
