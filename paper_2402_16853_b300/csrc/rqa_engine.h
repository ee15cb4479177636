// rqa_engine.h -- run engine shared by the single-series, batched and served
// entry points: plans device memory for a set of series, launches prepare ->
// embed -> tile (one persistent launch per kernel class) -> merge ->
// finalize on one stream, and turns the histograms into measures.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/rqa.h"
#include "rqa_internal.h"

namespace rqa {

struct SeriesInput {
  rqa_settings st;
  const double* host = nullptr;  // copied to the device
  const double* dev = nullptr;   // used in place (caller's device memory)
  int64_t N = 0;
  // cross recurrence (Sect. 3.3): the column series, host or device
  bool cross = false;
  const double* host2 = nullptr;
  const double* dev2 = nullptr;
  int64_t N2 = 0;
  // precomputed matrix (Sect. 9): N rows x N2 columns of bits, row-major,
  // ceil(N2 / 32) words per row, host or device (cross is set as well)
  bool matrix = false;
  const uint32_t* bits_host = nullptr;
  const uint32_t* bits_dev = nullptr;
  // self-test of the bounded ring waits (rqa_selftest_ring_timeout): run
  // the tile kernel's test instantiation with warp withhold_warp - 1
  // withholding its hand-overs from the withhold_seq-th on (0: off)
  int32_t withhold_warp = 0, withhold_seq = 0;
};

struct SeriesResult {
  int status = RQA_OK;
  int64_t n = 0;               // rows (embedded vectors of the series)
  int64_t n2 = 0;              // columns (== n for RQA)
  int64_t hl = 0;              // histogram length - 1: n, or max(n, n2)
  // 3 * (hl + 1) counts: diagonal, vertical, white vertical.  Points into
  // the engine's pinned staging buffer: valid until the engine's next run.
  const uint64_t* hist = nullptr;
  rqa_measures_t meas{};
  rqa_stats_t stats{};
};

// Validation shared by every entry point.  Returns RQA_OK or an error code
// and a message.
int validate_settings(const rqa_settings* st, std::string* msg);

// Tile configuration (warps per CTA strip, columns per lane, row-band
// scale) for a matrix of n columns of kernel kind 0 (RQA), 1 (cross
// recurrence) or 2 (matrix input): the autotuner's choice for the class
// (kind, m, norm, f64, ceil(log2 n)) if it recorded or loaded one, else a
// rule by size.  RQA_TILE_WARPS / RQA_TILE_COLS, then a sweep forced on the
// calling thread (tune_force), override both.  FP64 and matrix input always
// use four columns per lane.
TileConfig choose_tile(int64_t n, int m, int norm, bool f64 = false, int kind = 0);

// The autotuner's table (process-wide, thread-safe; rqa_tune.cpp).
bool tune_lookup(int kind, int m, int norm, bool f64, int64_t n, TileConfig* out);
void tune_record(int kind, int m, int norm, bool f64, int64_t n, const TileConfig& c);
void tune_clear();
// Force a configuration on this thread only (fields <= 0 / band_scale out of
// -1..1 leave the choice alone); tune_force_clear() ends it.
void tune_force(int warps, int cols, int band_scale);
void tune_force_clear();
void tune_apply_forced(TileConfig* c);

// Device bytes a series of length N needs at most, whatever strip width
// runs it (for admission control).
size_t series_device_bytes(const rqa_settings& st, int64_t N);

void measures_from_histograms(const uint64_t* hd, const uint64_t* hv, const uint64_t* hw,
                              int64_t n, int32_t l_min, int32_t v_min, int32_t w_min,
                              rqa_measures_t* out);
// The same for a rows x cols (cross-recurrence) matrix with histograms of
// length hl + 1; RR = RP / (rows * cols).
void measures_from_histograms_rect(const uint64_t* hd, const uint64_t* hv, const uint64_t* hw,
                                   int64_t hl, int64_t rows, int64_t cols, int32_t l_min,
                                   int32_t v_min, int32_t w_min, rqa_measures_t* out);
// The same, reading histogram t only up to last[t] (every bin above it is
// zero, as the device recorded); the result is identical.
void measures_from_histograms_last(const uint64_t* hd, const uint64_t* hv, const uint64_t* hw,
                                   const int64_t last[3], int64_t rows, int64_t cols,
                                   int32_t l_min, int32_t v_min, int32_t w_min,
                                   rqa_measures_t* out);

class Engine {
 public:
  explicit Engine(int device);
  ~Engine();
  Engine(const Engine&) = delete;
  Engine& operator=(const Engine&) = delete;

  // How a run's launch sequence is issued: as plain launches, always through
  // a cached CUDA graph (captured when the plan changes), or through the graph
  // from the second consecutive run with the same plan (single-series calls:
  // a one-off run pays no capture, a repeated one no launch overhead).
  enum GraphMode { kNoGraph = 0, kGraph = 1, kGraphOnRepeat = 2 };

  // Run a set of series on `stream` (nullptr: the engine's own stream).
  // Returns RQA_OK if the set ran (per-series failures are in
  // results[q].status), or an error that affected the whole set.
  int run(const std::vector<SeriesInput>& in, std::vector<SeriesResult>& results,
          cudaStream_t stream, GraphMode mode);

  // Decisions R_ij of series 0 of the last run (needs its buffers alive;
  // RQA_EINVAL after a precomputed-matrix run, which has no decisions).
  int sample(const int64_t* i, const int64_t* j, int64_t count, uint8_t* out);

  const std::string& error() const { return err_; }
  int device() const { return dev_; }
  int sm_count() const { return sms_; }
  float last_tile_ms() const { return tile_ms_; }
  float last_total_ms() const { return total_ms_; }
  // Device arena held between runs, and its release (after the last run on
  // the engine's own stream has completed; the next run allocates again).
  size_t arena_bytes() const { return arena_cap_; }
  void release_arena();

 private:
  int run_impl(const std::vector<SeriesInput>& in, std::vector<SeriesResult>& results,
               cudaStream_t stream, GraphMode mode);
  int ensure_arena(size_t bytes, cudaStream_t st);
  size_t desc_budget() const;
  int ensure_host(size_t bytes);
  void free_arena(cudaStream_t st);
  int fail(int code, const std::string& msg);
  int cuda_fail(cudaError_t e, const char* what);

  int dev_ = 0, sms_ = 0;
  cudaStream_t own_ = nullptr;
  unsigned char* arena_ = nullptr;
  size_t arena_cap_ = 0;
  // the arena comes from this engine's own stream-ordered pool, so growing
  // it does not synchronise the device (other engines' work keeps running)
  cudaMemPool_t pool_ = nullptr;
  unsigned char* host_ = nullptr;  // pinned staging
  size_t host_cap_ = 0;
  cudaEvent_t ev_[4] = {nullptr, nullptr, nullptr, nullptr};
  // side streams: the tile launches of several kernel classes overlap
  static constexpr int kAux = 4;
  cudaStream_t aux_[kAux] = {};
  cudaEvent_t fork_ = nullptr;
  cudaEvent_t order_ = nullptr;  // orders the own stream after the legacy default stream
  cudaEvent_t join_[kAux] = {};
  // per stream group: its tile kernels are done (timing) / its histograms
  // and counters have landed in the pinned staging (waited on by the host)
  cudaEvent_t tiled_[kAux] = {};
  cudaEvent_t done_[kAux] = {};
  std::string err_;
  float tile_ms_ = 0.f, total_ms_ = 0.f;
  // last run, for sample()
  SeriesDesc* last_sd_ = nullptr;
  bool last_f64_ = false;
  bool last_matrix_ = false;
  cudaStream_t last_stream_ = nullptr;
  // graph cache (runs with an unchanged plan); prev_key_: the plan of the
  // last run issued without the graph, for kGraphOnRepeat
  cudaGraphExec_t graph_ = nullptr;
  std::vector<int64_t> graph_key_;
  std::vector<int64_t> prev_key_;
  int graph_launches_ = 0;      // kernel launches and CTAs of the cached graph
  int64_t graph_ctas_ = 0;
};

}  // namespace rqa
