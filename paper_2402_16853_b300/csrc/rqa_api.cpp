// rqa_api.cpp -- the extern "C" entry points of include/rqa.h for single
// series (rqa_*) and batches (rqa_batch_*).  Argument checks and marshalling
// only; all computation is in the engine's CUDA kernels.
#include <cuda_runtime.h>

#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/rqa.h"
#include "rqa_engine.h"
#include "rqa_kernels.h"

struct rqa_handle {
  rqa_settings st{};
  std::unique_ptr<rqa::Engine> eng;
  rqa::SeriesResult res;
  bool have = false;
  std::string err;
};

struct rqa_batch {
  std::unique_ptr<rqa::Engine> eng;
  std::vector<rqa::SeriesResult> res;
  rqa_stats_t stats{};
  std::string err;
};

namespace {

int find_device(int* dev, std::string* msg) {
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || count == 0) {
    cudaGetLastError();
    *msg = std::string("no CUDA device: ") + (e != cudaSuccess ? cudaGetErrorString(e) : "count 0");
    return RQA_ENODEV;
  }
  int cur = 0;
  cudaGetDevice(&cur);
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, cur);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, cur);
  if (major != 10 || minor != 3) {
    *msg = "current CUDA device is compute capability " + std::to_string(major) + "." +
           std::to_string(minor) + "; this library is built for sm_103a (B300)";
    return RQA_ENODEV;
  }
  *dev = cur;
  return RQA_OK;
}

int copy_hist(const rqa::SeriesResult& r, int32_t kind, uint64_t* out, int64_t cap, int64_t* len) {
  if (kind < 0 || kind > 2) return RQA_EINVAL;
  const int64_t need = r.hl + 1;
  if (len) *len = need;
  if (!out || cap < need) return RQA_EINVAL;
  if (!r.hist) return RQA_EINVAL;
  std::memcpy(out, r.hist + kind * need, sizeof(uint64_t) * need);
  return RQA_OK;
}

}  // namespace

extern "C" {

const char* rqa_strerror(int status) {
  switch (status) {
    case RQA_OK: return "ok";
    case RQA_EINVAL: return "invalid argument";
    case RQA_ESHORT: return "series too short for the embedding";
    case RQA_ENAN: return "series contains NaN or infinite values";
    case RQA_ENOMEM: return "out of device memory or over the memory budget";
    case RQA_ECUDA: return "CUDA error";
    case RQA_ETIMEOUT: return "a bounded device-side wait gave up";
    case RQA_PENDING: return "pending";
    case RQA_ENODEV: return "no usable CUDA device (sm_103a)";
    case RQA_ETOOBIG: return "size above the supported maximum";
    case RQA_ENOTFOUND: return "unknown ticket";
    default: return "unknown status";
  }
}

int rqa_create(const rqa_settings* settings, rqa_handle** out) {
  if (!out) return RQA_EINVAL;
  *out = nullptr;
  std::string msg;
  int rc = rqa::validate_settings(settings, &msg);
  if (rc != RQA_OK) return rc;
  int dev = 0;
  rc = find_device(&dev, &msg);
  if (rc != RQA_OK) return rc;
  rqa_handle* h = new (std::nothrow) rqa_handle();
  if (!h) return RQA_ENOMEM;
  h->st = *settings;
  h->eng.reset(new (std::nothrow) rqa::Engine(dev));
  if (!h->eng) {
    delete h;
    return RQA_ENOMEM;
  }
  *out = h;
  return RQA_OK;
}

int rqa_set_settings(rqa_handle* h, const rqa_settings* settings) {
  if (!h) return RQA_EINVAL;
  std::string msg;
  const int rc = rqa::validate_settings(settings, &msg);
  if (rc != RQA_OK) {
    h->err = msg;
    return rc;
  }
  h->st = *settings;
  h->have = false;  // the last result no longer matches the settings
  h->err.clear();
  return RQA_OK;
}

static int run_input(rqa_handle* h, std::vector<rqa::SeriesInput>& in, void* stream) {
  std::vector<rqa::SeriesResult> res;
  int rc = h->eng->run(in, res, static_cast<cudaStream_t>(stream), rqa::Engine::kGraphOnRepeat);
  if (rc != RQA_OK) {
    h->err = h->eng->error();
    return rc;
  }
  h->res = std::move(res[0]);
  h->have = true;
  return RQA_OK;
}

static int run_common(rqa_handle* h, const double* host, const double* dev, int64_t n,
                      void* stream, bool cross = false, const double* host2 = nullptr,
                      const double* dev2 = nullptr, int64_t n2 = 0) {
  if (!h) return RQA_EINVAL;
  h->have = false;
  h->err.clear();
  if ((!host && !dev) || (cross && !host2 && !dev2)) {
    h->err = "series pointer is NULL";
    return RQA_EINVAL;
  }
  std::vector<rqa::SeriesInput> in(1);
  in[0].st = h->st;
  in[0].host = host;
  in[0].dev = dev;
  in[0].N = n;
  in[0].cross = cross;
  in[0].host2 = host2;
  in[0].dev2 = dev2;
  in[0].N2 = n2;
  return run_input(h, in, stream);
}

static int run_matrix(rqa_handle* h, const uint32_t* host_bits, const uint32_t* dev_bits,
                      int64_t rows, int64_t cols, void* stream) {
  if (!h) return RQA_EINVAL;
  h->have = false;
  h->err.clear();
  if (!host_bits && !dev_bits) {
    h->err = "matrix pointer is NULL";
    return RQA_EINVAL;
  }
  std::vector<rqa::SeriesInput> in(1);
  in[0].st = h->st;
  in[0].matrix = true;
  in[0].cross = true;
  in[0].bits_host = host_bits;
  in[0].bits_dev = dev_bits;
  in[0].N = rows;
  in[0].N2 = cols;
  return run_input(h, in, stream);
}

int rqa_run(rqa_handle* h, const double* host_series, int64_t n) {
  return run_common(h, host_series, nullptr, n, nullptr);
}

int rqa_run_device(rqa_handle* h, const double* dev_series, int64_t n, void* cuda_stream) {
  return run_common(h, nullptr, dev_series, n, cuda_stream);
}

int rqa_run_cross(rqa_handle* h, const double* host_x, int64_t n_x, const double* host_y,
                  int64_t n_y) {
  return run_common(h, host_x, nullptr, n_x, nullptr, true, host_y, nullptr, n_y);
}

int rqa_run_cross_device(rqa_handle* h, const double* dev_x, int64_t n_x, const double* dev_y,
                         int64_t n_y, void* cuda_stream) {
  return run_common(h, nullptr, dev_x, n_x, cuda_stream, true, nullptr, dev_y, n_y);
}

int rqa_run_matrix(rqa_handle* h, const uint32_t* host_bits, int64_t rows, int64_t cols) {
  return run_matrix(h, host_bits, nullptr, rows, cols, nullptr);
}

int rqa_run_matrix_device(rqa_handle* h, const uint32_t* dev_bits, int64_t rows, int64_t cols,
                          void* cuda_stream) {
  return run_matrix(h, nullptr, dev_bits, rows, cols, cuda_stream);
}

int rqa_measures(const rqa_handle* h, rqa_measures_t* out) {
  if (!h || !out) return RQA_EINVAL;
  if (!h->have) return RQA_EINVAL;
  *out = h->res.meas;
  return RQA_OK;
}

int rqa_histogram(const rqa_handle* h, int32_t kind, uint64_t* out, int64_t cap, int64_t* len) {
  if (!h || !h->have) return RQA_EINVAL;
  return copy_hist(h->res, kind, out, cap, len);
}

int rqa_stats(const rqa_handle* h, rqa_stats_t* out) {
  if (!h || !out || !h->have) return RQA_EINVAL;
  *out = h->res.stats;
  return RQA_OK;
}

int rqa_sample_decisions(rqa_handle* h, const int64_t* i, const int64_t* j, int64_t count,
                         uint8_t* out) {
  if (!h || !h->have || count < 0 || (count > 0 && (!i || !j || !out))) return RQA_EINVAL;
  int rc = h->eng->sample(i, j, count, out);
  if (rc != RQA_OK) h->err = h->eng->error();
  return rc;
}

void rqa_destroy(rqa_handle* h) { delete h; }

const char* rqa_last_error(const rqa_handle* h) { return h ? h->err.c_str() : "null handle"; }

// ------------------------------------------------------------------ batch
int rqa_batch_create(rqa_batch** out) {
  if (!out) return RQA_EINVAL;
  *out = nullptr;
  std::string msg;
  int dev = 0;
  int rc = find_device(&dev, &msg);
  if (rc != RQA_OK) return rc;
  rqa_batch* b = new (std::nothrow) rqa_batch();
  if (!b) return RQA_ENOMEM;
  b->eng.reset(new (std::nothrow) rqa::Engine(dev));
  if (!b->eng) {
    delete b;
    return RQA_ENOMEM;
  }
  *out = b;
  return RQA_OK;
}

int rqa_preload_kernels(int32_t* loaded) {
  std::string msg;
  int dev = 0;
  const int rc = find_device(&dev, &msg);
  if (rc != RQA_OK) return rc;
  // once per device and process; the lock also keeps two first callers from
  // loading at the same time
  static std::mutex mu;
  static uint64_t done = 0;  // bit d: device d preloaded
  static int32_t count[64] = {};
  std::lock_guard<std::mutex> lk(mu);
  const uint64_t bit = dev < 64 ? (1ull << dev) : 0;
  if (!(done & bit)) {
    const int t = rqa::preload_tile_kernels();
    const int a0 = t < 0 ? -1 : rqa::preload_aux_kernels();
    const int z = a0 < 0 ? -1 : rqa::preload_noalloc();
    const int a = z < 0 ? -1 : a0 + z;
    if (t < 0 || a < 0) {
      cudaGetLastError();
      return RQA_ECUDA;
    }
    if (bit) {
      done |= bit;
      count[dev] = t + a;
    }
    if (loaded) *loaded = t + a;
    return RQA_OK;
  }
  if (loaded) *loaded = count[dev];
  return RQA_OK;
}

int rqa_selftest_ring_timeout(rqa_handle* h, const double* host_series, int64_t n_points,
                              int32_t warp, int32_t from_handover) {
  if (!h || !host_series) return RQA_EINVAL;
  if (h->st.m != 3 || h->st.norm != RQA_NORM_L2 || h->st.precision == RQA_PREC_FP64) {
    h->err = "the ring-timeout self-test runs m = 3, L2, FP32 distances";
    return RQA_EINVAL;
  }
  if (warp < 0 || warp > 6 || from_handover < 1) {
    h->err = "warp must be 0..6 (it needs a right neighbour's consumer) and the hand-over >= 1";
    return RQA_EINVAL;
  }
  h->have = false;
  h->err.clear();
  std::vector<rqa::SeriesInput> in(1);
  in[0].st = h->st;
  in[0].host = host_series;
  in[0].N = n_points;
  in[0].withhold_warp = warp + 1;
  in[0].withhold_seq = from_handover;
  rqa::tune_force(8, 4, 0);  // eight warps per strip, so the warp has a consumer
  std::vector<rqa::SeriesResult> res;
  const int rc = h->eng->run(in, res, nullptr, rqa::Engine::kNoGraph);
  rqa::tune_force_clear();
  if (rc != RQA_OK) {
    h->err = h->eng->error();
    return rc;
  }
  h->res = std::move(res[0]);  // the withheld hand-over was never reached
  h->have = true;
  return RQA_OK;
}

int rqa_selftest_bounded_wait(int32_t* status, int64_t* cycles_waited) {
  std::string msg;
  int dev = 0;
  int rc = find_device(&dev, &msg);
  if (rc != RQA_OK) return rc;
  unsigned long long* d = nullptr;
  unsigned long long h[3] = {0, 0, 0};
  cudaError_t e = cudaMalloc(&d, sizeof(h));
  if (e != cudaSuccess) return RQA_ENOMEM;
  rc = RQA_OK;
  if ((e = cudaMemset(d, 0, sizeof(h))) != cudaSuccess) {
    rc = RQA_ECUDA;
  } else {
    rqa::launch_wait_selftest(d, nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost)) != cudaSuccess)
      rc = RQA_ECUDA;
  }
  cudaFree(d);
  if (rc != RQA_OK) return rc;
  if (status) *status = static_cast<int32_t>(h[0]);
  if (cycles_waited) *cycles_waited = static_cast<int64_t>(h[1]);
  return h[2] == 1 ? RQA_OK : RQA_ECUDA;  // the abort flag must be raised
}

namespace {
int batch_run_on(rqa_batch* b, const rqa_settings* settings, const double* const* series,
                 const int64_t* lens, int32_t count, rqa_measures_t* out, int32_t* status,
                 cudaStream_t stream) {
  if (!b || count < 0 || (count > 0 && (!settings || !series || !lens))) return RQA_EINVAL;
  std::vector<rqa::SeriesInput> in(count);
  for (int32_t q = 0; q < count; ++q) {
    in[q].st = settings[q];
    in[q].host = series[q];
    in[q].N = lens[q];
  }
  int rc = b->eng->run(in, b->res, stream, rqa::Engine::kGraph);
  b->err = b->eng->error();
  b->stats = rqa_stats_t{};
  for (int32_t q = 0; q < count && q < static_cast<int32_t>(b->res.size()); ++q) {
    if (status) status[q] = b->res[q].status;
    if (out) {
      if (b->res[q].status == RQA_OK)
        out[q] = b->res[q].meas;
      else
        std::memset(&out[q], 0, sizeof(rqa_measures_t));
    }
    b->stats.n_vec += b->res[q].n;
    b->stats.pairs += b->res[q].stats.pairs;
    b->stats.rechecks += b->res[q].stats.rechecks;
  }
  if (!b->res.empty()) {
    b->stats.h2d_bytes = b->res[0].stats.h2d_bytes;
    b->stats.d2h_bytes = b->res[0].stats.d2h_bytes;
    b->stats.launches = b->res[0].stats.launches;
    b->stats.ctas = b->res[0].stats.ctas;
  }
  b->stats.kernel_ms = b->eng->last_tile_ms();
  b->stats.total_ms = b->eng->last_total_ms();
  return rc;
}

// The batch object behind rqa_run_batch: one per host thread and device,
// kept for reuse (its buffers and captured graph) until rqa_run_batch_release.
thread_local rqa_batch* t_run_batch = nullptr;
thread_local int t_run_batch_dev = -1;
}  // namespace

int rqa_batch_run(rqa_batch* b, const rqa_settings* settings, const double* const* series,
                  const int64_t* lens, int32_t count, rqa_measures_t* out, int32_t* status) {
  return batch_run_on(b, settings, series, lens, count, out, status, nullptr);
}

int rqa_run_batch(const rqa_settings* settings, const double* const* series, const int64_t* lens,
                  int32_t count, rqa_measures_t* out, void* stream) {
  if (count < 0 || (count > 0 && (!settings || !series || !lens || !out))) return RQA_EINVAL;
  std::string msg;
  int dev = 0;
  int rc = find_device(&dev, &msg);
  if (rc != RQA_OK) return rc;
  if (t_run_batch && t_run_batch_dev != dev) rqa_run_batch_release();
  if (!t_run_batch) {
    rc = rqa_batch_create(&t_run_batch);
    if (rc != RQA_OK) return rc;
    t_run_batch_dev = dev;
  }
  return batch_run_on(t_run_batch, settings, series, lens, count, out, nullptr,
                      static_cast<cudaStream_t>(stream));
}

void rqa_run_batch_release(void) {
  if (t_run_batch) rqa_batch_destroy(t_run_batch);
  t_run_batch = nullptr;
  t_run_batch_dev = -1;
}

int rqa_batch_histogram(const rqa_batch* b, int32_t q, int32_t kind, uint64_t* out, int64_t cap,
                        int64_t* len) {
  if (!b || q < 0 || q >= static_cast<int32_t>(b->res.size())) return RQA_EINVAL;
  if (b->res[q].status != RQA_OK) return b->res[q].status;
  return copy_hist(b->res[q], kind, out, cap, len);
}

int rqa_batch_stats(const rqa_batch* b, rqa_stats_t* out) {
  if (!b || !out) return RQA_EINVAL;
  *out = b->stats;
  return RQA_OK;
}

void rqa_batch_destroy(rqa_batch* b) { delete b; }

}  // extern "C"
