// rqa_plot.cpp -- rqa_recurrence_plot(): a window of the recurrence matrix,
// bit-packed, computed on the GPU with the same decisions as rqa_run (the
// paper's RecurrencePlotComputation, Table 2; Sect. 2 describes the plot as
// the visual form of the matrix).  The output is a plain buffer; turning it
// into an image is left to the caller (the Python binding writes PGM).
#include <cuda_runtime.h>

#include <cstring>
#include <string>

#include "../../include/rqa.h"
#include "rqa_engine.h"
#include "rqa_kernels.h"

namespace {
size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }
thread_local std::string t_plot_error;
int plot_fail(int code, const std::string& m) {
  t_plot_error = m;
  return code;
}
}  // namespace

extern "C" const char* rqa_plot_last_error(void) { return t_plot_error.c_str(); }

extern "C" int rqa_recurrence_plot(const rqa_settings* settings, const double* host_series,
                                   int64_t n_points, int64_t i0, int64_t j0, int64_t rows,
                                   int64_t cols, uint32_t* out_bits) {
  using namespace rqa;
  t_plot_error.clear();
  std::string msg;
  int rc = validate_settings(settings, &msg);
  if (rc != RQA_OK) return plot_fail(rc, msg);
  if (!host_series || !out_bits) return plot_fail(RQA_EINVAL, "NULL pointer");
  if (rows < 0 || cols < 0 || i0 < 0 || j0 < 0) return plot_fail(RQA_EINVAL, "negative window");
  const int64_t n = n_points - static_cast<int64_t>(settings->m - 1) * settings->tau;
  if (n_points < 1 || n < 1) return plot_fail(RQA_ESHORT, "series shorter than the embedding");
  if (n > RQA_MAX_N) return plot_fail(RQA_ETOOBIG, "more than RQA_MAX_N embedded vectors");
  const int64_t wpr = (cols + 31) / 32;
  const size_t out_bytes = sizeof(uint32_t) * static_cast<size_t>(rows) * wpr;
  if (out_bytes > (size_t(4) << 30)) return plot_fail(RQA_ETOOBIG, "plot above 4 GiB");
  if (rows == 0 || cols == 0) return RQA_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return plot_fail(RQA_ENODEV, cudaGetErrorString(e));
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const bool f64 = settings->precision == RQA_PREC_FP64;
  const int mp = f64 ? 0 : ((settings->m + 3) / 4) * 4;
  const size_t o_sd = 0;
  const size_t o_cnt = align256(sizeof(SeriesDesc));
  const size_t o_s = o_cnt + 256;
  const size_t o_xe = o_s + align256(sizeof(double) * static_cast<size_t>(n_points));
  const size_t o_out = o_xe + align256(sizeof(float) * static_cast<size_t>(n) * mp);
  const size_t total = o_out + align256(out_bytes);
  unsigned char* base = nullptr;
  if ((e = cudaMalloc(&base, total)) != cudaSuccess) {
    cudaGetLastError();
    return plot_fail(RQA_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  SeriesDesc d;
  std::memset(&d, 0, sizeof(d));
  d.s = reinterpret_cast<const double*>(base + o_s);
  d.xe = f64 ? nullptr : reinterpret_cast<float*>(base + o_xe);
  d.N = n_points;
  d.n = n;
  d.m = settings->m;
  d.tau = settings->tau;
  d.norm = settings->norm;
  d.w = settings->theiler;
  d.mp = mp;
  d.eps = settings->eps;
  d.band_override = settings->band_override;
  d.counters = reinterpret_cast<unsigned long long*>(base + o_cnt);
  SeriesDesc* d_sd = reinterpret_cast<SeriesDesc*>(base + o_sd);
  uint32_t* d_out = reinterpret_cast<uint32_t*>(base + o_out);
  cudaStream_t st = nullptr;
  unsigned long long status = 0;
  rc = RQA_OK;
  if ((e = cudaMemsetAsync(base + o_cnt, 0, 256, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_sd, &d, sizeof(d), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(base + o_s, host_series, sizeof(double) * n_points,
                           cudaMemcpyHostToDevice, st)) != cudaSuccess) {
    rc = plot_fail(RQA_ECUDA, cudaGetErrorString(e));
  } else {
    launch_prepare(d_sd, 1, st);
    if (!f64) launch_embed(d_sd, 1, n * mp, sms, st);
    launch_plot(d_sd, i0, j0, rows, cols, d_out, f64 ? 1 : 0, sms, st);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(out_bits, d_out, out_bytes, cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(&status, d.counters + CNT_STATUS, sizeof(status),
                             cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      rc = plot_fail(RQA_ECUDA, cudaGetErrorString(e));
    else if (status == 3)
      rc = plot_fail(RQA_ENAN, "series contains NaN or infinite values");
  }
  cudaFree(base);
  return rc;
}
