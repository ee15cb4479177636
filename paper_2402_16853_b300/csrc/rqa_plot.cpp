// rqa_plot.cpp -- rqa_recurrence_plot() and rqa_cross_recurrence_plot(): a
// window of the recurrence (or cross-recurrence) matrix,
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

namespace {

// One plot window.  host_y == nullptr: the RQA matrix of host_x; otherwise
// the cross-recurrence matrix, rows from host_x and columns from host_y.
int plot_common(const rqa_settings* settings, const double* host_x, int64_t nx,
                const double* host_y, int64_t ny, int64_t i0, int64_t j0, int64_t rows,
                int64_t cols, uint32_t* out_bits) {
  using namespace rqa;
  t_plot_error.clear();
  std::string msg;
  int rc = validate_settings(settings, &msg);
  if (rc != RQA_OK) return plot_fail(rc, msg);
  const bool cross = host_y != nullptr;
  if (!host_x || !out_bits) return plot_fail(RQA_EINVAL, "NULL pointer");
  if (rows < 0 || cols < 0 || i0 < 0 || j0 < 0) return plot_fail(RQA_EINVAL, "negative window");
  const int64_t span = static_cast<int64_t>(settings->m - 1) * settings->tau;
  const int64_t n = nx - span;
  const int64_t n2 = cross ? ny - span : n;
  if (nx < 1 || n < 1 || (cross && (ny < 1 || n2 < 1)))
    return plot_fail(RQA_ESHORT, "series shorter than the embedding");
  if (n > RQA_MAX_N || n2 > RQA_MAX_N)
    return plot_fail(RQA_ETOOBIG, "more than RQA_MAX_N embedded vectors");
  // window origin far beyond any matrix, or a plot above 4 GiB (tested by
  // division, so that no product can wrap)
  if (i0 > (int64_t(1) << 40) || j0 > (int64_t(1) << 40))
    return plot_fail(RQA_EINVAL, "window origin beyond 2^40");
  const int64_t wpr = cols / 32 + (cols % 32 != 0);
  if (wpr > 0 && rows > (int64_t(1) << 30) / wpr) return plot_fail(RQA_ETOOBIG, "plot above 4 GiB");
  const size_t out_bytes = sizeof(uint32_t) * static_cast<size_t>(rows) * static_cast<size_t>(wpr);
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
  const size_t o_s2 = o_s + align256(sizeof(double) * static_cast<size_t>(nx));
  const size_t o_xe = o_s2 + (cross ? align256(sizeof(double) * static_cast<size_t>(ny)) : 0);
  const size_t o_xe2 = o_xe + align256(sizeof(float) * static_cast<size_t>(n) * mp);
  const size_t o_out = o_xe2 + (cross ? align256(sizeof(float) * static_cast<size_t>(n2) * mp) : 0);
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
  d.N = nx;
  d.n = n;
  d.m = settings->m;
  d.tau = settings->tau;
  d.norm = settings->norm;
  d.w = settings->theiler;
  d.mp = mp;
  d.eps = settings->eps;
  d.band_override = settings->band_override;
  d.counters = reinterpret_cast<unsigned long long*>(base + o_cnt);
  desc_set_symmetric(d);
  if (cross) {
    d.s2 = reinterpret_cast<const double*>(base + o_s2);
    d.xe2 = f64 ? nullptr : reinterpret_cast<float*>(base + o_xe2);
    d.N2 = ny;
    d.n2 = n2;
    d.hl = n > n2 ? n : n2;
    d.cross = 1;
  }
  SeriesDesc* d_sd = reinterpret_cast<SeriesDesc*>(base + o_sd);
  uint32_t* d_out = reinterpret_cast<uint32_t*>(base + o_out);
  cudaStream_t st = nullptr;
  unsigned long long status = 0;
  rc = RQA_OK;
  if ((e = cudaMemsetAsync(base + o_cnt, 0, 256, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_sd, &d, sizeof(d), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(base + o_s, host_x, sizeof(double) * nx, cudaMemcpyHostToDevice,
                           st)) != cudaSuccess ||
      (cross && (e = cudaMemcpyAsync(base + o_s2, host_y, sizeof(double) * ny,
                                     cudaMemcpyHostToDevice, st)) != cudaSuccess)) {
    rc = plot_fail(RQA_ECUDA, cudaGetErrorString(e));
  } else {
    launch_prepare(d_sd, 1, nx + (cross ? ny : 0), sms, st);
    if (!f64) launch_embed(d_sd, 1, (n + (cross ? n2 : 0)) * mp, sms, st);
    launch_plot(d_sd, i0, j0, rows, cols, d_out, f64 ? 1 : 0, settings->m, settings->norm, sms,
                st);
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

}  // namespace

extern "C" int rqa_recurrence_plot(const rqa_settings* settings, const double* host_series,
                                   int64_t n_points, int64_t i0, int64_t j0, int64_t rows,
                                   int64_t cols, uint32_t* out_bits) {
  return plot_common(settings, host_series, n_points, nullptr, 0, i0, j0, rows, cols, out_bits);
}

extern "C" int rqa_cross_recurrence_plot(const rqa_settings* settings, const double* host_x,
                                         int64_t nx, const double* host_y, int64_t ny,
                                         int64_t i0, int64_t j0, int64_t rows, int64_t cols,
                                         uint32_t* out_bits) {
  if (!host_y) return plot_fail(RQA_EINVAL, "NULL pointer");
  return plot_common(settings, host_x, nx, host_y, ny, i0, j0, rows, cols, out_bits);
}
