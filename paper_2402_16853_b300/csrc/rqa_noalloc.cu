// rqa_noalloc.cu -- rqa_run_noalloc(): one RQA computation whose scratch
// memory lives in a fixed, file-scope device array instead of memory the
// library allocates.
//
// Some callers cannot let a library allocate device memory: applications
// that hand the whole GPU to their own memory pool, processes in which
// cudaMalloc's implicit device synchronisation would stall other streams at
// an unpredictable moment, and embedded or long-running services that must
// show a fixed device footprint from start-up.  For them this entry point
// runs the same kernels as rqa_run_device() -- prepare, embed, the fused tile
// kernel, the boundary merges and the line-of-identity join -- with every
// intermediate buffer (per-series state, work items, FP32 vectors, boundary
// descriptors, run ends, counters) carved out of g_noalloc_scratch below.
// The caller passes the input series and the output histograms, both in
// device memory.
//
// Costs and limits:
//   * every GPU that loads the library holds the array (RQA_NOALLOC_SCRATCH_BYTES)
//     until the process exits;
//   * series of at most RQA_NOALLOC_MAX_N embedded vectors (larger ones are
//     rejected with RQA_ETOOBIG and a clear message, before any launch);
//   * all calls share the one array, so two calls whose work overlaps on the
//     GPU (different streams, different host threads) race and corrupt each
//     other: serialise them;
//   * the first call on a device looks up the array's device address with
//     cudaGetSymbolAddress, which loads this file's module (and with it the
//     array) if CUDA's lazy loading has not done so yet; rqa_preload_kernels()
//     does the same look-up ahead of time, so that no later call pays for it;
//   * every call blocks until its work on the stream has finished (it reads
//     the status word back), so it must not be issued on a stream that is
//     being captured into a CUDA graph;
//   * only the automatic recheck band (band_override < 0) or rechecking every
//     pair (band_override = +inf) is accepted: with no statistics to return,
//     a call could not report a result made inexact by a narrower band.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/rqa.h"
#include "rqa_internal.h"
#include "rqa_kernels.h"

namespace {

// All scratch of rqa_run_noalloc().  In host code this name is only a
// stand-in for the symbol; the device address comes from
// cudaGetSymbolAddress() (scratch_base below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[RQA_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_base[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// Device address of g_noalloc_scratch on `dev` (the current device),
// looked up once per device.
int scratch_base(int dev, void** out, std::string* msg) {
  if (dev < 0 || dev >= kMaxDevices) {
    *msg = "device ordinal out of range";
    return RQA_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_base[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      *msg = std::string("cudaGetSymbolAddress(g_noalloc_scratch): ") + cudaGetErrorString(e);
      return RQA_ECUDA;
    }
    g_base[dev] = p;
  }
  *out = g_base[dev];
  return RQA_OK;
}

// Writes the per-series state and the work items into the scratch (so no
// host-to-device copy of them is needed).
__global__ void noalloc_setup_kernel(rqa::SeriesDesc* sd, rqa::Item* items, int nitems,
                                     rqa::SeriesDesc init) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *sd = init;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nitems; q += gridDim.x * blockDim.x)
    items[q] = rqa::Item{0, q};
}

// Tile shape for this entry point: a fixed rule of the series length (the
// other entry points may be retuned; this one keeps its scratch bound).
rqa::TileConfig choose_tile_noalloc(int64_t n) {
  rqa::TileConfig c{1, 4};
  if (n >= 16384)
    c.warps = 4;
  else if (n >= 4096)
    c.warps = 2;
  return c;
}

thread_local std::string t_last_error;

int fail(int code, const std::string& msg) {
  t_last_error = msg;
  return code;
}

}  // namespace

namespace rqa {
// Resolves the scratch address on the current device and loads this file's
// kernel, so that the first rqa_run_noalloc() call does no module loading.
// Returns the number of kernels loaded, or -1 on a CUDA error.
int preload_noalloc() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  void* p = nullptr;
  std::string msg;
  if (scratch_base(dev, &p, &msg) != RQA_OK) return -1;
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, reinterpret_cast<const void*>(noalloc_setup_kernel)) !=
      cudaSuccess)
    return -1;
  return 1;
}
}  // namespace rqa

extern "C" const char* rqa_noalloc_last_error(void) { return t_last_error.c_str(); }

extern "C" int rqa_run_noalloc(const rqa_settings* settings, const double* dev_series,
                               int64_t n_points, uint64_t* dev_hist, void* cuda_stream) {
  using namespace rqa;
  t_last_error.clear();
  if (!settings) return fail(RQA_EINVAL, "settings pointer is NULL");
  if (!dev_series || !dev_hist) return fail(RQA_EINVAL, "series or histogram pointer is NULL");
  const rqa_settings& s = *settings;
  if (s.m < 1 || s.tau < 1 || !(s.eps > 0.0) || s.eps != s.eps || s.eps > 1.7e308 ||
      s.norm < 0 || s.norm > 2 || s.theiler < 0 || s.l_min < 1 || s.v_min < 1 || s.w_min < 1 ||
      s.precision < 0 || s.precision > 2 || s.band_override != s.band_override)
    return fail(RQA_EINVAL, "invalid settings");
  if (s.band_override >= 0.0 && s.band_override != __builtin_inf())
    return fail(RQA_EINVAL,
                "rqa_run_noalloc accepts band_override < 0 (automatic band) or +inf only: it "
                "cannot report a result made inexact by a narrower band");
  if (s.m > RQA_MAX_M) return fail(RQA_ETOOBIG, "embedding dimension above RQA_MAX_M");
  const int64_t n = n_points - static_cast<int64_t>(s.m - 1) * s.tau;
  if (n_points < 1 || n < 1) return fail(RQA_ESHORT, "series shorter than the embedding window");
  if (n > RQA_NOALLOC_MAX_N)
    return fail(RQA_ETOOBIG, "rqa_run_noalloc takes at most RQA_NOALLOC_MAX_N (" +
                                 std::to_string(RQA_NOALLOC_MAX_N) + ") embedded vectors, got " +
                                 std::to_string(n));
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(RQA_ECUDA, cudaGetErrorString(e));
  const char* why = nullptr;
  if (check_device_pointer(dev_series, 8, dev, &why) != RQA_OK ||
      check_device_pointer(dev_hist, 8, dev, &why) != RQA_OK)
    return fail(RQA_EINVAL, why);
  void* basep = nullptr;
  std::string msg;
  int rc = scratch_base(dev, &basep, &msg);
  if (rc != RQA_OK) return fail(rc, msg);
  unsigned char* base = static_cast<unsigned char*>(basep);
  int sms = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return fail(RQA_ECUDA, cudaGetErrorString(e));

  // ---- layout inside the scratch
  const bool f64 = s.precision == RQA_PREC_FP64;
  const int mp = f64 ? 0 : ((s.m + 3) / 4) * 4;
  const TileConfig tc = choose_tile_noalloc(n);
  const int64_t sw = 32LL * tc.warps * tc.cols;
  const int64_t nstrips = num_strips(n, sw);
  const int64_t ndesc = strip_offset(n, sw, nstrips);
  size_t off = 0;
  const size_t o_sd = off;
  off += align256(sizeof(SeriesDesc));
  const size_t o_items = off;
  off += align256(sizeof(Item) * static_cast<size_t>(nstrips > 0 ? nstrips : 1));
  const size_t o_zero = off;  // queue counter | status counters | run ends | descriptors
  const size_t o_queue = off;
  off += 256;
  const size_t o_cnt = off;
  off += align256(sizeof(unsigned long long) * CNT_WORDS);
  const size_t o_ends = off;
  off += align256(sizeof(uint32_t) * 2 * static_cast<size_t>(n));
  const size_t dbytes = align256(sizeof(uint16_t) * static_cast<size_t>(ndesc));
  const size_t o_desc = off;
  off += 4 * dbytes;
  const size_t zero_bytes = off - o_zero;
  const size_t o_xe = off;
  off += align256(sizeof(float) * static_cast<size_t>(n) * mp);
  if (off > RQA_NOALLOC_SCRATCH_BYTES)
    return fail(RQA_ETOOBIG, "series needs " + std::to_string(off) +
                                 " scratch bytes, above RQA_NOALLOC_SCRATCH_BYTES");

  SeriesDesc init;
  std::memset(&init, 0, sizeof(init));
  init.s = dev_series;
  init.xe = f64 ? nullptr : reinterpret_cast<float*>(base + o_xe);
  init.N = n_points;
  init.n = n;
  init.m = s.m;
  init.tau = s.tau;
  init.norm = s.norm;
  // a window of n or more removes every cell, as any wider one does; capping
  // it keeps the kernels' index arithmetic (j - w - r0) inside int range
  init.w = static_cast<int32_t>(std::min<int64_t>(s.theiler, n));
  init.mp = mp;
  init.sw = static_cast<int32_t>(sw);
  init.eps = s.eps;
  init.band_override = s.band_override;
  init.hist = reinterpret_cast<unsigned long long*>(dev_hist);
  init.row_a = reinterpret_cast<uint16_t*>(base + o_desc);
  init.row_z = reinterpret_cast<uint16_t*>(base + o_desc + dbytes);
  init.dia_a = reinterpret_cast<uint16_t*>(base + o_desc + 2 * dbytes);
  init.dia_z = reinterpret_cast<uint16_t*>(base + o_desc + 3 * dbytes);
  init.colend = reinterpret_cast<uint32_t*>(base + o_ends);
  init.rowend = init.colend + n;
  init.counters = reinterpret_cast<unsigned long long*>(base + o_cnt);
  desc_set_symmetric(init);
  SeriesDesc* d_sd = reinterpret_cast<SeriesDesc*>(base + o_sd);
  Item* d_items = reinterpret_cast<Item*>(base + o_items);
  int* d_queue = reinterpret_cast<int*>(base + o_queue);

  // ---- the previous call's contents stay in the array: clear what starts at zero
  if ((e = cudaMemsetAsync(base + o_zero, 0, zero_bytes, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(dev_hist, 0, sizeof(uint64_t) * 3 * static_cast<size_t>(n + 1), st)) !=
          cudaSuccess)
    return fail(RQA_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  noalloc_setup_kernel<<<1, 256, 0, st>>>(d_sd, d_items, static_cast<int>(nstrips), init);
  launch_prepare(d_sd, 1, init.N, sms, st);
  if (!f64) launch_embed(d_sd, 1, n * mp, sms, st);
  if (nstrips > 0) {
    TileFn fn = tile_kernel_for(s.m, s.norm, tc.cols, f64, false);
    if (!fn) return fail(RQA_EINVAL, "no tile kernel for this (m, norm)");
    const size_t smem = tile_smem_for(s.m, s.norm, f64, tc.warps, tc.cols);
    if ((e = cudaFuncSetAttribute(reinterpret_cast<const void*>(fn),
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(smem))) != cudaSuccess)
      return fail(RQA_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
             &per_sm, reinterpret_cast<const void*>(fn), 32 * tc.warps, smem)) != cudaSuccess)
      return fail(RQA_ECUDA, std::string("occupancy query: ") + cudaGetErrorString(e));
    int64_t grid = static_cast<int64_t>(per_sm) * sms;
    if (grid > nstrips) grid = nstrips;
    if (grid < 1) grid = 1;
    const SeriesDesc* a_sd = d_sd;
    const Item* a_items = d_items;
    int a_n = static_cast<int>(nstrips);
    int* a_queue = d_queue;
    void* args[] = {&a_sd, &a_items, &a_n, &a_queue};
    if ((e = cudaLaunchKernel(reinterpret_cast<const void*>(fn), dim3(static_cast<unsigned>(grid)),
                              dim3(32 * tc.warps), args, smem, st)) != cudaSuccess)
      return fail(RQA_ECUDA, std::string("tile kernel launch: ") + cudaGetErrorString(e));
  }
  launch_merges(d_sd, 1, n, true, false, false, sms, st);
  if ((e = cudaGetLastError()) != cudaSuccess)
    return fail(RQA_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  unsigned long long status = 0;
  if ((e = cudaMemcpyAsync(&status, init.counters + CNT_STATUS, sizeof(status),
                           cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail(RQA_ECUDA, std::string("synchronise: ") + cudaGetErrorString(e));
  if (status == 3) return fail(RQA_ENAN, "series contains NaN or infinite values");
  if (status == 6) return fail(RQA_ETIMEOUT, "a bounded device-side wait gave up");
  if (status != 0) return fail(RQA_ECUDA, "internal error: a line length outside 1..n");
  return RQA_OK;
}
