// rqa_engine.cpp -- plans, launches and reads back one set of series.
#include "rqa_engine.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <thread>
#include <tuple>

#include "rqa_kernels.h"

namespace rqa {

namespace {

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// f(q) for q in [0, count) on up to 16 host threads, at least `per_thread`
// items each (serially when that leaves one thread).
template <class F>
void parallel_for(int count, int per_thread, F&& f) {
  const int hw = static_cast<int>(std::thread::hardware_concurrency());
  const int T = std::min({16, std::max(hw, 1), count / std::max(per_thread, 1)});
  if (T <= 1) {
    for (int q = 0; q < count; ++q) f(q);
    return;
  }
  std::atomic<int> next{0};
  std::vector<std::thread> th;
  th.reserve(T);
  for (int t = 0; t < T; ++t)
    th.emplace_back([&] {
      for (int q; (q = next.fetch_add(1)) < count;) f(q);
    });
  for (auto& x : th) x.join();
}

// RQA_TRACE=1: one line per run on stderr with the host phases of the run
// (plan, staging, enqueue, the device run with the measures computed as each
// stream group's results land, the finish) and the device times, for finding
// where a call spends its time.
bool trace_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("RQA_TRACE");
    return e && *e && *e != '0';
  }();
  return on;
}

struct HostCopy {
  void* dst;
  const void* src;
  size_t bytes;
};

int64_t nvec_of(const rqa_settings& st, int64_t N) {
  return N - static_cast<int64_t>(st.m - 1) * st.tau;
}

// Unique off-window pairs i < j with j - i >= max(w, 1).
int64_t pair_count(int64_t n, int w) {
  const int64_t k0 = w < 1 ? 1 : w;
  if (k0 > n - 1) return 0;
  const int64_t cnt = n - k0;  // diagonals k0 .. n-1, lengths n-k0 .. 1
  return cnt * (cnt + 1) / 2;
}

// Cells of the n1 x n2 cross matrix outside the Theiler window |i - j| < w.
int64_t cross_cell_count(int64_t n1, int64_t n2, int64_t w) {
  int64_t cells = n1 * n2;
  for (int64_t k = -(w - 1); k <= w - 1; ++k) {  // diagonal k: cells (i, i + k)
    const int64_t lo = k < 0 ? -k : 0;
    const int64_t hi = std::min(n1, n2 - k);
    if (hi > lo) cells -= hi - lo;
  }
  return cells;
}

struct Sizes {
  int64_t n = 0, n2 = 0, hl = 0, nstrips = 0, ndesc = 0, nrowdesc = 0, wpr = 0;
  int64_t nitems = 0;          // work items: strips, or (strip, band) pairs
  int64_t band_h = 0, nbands = 1;
  // strip groups (a single RQA series whose descriptors would exceed the
  // budget): gstrips strips per group, descriptors sized for one group
  int64_t gstrips = 0, ngroups = 1;
  size_t carry = 0;   // rcarry + dcarry
  size_t desc_full = 0;  // descriptor bytes of all strips at once
  int mp = 0;
  TileConfig tc{1, 4};
  bool f64 = false, cross = false, matrix = false;
  size_t hist = 0, ends = 0, cnt = 0, desc = 0, series = 0, series2 = 0, xe = 0, xe2 = 0;
  size_t tab = 0, cols = 0;    // banded: item offset table, column descriptors
};

// Row-band height: RQA_BAND_ROWS if set (rounded up to a multiple of 32; for
// tests and tuning), else bands only when the strips alone give fewer than
// 7,104 warps (two per resident warp slot of the 80-register kernel on 148
// SMs) -- about 2,048 items of at least 128 rows.  `rows` is the number of
// rows summed over the strips.
int64_t band_rows_for(int64_t n, int64_t rows, int64_t nstrips, int warps, int band_scale) {
  if (const char* e = std::getenv("RQA_BAND_ROWS")) {
    const int64_t h = std::atoll(e);
    return h > 0 ? (h + 31) / 32 * 32 : 0;
  }
  if (n < 512 || nstrips * warps >= 7104) return 0;
  int64_t h = (rows + 2047) / 2048;
  h = std::max<int64_t>(128, (h + 31) / 32 * 32);
  // the autotuner may halve or double the rule's height (never below 64 rows)
  if (band_scale < 0) h = std::max<int64_t>(64, (h / 2 + 31) / 32 * 32);
  if (band_scale > 0) h *= 2;
  return h;
}

// Visit the items (Q, g) of a banded series with the rows they hold and the
// number of diagonals k that can cross them: RQA strips hold the rows above
// the line of identity, cross-recurrence and matrix strips all n rows.
template <class F>
void for_each_band_item(const Sizes& z, F&& f) {
  const int64_t sw = 32LL * z.tc.warps * z.tc.cols;
  for (int64_t Q = 0; Q < z.nstrips; ++Q) {
    const int64_t J1 = (z.cross ? z.n2 : z.n) - Q * sw;
    for (int64_t g = 0; g < z.nbands; ++g) {
      const int64_t R0 = g * z.band_h;
      const int64_t R1 = std::min(R0 + z.band_h, z.n);
      if (z.cross) {
        f(Q, g, R1 - R0, sw + (R1 - R0) - 1);
        continue;
      }
      if (R0 > J1 - 2) break;  // no row of the upper triangle in this band
      const int64_t klo = band_klo(J1, sw, R1), khi = J1 - 1 - R0;
      f(Q, g, std::min(R1, J1 - 1) - R0, khi - klo + 1);
    }
  }
}

// Device buffers of one series (RQA), one pair of series (cross
// recurrence: rows from the N values, columns from the N2 values) or one
// precomputed N x N2 bit matrix (its copy counted in `series`).
Sizes sizes_for(const rqa_settings& st, int64_t N, bool copy_series, bool cross = false,
                int64_t N2 = 0, bool copy_series2 = false, bool matrix = false,
                int warps = 0, bool allow_bands = false, int cols = 0, size_t desc_budget = 0) {
  Sizes z;
  z.matrix = matrix;
  z.n = matrix ? N : nvec_of(st, N);
  z.cross = cross || matrix;
  z.n2 = matrix ? N2 : cross ? nvec_of(st, N2) : z.n;
  z.hl = std::max(z.n, z.n2);
  z.f64 = !matrix && st.precision == RQA_PREC_FP64;
  z.mp = (z.f64 || matrix) ? 0 : ((st.m + 3) / 4) * 4;
  z.tc = choose_tile(z.n2, st.m, st.norm, z.f64, matrix ? 2 : cross ? 1 : 0);
  if (warps > 0) z.tc.warps = warps;
  if (cols > 0) z.tc.cols = cols;
  // two columns per lane exist for the FP32 distance kernels only
  if (z.f64 || matrix) z.tc.cols = 4;
  const int64_t sw = 32LL * z.tc.warps * z.tc.cols;
  if (z.cross) {
    z.nstrips = cross_num_strips(z.n2, sw);
    z.ndesc = z.nstrips * cross_strip_diags(z.n, sw);
  } else {
    z.nstrips = num_strips(z.n, sw);
    z.ndesc = strip_offset(z.n, sw, z.nstrips);
    z.nrowdesc = z.ndesc;  // rows: strip-triangular, banded or not
  }
  {
    const int64_t rows = z.cross ? z.n * z.nstrips : z.nrowdesc;  // rows over all strips
    const int64_t h =
        allow_bands ? band_rows_for(z.n, rows, z.nstrips, z.tc.warps, z.tc.band_scale) : 0;
    if (h > 0 && h < z.n) {
      z.band_h = h;
      z.nbands = (z.n + h - 1) / h;
      z.ndesc = 0;
      for_each_band_item(z, [&](int64_t, int64_t, int64_t, int64_t cnt) {
        z.ndesc += cnt;
        ++z.nitems;
      });
      z.tab = align256(sizeof(int64_t) * static_cast<size_t>(z.nstrips * z.nbands));
      z.cols = 2 * align256(sizeof(uint32_t) * static_cast<size_t>(z.nbands * z.n2));
    }
  }
  if (z.nitems == 0) z.nitems = z.nstrips;
  z.hist = align256(sizeof(uint64_t) * 3 * static_cast<size_t>(z.hl + 1));
  z.ends = z.cross ? 0 : align256(sizeof(uint32_t) * 2 * static_cast<size_t>(z.n));
  z.cnt = align256(sizeof(uint64_t) * CNT_WORDS);
  // RQA: row_a, row_z, dia_a, dia_z; cross recurrence and matrices: dia_a, dia_z
  z.desc = 2 * align256(sizeof(uint16_t) * static_cast<size_t>(z.ndesc)) +
           2 * align256(sizeof(uint16_t) * static_cast<size_t>(z.nrowdesc));
  z.desc_full = z.desc;
  if (desc_budget > 0 && !z.cross && z.nbands <= 1 && z.desc > desc_budget && z.nstrips > 1) {
    // Divide & Recombine with bounded memory (Sect. 4.1's carryover buffers):
    // the most strips per group whose descriptors fit the budget (the first
    // group, of the tallest strips, is the largest)
    const int64_t sw = 32LL * z.tc.warps * z.tc.cols;
    int64_t lo = 1, hi = z.nstrips;  // the largest g with 8 bytes per descriptor in budget
    while (lo < hi) {
      const int64_t mid = lo + (hi - lo + 1) / 2;
      if (static_cast<size_t>(strip_offset(z.n, sw, mid)) * 8 <= desc_budget)
        lo = mid;
      else
        hi = mid - 1;
    }
    const int64_t g = lo;
    z.gstrips = g;
    z.ngroups = (z.nstrips + g - 1) / g;
    z.ndesc = z.nrowdesc = strip_offset(z.n, sw, g);
    z.desc = 4 * align256(sizeof(uint16_t) * static_cast<size_t>(z.ndesc));
    z.carry = 2 * align256(sizeof(uint32_t) * static_cast<size_t>(z.n));
  }
  if (matrix) {
    z.wpr = (z.n2 + 31) / 32;
    z.series = copy_series ? align256(sizeof(uint32_t) * static_cast<size_t>(z.n * z.wpr)) : 0;
    return z;
  }
  z.series = copy_series ? align256(sizeof(double) * static_cast<size_t>(N)) : 0;
  z.series2 = cross && copy_series2 ? align256(sizeof(double) * static_cast<size_t>(N2)) : 0;
  z.xe = align256(sizeof(float) * static_cast<size_t>(z.n) * z.mp);
  z.xe2 = cross ? align256(sizeof(float) * static_cast<size_t>(z.n2) * z.mp) : 0;
  return z;
}

// Validation of one input beyond its settings: pointers, lengths, limits.
int validate_input(const SeriesInput& in, std::string* msg) {
  int s = validate_settings(&in.st, msg);
  if (s != RQA_OK) return s;
  if (in.matrix) {  // a precomputed matrix: N rows, N2 columns
    if (!in.bits_host && !in.bits_dev) {
      *msg = "matrix pointer is NULL";
      return RQA_EINVAL;
    }
    if (in.N < 1 || in.N2 < 1) {
      *msg = "matrix has no rows or no columns";
      return RQA_ESHORT;
    }
    if (in.N > RQA_MAX_N_RECT || in.N2 > RQA_MAX_N_RECT) {
      *msg = "more than RQA_MAX_N_RECT rows or columns";
      return RQA_ETOOBIG;
    }
    return RQA_OK;
  }
  if (!in.host && !in.dev) {
    *msg = "series pointer is NULL";
    return RQA_EINVAL;
  }
  if (in.N < 1) {
    *msg = "series is empty";
    return RQA_ESHORT;
  }
  if (nvec_of(in.st, in.N) < 1) {
    *msg = "series shorter than the embedding window (m-1)*tau + 1";
    return RQA_ESHORT;
  }
  if (nvec_of(in.st, in.N) > RQA_MAX_N) {
    *msg = "more than RQA_MAX_N embedded vectors";
    return RQA_ETOOBIG;
  }
  if (in.cross && nvec_of(in.st, in.N) > RQA_MAX_N_RECT) {
    *msg = "more than RQA_MAX_N_RECT embedded vectors in the first series";
    return RQA_ETOOBIG;
  }
  if (in.cross) {
    if (!in.host2 && !in.dev2) {
      *msg = "second series pointer is NULL";
      return RQA_EINVAL;
    }
    if (in.N2 < 1 || nvec_of(in.st, in.N2) < 1) {
      *msg = "second series shorter than the embedding window (m-1)*tau + 1";
      return RQA_ESHORT;
    }
    if (nvec_of(in.st, in.N2) > RQA_MAX_N_RECT) {
      *msg = "more than RQA_MAX_N_RECT embedded vectors in the second series";
      return RQA_ETOOBIG;
    }
  }
  return RQA_OK;
}

// Kernel classes onto side streams: longest work first, each class to the
// least loaded of `nside` streams (-1: the main stream, when nside is 0).
void assign_streams(const std::vector<double>& work, int nside, std::vector<int>& order,
                    std::vector<int>& stream_of) {
  const int ncls = static_cast<int>(work.size());
  order.resize(ncls);
  stream_of.assign(ncls, -1);
  for (int c = 0; c < ncls; ++c) order[c] = c;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
  if (nside == 0) return;
  std::vector<double> load(nside, 0.0);
  for (int c : order) {
    int best = 0;
    for (int k = 1; k < nside; ++k)
      if (load[k] < load[best]) best = k;
    stream_of[c] = best;
    load[best] += work[c];
  }
}

}  // namespace

int check_device_pointer(const void* p, size_t align, int device, const char** what_failed) {
  if (reinterpret_cast<uintptr_t>(p) % align != 0) {
    *what_failed = align == 8 ? "device pointer is not 8-byte aligned"
                              : "device pointer is not 4-byte aligned";
    return RQA_EINVAL;
  }
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    *what_failed = "not a pointer CUDA knows";
    return RQA_EINVAL;
  }
  const bool ok = (a.type == cudaMemoryTypeDevice && a.device == device) ||
                  a.type == cudaMemoryTypeManaged ||
                  (a.type == cudaMemoryTypeHost && a.devicePointer == p);
  if (!ok) {
    *what_failed = a.type == cudaMemoryTypeDevice
                       ? "device pointer belongs to another device"
                       : "host memory the device cannot read (pass it to the host entry point)";
    return RQA_EINVAL;
  }
  return RQA_OK;
}


int validate_settings(const rqa_settings* st, std::string* msg) {
  if (!st) {
    *msg = "settings pointer is NULL";
    return RQA_EINVAL;
  }
  if (st->m < 1) {
    *msg = "embedding dimension m must be >= 1";
    return RQA_EINVAL;
  }
  if (st->m > RQA_MAX_M) {
    *msg = "embedding dimension m is above RQA_MAX_M (10)";
    return RQA_ETOOBIG;
  }
  if (st->tau < 1) {
    *msg = "time delay tau must be >= 1";
    return RQA_EINVAL;
  }
  if (!std::isfinite(st->eps) || !(st->eps > 0.0)) {
    *msg = "radius eps must be finite and > 0";
    return RQA_EINVAL;
  }
  if (st->norm < 0 || st->norm > 2) {
    *msg = "norm must be RQA_NORM_MAX, RQA_NORM_L2 or RQA_NORM_L1";
    return RQA_EINVAL;
  }
  if (st->theiler < 0) {
    *msg = "Theiler window must be >= 0";
    return RQA_EINVAL;
  }
  if (st->l_min < 1 || st->v_min < 1 || st->w_min < 1) {
    *msg = "minimum line lengths must be >= 1";
    return RQA_EINVAL;
  }
  if (st->precision < 0 || st->precision > 2) {
    *msg = "precision must be RQA_PREC_AUTO, RQA_PREC_FP32_RECHECK or RQA_PREC_FP64";
    return RQA_EINVAL;
  }
  if (std::isnan(st->band_override)) {
    *msg = "band_override is NaN";
    return RQA_EINVAL;
  }
  return RQA_OK;
}

TileConfig choose_tile(int64_t n, int m, int norm, bool f64, int kind) {
  TileConfig c{1, 4, 0};
  if (n >= 65536)
    c.warps = 8;
  else if (n >= 16384)
    c.warps = 4;
  else if (n >= 4096)
    c.warps = 2;
  TileConfig t{};
  if (tune_lookup(kind, m, norm, f64, n, &t)) c = t;
  if (const char* e = std::getenv("RQA_TILE_WARPS")) {
    const int w = std::atoi(e);
    if (w >= 1 && w <= 8) c.warps = w;
  }
  if (const char* e = std::getenv("RQA_TILE_COLS")) {
    const int k = std::atoi(e);
    if (k == 2 || k == 4) c.cols = k;
  }
  tune_apply_forced(&c);
  if (f64 || kind == 2) c.cols = 4;  // two columns per lane: FP32 distances only
  return c;
}

size_t series_device_bytes(const rqa_settings& st, int64_t N) {
  // the narrowest strips (one warp) need the most descriptors: a run that
  // batches this series with others, or an autotuned width, never needs more;
  // row bands add item tables and column descriptors
  size_t worst = 0;
  for (const bool bands : {false, true}) {
    const Sizes z = sizes_for(st, N, true, false, 0, false, false, 1, bands, 2);
    worst = std::max(worst, z.hist + z.ends + z.cnt + z.desc + z.series + z.xe + z.tab +
                                z.cols + align256(sizeof(SeriesDesc)) +
                                align256(sizeof(Item) * static_cast<size_t>(z.nitems)) + 256);
  }
  return worst;
}

Engine::Engine(int device) : dev_(device) {
  cudaSetDevice(dev_);
  cudaDeviceGetAttribute(&sms_, cudaDevAttrMultiProcessorCount, dev_);
  cudaStreamCreateWithFlags(&own_, cudaStreamNonBlocking);
  for (auto& e : ev_) cudaEventCreate(&e);
  for (auto& a : aux_) cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking);
  cudaEventCreateWithFlags(&fork_, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&order_, cudaEventDisableTiming);
  for (auto& j : join_) cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
  for (auto& t : tiled_) cudaEventCreate(&t);
  for (auto& d : done_) cudaEventCreateWithFlags(&d, cudaEventDisableTiming);
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev_;
  if (cudaMemPoolCreate(&pool_, &props) != cudaSuccess) {  // plain cudaMalloc then
    cudaGetLastError();
    pool_ = nullptr;
  }
}

Engine::~Engine() {
  cudaSetDevice(dev_);
  if (graph_) cudaGraphExecDestroy(graph_);
  for (auto& e : ev_)
    if (e) cudaEventDestroy(e);
  for (auto& j : join_)
    if (j) cudaEventDestroy(j);
  for (auto& t : tiled_)
    if (t) cudaEventDestroy(t);
  for (auto& d : done_)
    if (d) cudaEventDestroy(d);
  if (fork_) cudaEventDestroy(fork_);
  if (order_) cudaEventDestroy(order_);
  free_arena(own_);  // every run ended with its stream idle
  cudaStreamSynchronize(own_);
  if (pool_) cudaMemPoolDestroy(pool_);
  for (auto& a : aux_)
    if (a) cudaStreamDestroy(a);
  if (own_) cudaStreamDestroy(own_);
  if (host_) cudaFreeHost(host_);
}

int Engine::fail(int code, const std::string& msg) {
  err_ = msg;
  return code;
}

int Engine::cuda_fail(cudaError_t e, const char* what) {
  err_ = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return e == cudaErrorMemoryAllocation ? RQA_ENOMEM : RQA_ECUDA;
}

void Engine::release_arena() {
  cudaSetDevice(dev_);
  if (graph_) {  // the captured graph points into the arena
    cudaGraphExecDestroy(graph_);
    graph_ = nullptr;
    graph_key_.clear();
  }
  free_arena(own_);
  cudaStreamSynchronize(own_);
}

void Engine::free_arena(cudaStream_t st) {
  if (!arena_) return;
  if (pool_)
    cudaFreeAsync(arena_, st);
  else
    cudaFree(arena_);
  arena_ = nullptr;
  arena_cap_ = 0;
}

// Grow the arena to at least `bytes` (by half again, so growth stays rare).
// From the pool, the old block is released and the new one taken in the
// order of `st`, which every previous run of this engine has completed on.
// Boundary-descriptor budget of a single RQA series, above which its strips
// run in groups: RQA_DESC_BUDGET bytes if set, else a fifth of the device's
// memory (55 GB on a B300: the 1,048,576-point series, 4.3 GB, runs in one
// group; 2^22 vectors, 69 GB, in three).
size_t Engine::desc_budget() const {
  if (const char* e = std::getenv("RQA_DESC_BUDGET")) {
    const long long b = std::atoll(e);
    if (b > 0) return static_cast<size_t>(b);
  }
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return size_t(16) << 30;
  }
  return tot / 5;
}

int Engine::ensure_arena(size_t bytes, cudaStream_t st) {
  if (bytes <= arena_cap_) return RQA_OK;
  if (graph_) {
    cudaGraphExecDestroy(graph_);
    graph_ = nullptr;
    graph_key_.clear();
  }
  free_arena(st);
  // room to grow by half again, at most 1 GiB more (large series run in
  // strip groups whose arena is sized by the descriptor budget)
  const size_t cap = bytes + std::min<size_t>(bytes / 2, size_t(1) << 30);
  void* p = nullptr;
  cudaError_t e = pool_ ? cudaMallocFromPoolAsync(&p, cap, pool_, st) : cudaMalloc(&p, cap);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "device arena allocation");
  }
  arena_ = static_cast<unsigned char*>(p);
  arena_cap_ = cap;
  return RQA_OK;
}

int Engine::ensure_host(size_t bytes) {
  if (bytes <= host_cap_) return RQA_OK;
  if (graph_) {
    cudaGraphExecDestroy(graph_);
    graph_ = nullptr;
    graph_key_.clear();
  }
  if (host_) {
    cudaFreeHost(host_);
    host_ = nullptr;
    host_cap_ = 0;
  }
  const size_t cap = bytes + bytes / 2;
  cudaError_t e = cudaMallocHost(&host_, cap);
  if (e != cudaSuccess) {
    cudaGetLastError();
    host_ = nullptr;
    return cuda_fail(e, "cudaMallocHost(staging)");
  }
  host_cap_ = cap;
  return RQA_OK;
}

int Engine::run(const std::vector<SeriesInput>& in, std::vector<SeriesResult>& results,
                cudaStream_t stream, GraphMode mode) {
  const int rc = run_impl(in, results, stream, mode);
  if (rc != RQA_OK) {
    // a failure of the whole set marks every unfinished series
    for (auto& r : results)
      if (r.status == RQA_OK && !r.hist) r.status = rc;
    // nothing of this run may still use the arena when the next one grows it
    cudaStreamSynchronize(stream ? stream : own_);
    for (auto& a : aux_) cudaStreamSynchronize(a);
    cudaGetLastError();
  }
  return rc;
}

int Engine::run_impl(const std::vector<SeriesInput>& in, std::vector<SeriesResult>& results,
                     cudaStream_t stream, GraphMode mode) {
  err_.clear();
  cudaError_t ce = cudaSetDevice(dev_);
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaSetDevice");
  const int count = static_cast<int>(in.size());
  results.assign(count, SeriesResult{});
  if (count == 0) return RQA_OK;
  cudaStream_t st = stream ? stream : own_;

  using clk = std::chrono::steady_clock;
  const bool tracing = trace_enabled();
  clk::time_point tp[6];
  tp[0] = clk::now();
  // ---- plan: validation, sizes, kernel classes
  struct P {
    Sizes z;
    int cls = -1;
    bool run = false;
    size_t o_hist, o_ends, o_cnt, o_desc, o_series, o_series2, o_xe, o_xe2, o_tab, o_cols,
        o_carry;
  };
  std::vector<P> plan(count);
  std::vector<int> dev_idx(count, -1);  // device slot of each runnable series
  int nrun = 0;
  // m, norm, f64, warps, kind, cols, wait test
  using Key = std::tuple<int, int, int, int, int, int, int>;
  std::map<Key, int> cls_of;
  std::vector<Key> classes;
  int64_t max_n_mp = 0, total_items = 0, max_len = 0;
  bool any_fp32 = false;
  for (int q = 0; q < count; ++q) {
    std::string msg;
    int s = validate_input(in[q], &msg);
    const char* why = nullptr;
    if (s == RQA_OK && in[q].dev) s = check_device_pointer(in[q].dev, 8, dev_, &why);
    if (s == RQA_OK && in[q].dev2) s = check_device_pointer(in[q].dev2, 8, dev_, &why);
    if (s == RQA_OK && in[q].bits_dev) s = check_device_pointer(in[q].bits_dev, 4, dev_, &why);
    if (why) msg = why;
    if (s != RQA_OK) {
      results[q].status = s;
      if (count == 1) return fail(s, msg);
      continue;
    }
    plan[q].run = true;
  }
  // In a set of several series, every series of a kernel group (kind, m,
  // norm, precision) gets the strip width chosen for the group's widest
  // matrix, so the group is one persistent launch (measured: 21 launches at
  // one width each beat 63 launches at per-series widths by 14 % on the
  // 4,096-series batch).
  using GroupKey = std::tuple<int, int, int, int>;
  std::map<GroupKey, int64_t> group_cols;
  auto group_of = [&](int q) {
    const rqa_settings& st = in[q].st;
    if (in[q].matrix) return GroupKey{2, 0, 0, 0};
    return GroupKey{in[q].cross ? 1 : 0, st.m, st.norm, st.precision == RQA_PREC_FP64 ? 1 : 0};
  };
  auto cols_of = [&](int q) {
    if (in[q].matrix) return in[q].N2;
    return nvec_of(in[q].st, in[q].cross ? in[q].N2 : in[q].N);
  };
  if (count > 1)
    for (int q = 0; q < count; ++q)
      if (plan[q].run) {
        int64_t& g = group_cols[group_of(q)];
        g = std::max(g, cols_of(q));
      }
  // Row bands in a set of several series: a series is cut into bands when
  // its tallest strip (rows / 32 block rows for one CTA) would outlast the
  // set's balanced share per resident CTA, i.e. when it alone would form
  // the launch's tail.  The set's work is counted in block rows of
  // 1,024-column strips (a rows x cols series: cols/1024 strips, rows/64
  // block rows on average for a triangle, rows/32 for a rectangle).
  double set_block_rows = 0.0;
  if (count > 1)
    for (int q = 0; q < count; ++q)
      if (plan[q].run) {
        const double rows =
            static_cast<double>(in[q].matrix ? in[q].N : nvec_of(in[q].st, in[q].N));
        const double cols = static_cast<double>(cols_of(q));
        const double per_strip = rows / ((in[q].cross || in[q].matrix) ? 32.0 : 64.0);
        set_block_rows += (cols / 1024.0 + 1.0) * per_strip;
      }
  const double share = set_block_rows / (3.0 * sms_);
  for (int q = 0; q < count; ++q) {
    P& p = plan[q];
    if (!p.run) continue;
    int warps = 0, cols = 0;
    if (count > 1) {
      const GroupKey g = group_of(q);
      const TileConfig gt = choose_tile(group_cols[g], std::get<1>(g), std::get<2>(g),
                                        std::get<3>(g) != 0, std::get<0>(g));
      warps = gt.warps;
      cols = gt.cols;
    }
    // row bands for a single series, or for one that would be the set's tail
    const double rows_q =
        static_cast<double>(in[q].matrix ? in[q].N : nvec_of(in[q].st, in[q].N));
    const bool bands_ok = in[q].withhold_warp == 0 && (count == 1 || rows_q / 32.0 > share);
    if (in[q].matrix)
      p.z = sizes_for(in[q].st, in[q].N, in[q].bits_dev == nullptr, true, in[q].N2, false, true,
                      warps, bands_ok, cols);
    else
      p.z = sizes_for(in[q].st, in[q].N, in[q].dev == nullptr, in[q].cross, in[q].N2,
                      in[q].dev2 == nullptr, false, warps, bands_ok, cols,
                      count == 1 && in[q].withhold_warp == 0 ? desc_budget() : 0);
    dev_idx[q] = nrun++;
    // kernel class: (m, norm, f64, warps, kind, columns per lane), kind 0
    // RQA, 1 cross, 2 matrix, plus 3 for the row-band instantiation of each
    const int bk = p.z.nbands > 1 ? 3 : 0;
    const int wt = in[q].withhold_warp > 0 ? 1 : 0;
    const Key k = p.z.matrix ? Key{0, 0, 0, p.z.tc.warps, 2 + bk, 4, 0}
                             : Key{in[q].st.m, in[q].st.norm, p.z.f64 ? 1 : 0, p.z.tc.warps,
                                   (p.z.cross ? 1 : 0) + bk, p.z.tc.cols, wt};
    auto it = cls_of.find(k);
    if (it == cls_of.end()) {
      it = cls_of.emplace(k, static_cast<int>(classes.size())).first;
      classes.push_back(k);
    }
    p.cls = it->second;
    if (!p.z.f64 && !p.z.matrix) {
      any_fp32 = true;
      max_n_mp = std::max(max_n_mp, (p.z.n + (p.z.cross ? p.z.n2 : 0)) * p.z.mp);
    }
    total_items += p.z.nitems;
    max_len = std::max(max_len, in[q].N + (in[q].cross ? in[q].N2 : 0));
  }
  const int ncls = static_cast<int>(classes.size());
  if (ncls == 0) {  // nothing runnable: report the first validation failure
    for (const auto& r : results)
      if (r.status != RQA_OK) return r.status;
    return RQA_OK;
  }

  // Classes run on up to kAux side streams so that small classes overlap
  // (their CTAs never wait on each other); the longest work goes first, each
  // class to the least loaded stream.  A single class runs on the main stream.
  std::vector<int> cls_order, cls_stream;
  const int nside = ncls > 1 ? std::min(ncls, kAux) : 0;
  std::vector<double> cls_work(ncls, 0.0);
  for (int q = 0; q < count; ++q)
    if (plan[q].run)
      cls_work[plan[q].cls] +=
          static_cast<double>(plan[q].z.n) * static_cast<double>(plan[q].z.n2);
  assign_streams(cls_work, nside, cls_order, cls_stream);
  // The series of each stream form a group (one group on the main stream
  // when nothing runs beside it) with contiguous descriptors, histograms and
  // counters: the group's merges and read-back follow its own tile kernels
  // on its stream, and the host computes its measures while the other groups
  // still run.
  const int ngrp = nside ? nside : 1;
  auto grp_of = [&](int q) { return nside ? cls_stream[plan[q].cls] : 0; };
  struct Grp {
    int first = 0, count = 0;
    int64_t max_n = 0;
    bool sym = false, cross = false, bands = false;
    double work = 0.0;
    size_t o_rb = 0, rb_bytes = 0;  // [histograms][counters] of the group
  };
  std::vector<Grp> grp(ngrp);
  std::vector<int> order;  // runnable series, group by group
  order.reserve(nrun);
  for (int g = 0; g < ngrp; ++g) {
    grp[g].first = static_cast<int>(order.size());
    for (int q = 0; q < count; ++q) {
      if (!plan[q].run || grp_of(q) != g) continue;
      const Sizes& z = plan[q].z;
      dev_idx[q] = static_cast<int>(order.size());
      order.push_back(q);
      grp[g].max_n = std::max(grp[g].max_n, z.cross ? z.n + z.n2 : z.n);
      (z.cross ? grp[g].cross : grp[g].sym) = true;
      grp[g].bands = grp[g].bands || z.nbands > 1;
      grp[g].work += static_cast<double>(z.n) * static_cast<double>(z.n2);
    }
    grp[g].count = static_cast<int>(order.size()) - grp[g].first;
  }

  // ---- arena layout: [descs][items][queues | hists | counters | ends | boundary
  // descriptors (zeroed)][series copies | FP32 vectors]
  size_t off = 0;
  const size_t o_sd = off;
  off += align256(sizeof(SeriesDesc) * nrun);
  const size_t o_items = off;
  off += align256(sizeof(Item) * static_cast<size_t>(std::max<int64_t>(total_items, 1)));
  const size_t o_tab0 = off;  // item offset tables of banded series
  for (auto& p : plan)
    if (p.run) {
      p.o_tab = off;
      off += p.z.tab;
    }
  // a single RQA series may run in strip groups, one tile launch (and work
  // queue counter) per group
  const int64_t ngroups = (count == 1 && plan[0].run) ? plan[0].z.ngroups : 1;
  const size_t o_zero = off;
  const size_t o_queue = off;
  off += align256(sizeof(int) * static_cast<size_t>(ncls + ngroups));
  const size_t o_hist0 = off;  // per group: [histograms][counters]
  size_t hist_bytes = 0, cnt_bytes = 0;
  for (Grp& gr : grp) {
    gr.o_rb = off;
    for (int i = gr.first; i < gr.first + gr.count; ++i) {
      P& p = plan[order[i]];
      p.o_hist = off;
      off += p.z.hist;
      hist_bytes += p.z.hist;
    }
    for (int i = gr.first; i < gr.first + gr.count; ++i) {
      P& p = plan[order[i]];
      p.o_cnt = off;
      off += p.z.cnt;
      cnt_bytes += p.z.cnt;
    }
    gr.rb_bytes = off - gr.o_rb;
  }
  for (auto& p : plan)
    if (p.run) {
      p.o_ends = off;
      off += p.z.ends;
      p.o_desc = off;
      off += p.z.desc;
      p.o_carry = off;
      off += p.z.carry;
      p.o_cols = off;
      off += p.z.cols;
    }
  const size_t zero_bytes = off - o_zero;
  const size_t o_series0 = off;
  for (auto& p : plan)
    if (p.run) {
      p.o_series = off;
      off += p.z.series;
      p.o_series2 = off;
      off += p.z.series2;
    }
  const size_t series_bytes = off - o_series0;
  for (auto& p : plan)
    if (p.run) {
      p.o_xe = off;
      off += p.z.xe;
      p.o_xe2 = off;
      off += p.z.xe2;
    }
  const size_t arena_bytes = off;

  // host staging: [descs][items][band tables] (the arena's first o_zero bytes,
  // copied in one piece) [histogram and counter read-back, laid out as on the
  // device from o_hist0][series]
  size_t hoff = 0;
  const size_t h_sd = hoff;
  const size_t h_items = o_items - o_sd;
  hoff += o_zero - o_sd;
  const size_t h_hist = hoff;
  hoff += hist_bytes + cnt_bytes;
  const size_t h_series = hoff;
  hoff += series_bytes;

  int rc = ensure_arena(arena_bytes, st);
  if (rc != RQA_OK) return rc;
  rc = ensure_host(hoff);
  if (rc != RQA_OK) return rc;

  tp[1] = clk::now();
  // ---- fill staging
  SeriesDesc* hsd = reinterpret_cast<SeriesDesc*>(host_ + h_sd);
  std::memset(hsd, 0, sizeof(SeriesDesc) * nrun);
  std::vector<HostCopy> copies;  // series into the pinned staging, done in parallel below
  for (int q = 0; q < count; ++q) {
    const P& p = plan[q];
    if (!p.run) continue;
    const rqa_settings& s = in[q].st;
    SeriesDesc& d = hsd[dev_idx[q]];
    if (p.z.matrix) {
      if (in[q].bits_dev) {
        d.bits = in[q].bits_dev;
      } else {
        d.bits = reinterpret_cast<const uint32_t*>(arena_ + p.o_series);
        copies.push_back({host_ + h_series + (p.o_series - o_series0), in[q].bits_host,
                          sizeof(uint32_t) * static_cast<size_t>(p.z.n * p.z.wpr)});
      }
      d.wpr = p.z.wpr;
    } else if (in[q].dev) {
      d.s = in[q].dev;
    } else {
      d.s = reinterpret_cast<const double*>(arena_ + p.o_series);
      copies.push_back({host_ + h_series + (p.o_series - o_series0), in[q].host,
                        sizeof(double) * static_cast<size_t>(in[q].N)});
    }
    d.xe = (p.z.f64 || p.z.matrix) ? nullptr : reinterpret_cast<float*>(arena_ + p.o_xe);
    d.N = in[q].N;
    d.withhold_warp = in[q].withhold_warp;
    d.withhold_seq = in[q].withhold_seq;
    d.n = p.z.n;
    desc_set_symmetric(d);
    if (p.z.matrix) {
      d.N2 = in[q].N2;
      d.n2 = p.z.n2;
      d.hl = p.z.hl;
      d.cross = 1;
    } else if (p.z.cross) {
      if (in[q].dev2) {
        d.s2 = in[q].dev2;
      } else {
        d.s2 = reinterpret_cast<const double*>(arena_ + p.o_series2);
        copies.push_back({host_ + h_series + (p.o_series2 - o_series0), in[q].host2,
                          sizeof(double) * static_cast<size_t>(in[q].N2)});
      }
      d.xe2 = p.z.f64 ? nullptr : reinterpret_cast<float*>(arena_ + p.o_xe2);
      d.N2 = in[q].N2;
      d.n2 = p.z.n2;
      d.hl = p.z.hl;
      d.cross = 1;
    }
    d.m = s.m;
    d.tau = s.tau;
    d.norm = s.norm;
    // a window of hl or more removes every cell, as any wider one does
    d.w = static_cast<int32_t>(std::min<int64_t>(s.theiler, p.z.hl));
    d.mp = p.z.mp;
    d.sw = 32 * p.z.tc.warps * p.z.tc.cols;
    d.eps = s.eps;
    d.band_override = s.band_override;
    d.hist = reinterpret_cast<unsigned long long*>(arena_ + p.o_hist);
    if (p.z.nbands > 1) {  // row bands: item offset table and column descriptors
      d.band_h = static_cast<int32_t>(p.z.band_h);
      d.nbands = static_cast<int32_t>(p.z.nbands);
      d.dia_off = reinterpret_cast<const int64_t*>(arena_ + p.o_tab);
      d.col_a = reinterpret_cast<uint32_t*>(arena_ + p.o_cols);
      d.col_z = d.col_a + (p.z.cols / 2) / sizeof(uint32_t);
    }
    {
      const size_t dbytes = align256(sizeof(uint16_t) * static_cast<size_t>(p.z.ndesc));
      const size_t rbytes = align256(sizeof(uint16_t) * static_cast<size_t>(p.z.nrowdesc));
      d.dia_a = reinterpret_cast<uint16_t*>(arena_ + p.o_desc);
      d.dia_z = reinterpret_cast<uint16_t*>(arena_ + p.o_desc + dbytes);
      if (!p.z.cross) {
        d.row_a = reinterpret_cast<uint16_t*>(arena_ + p.o_desc + 2 * dbytes);
        d.row_z = reinterpret_cast<uint16_t*>(arena_ + p.o_desc + 2 * dbytes + rbytes);
        d.colend = reinterpret_cast<uint32_t*>(arena_ + p.o_ends);
        d.rowend = d.colend + p.z.n;
        if (p.z.carry) {
          d.rcarry = reinterpret_cast<uint32_t*>(arena_ + p.o_carry);
          d.dcarry = reinterpret_cast<uint32_t*>(arena_ + p.o_carry + p.z.carry / 2);
        }
      }
    }
    d.counters = reinterpret_cast<unsigned long long*>(arena_ + p.o_cnt);
  }
  parallel_for(static_cast<int>(copies.size()), 8, [&](int k) {
    std::memcpy(copies[k].dst, copies[k].src, copies[k].bytes);
  });
  // work items per class, longest strips first
  Item* hitems = reinterpret_cast<Item*>(host_ + h_items);
  std::vector<int64_t> cls_start(ncls + 1, 0);
  {
    std::vector<std::vector<std::pair<int64_t, Item>>> per(ncls);
    for (int q = 0; q < count; ++q) {
      const P& p = plan[q];
      if (!p.run) continue;
      const int64_t sw = 32LL * p.z.tc.warps * p.z.tc.cols;
      if (p.z.nbands > 1) {  // items (Q, g), the table of their descriptor offsets
        int64_t* tab = reinterpret_cast<int64_t*>(host_ + h_sd + (p.o_tab - o_sd));
        std::fill(tab, tab + p.z.nstrips * p.z.nbands, int64_t(-1));
        int64_t dpos = 0;
        for_each_band_item(p.z, [&](int64_t Q, int64_t g, int64_t rows, int64_t cnt) {
          tab[Q * p.z.nbands + g] = dpos;
          dpos += cnt;
          per[p.cls].push_back({rows, Item{dev_idx[q], static_cast<int32_t>(Q),
                                           static_cast<int32_t>(g)}});
        });
      } else {
        for (int64_t Q = 0; Q < p.z.nstrips; ++Q) {  // strip height: the rows it spans
          const int64_t base = p.z.gstrips > 0 ? Q / p.z.gstrips * p.z.gstrips : 0;
          per[p.cls].push_back({p.z.cross ? p.z.n : p.z.n - Q * sw,
                                Item{dev_idx[q], static_cast<int32_t>(Q), 0,
                                     static_cast<int32_t>(base)}});
        }
      }
    }
    int64_t pos = 0;
    for (int c = 0; c < ncls; ++c) {
      std::stable_sort(per[c].begin(), per[c].end(),
                       [](const auto& a, const auto& b) { return a.first > b.first; });
      cls_start[c] = pos;
      for (auto& e : per[c]) hitems[pos++] = e.second;
    }
    cls_start[ncls] = pos;
  }

  tp[2] = clk::now();
  // ---- launch sequence
  SeriesDesc* d_sd = reinterpret_cast<SeriesDesc*>(arena_ + o_sd);
  Item* d_items = reinterpret_cast<Item*>(arena_ + o_items);
  int* d_queue = reinterpret_cast<int*>(arena_ + o_queue);

  std::vector<int64_t> key;
  if (mode != kNoGraph) {
    key.push_back(count);
    key.push_back(reinterpret_cast<int64_t>(arena_));
    key.push_back(reinterpret_cast<int64_t>(host_));
    key.push_back(reinterpret_cast<int64_t>(st));
    for (int q = 0; q < count; ++q) {
      key.push_back(in[q].N);
      key.push_back(plan[q].run ? 1 : 0);
      key.push_back(reinterpret_cast<int64_t>(in[q].dev));
      key.push_back(in[q].st.m);
      key.push_back(in[q].st.norm);
      key.push_back(in[q].st.precision);
      key.push_back(in[q].st.tau);
      key.push_back(in[q].cross ? 1 : 0);
      key.push_back(in[q].matrix ? 1 : 0);
      key.push_back(reinterpret_cast<int64_t>(in[q].bits_dev));
      // the plan's choices (strip width, row bands) may change between calls
      // with the same shapes (autotuning, environment overrides)
      key.push_back(plan[q].run ? plan[q].z.tc.warps : 0);
      key.push_back(plan[q].run ? plan[q].z.tc.cols : 0);
      key.push_back(plan[q].run ? plan[q].z.band_h : 0);
      key.push_back(plan[q].run ? plan[q].z.gstrips : 0);  // strip groups (descriptor budget)
      key.push_back(in[q].N2);
      key.push_back(reinterpret_cast<int64_t>(in[q].dev2));
    }
  }
  const bool cached = graph_ && key == graph_key_;
  const bool use_graph =
      mode == kGraph || (mode == kGraphOnRepeat && (cached || (!key.empty() && key == prev_key_)));
  if (mode == kGraphOnRepeat && !use_graph) prev_key_ = key;
  const bool replay = use_graph && cached;

  // timing events are external nodes when captured, so replays record them
  const unsigned evflags = use_graph ? cudaEventRecordExternal : cudaEventRecordDefault;

  int launches = 0;
  int64_t ctas_total = 0;
  auto enqueue = [&]() -> int {
    cudaError_t e;
    launches = 0;
    ctas_total = 0;
    if ((e = cudaEventRecordWithFlags(ev_[0], st, evflags)) != cudaSuccess)
      return cuda_fail(e, "cudaEventRecord");
    if ((e = cudaMemsetAsync(arena_ + o_zero, 0, zero_bytes, st)) != cudaSuccess)
      return cuda_fail(e, "cudaMemsetAsync");
    if ((e = cudaMemcpyAsync(arena_ + o_sd, host_ + h_sd, (o_zero - o_sd), cudaMemcpyHostToDevice,
                             st)) != cudaSuccess)
      return cuda_fail(e, "cudaMemcpyAsync(descriptors)");
    if (series_bytes &&
        (e = cudaMemcpyAsync(arena_ + o_series0, host_ + h_series, series_bytes,
                             cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return cuda_fail(e, "cudaMemcpyAsync(series)");
    launch_prepare(d_sd, nrun, max_len, sms_, st);
    launches += 2;
    if (any_fp32) {
      launch_embed(d_sd, nrun, max_n_mp, sms_, st);
      ++launches;
    }
    // the series state prepare wrote (error band and bound), read back before
    // the fork so that every group's completion implies it
    if ((e = cudaMemcpyAsync(host_ + h_sd, arena_ + o_sd, sizeof(SeriesDesc) * nrun,
                             cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return cuda_fail(e, "cudaMemcpyAsync(series state)");
    if ((e = cudaEventRecordWithFlags(ev_[1], st, evflags)) != cudaSuccess)
      return cuda_fail(e, "cudaEventRecord");
    if (nside) {
      if ((e = cudaEventRecord(fork_, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
      for (int k = 0; k < nside; ++k)
        if ((e = cudaStreamWaitEvent(aux_[k], fork_, 0)) != cudaSuccess)
          return cuda_fail(e, "cudaStreamWaitEvent");
    }
    for (int c : cls_order) {
      const int m = std::get<0>(classes[c]), norm = std::get<1>(classes[c]);
      const bool f64 = std::get<2>(classes[c]) != 0;
      const int warps = std::get<3>(classes[c]);
      const int kind = std::get<4>(classes[c]);
      const int cols = std::get<5>(classes[c]);
      const bool banded = kind >= 3;
      TileFn fn = kind % 3 == 2 ? tile_kernel_matrix(4, banded)
                                : tile_kernel_for(m, norm, cols, f64, kind % 3 == 1, banded);
      if (std::get<6>(classes[c])) fn = tile_kernel_wait_test();
      if (!fn) return fail(RQA_EINVAL, "no tile kernel for this (m, norm, columns per lane)");
      const size_t smem = tile_smem_for(kind % 3 == 2 ? 1 : m, norm, f64, warps, cols);
      if ((e = cudaFuncSetAttribute(reinterpret_cast<const void*>(fn),
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(smem))) != cudaSuccess)
        return cuda_fail(e, "cudaFuncSetAttribute");
      int per_sm = 0;
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
               &per_sm, reinterpret_cast<const void*>(fn), 32 * warps, smem)) != cudaSuccess)
        return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
      const int64_t nit = cls_start[c + 1] - cls_start[c];
      if (ngroups > 1) {
        // one series in strip groups (Sect. 4.1, Divide & Recombine with
        // carryover buffers): per group, the tile kernel over its strips
        // (their descriptors from the start of the buffer), then the row and
        // diagonal merges, which carry open runs to the next group
        const P& p = plan[0];
        for (int64_t gi = 0; gi < ngroups; ++gi) {
          const int64_t q0 = gi * p.z.gstrips;
          const int64_t q1 = std::min(p.z.nstrips, q0 + p.z.gstrips) - 1;
          if (gi > 0 &&
              (e = cudaMemsetAsync(arena_ + p.o_desc, 0, p.z.desc, st)) != cudaSuccess)
            return cuda_fail(e, "cudaMemsetAsync(group descriptors)");
          const int64_t gn = q1 - q0 + 1;
          const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(gn, (int64_t)per_sm * sms_));
          const SeriesDesc* a_sd = d_sd;
          const Item* a_items = d_items + cls_start[c] + q0;
          int a_n = static_cast<int>(gn);
          int* a_queue = d_queue + ncls + gi;
          void* args[] = {&a_sd, &a_items, &a_n, &a_queue};
          if ((e = cudaLaunchKernel(reinterpret_cast<const void*>(fn),
                                    dim3(static_cast<unsigned>(grid)), dim3(32 * warps), args,
                                    smem, st)) != cudaSuccess)
            return cuda_fail(e, "tile kernel launch");
          launches += 1 + launch_group_merges(d_sd, p.z.n, q0, q1, sms_, st);
          ctas_total += grid;
        }
        continue;
      }
      const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(nit, (int64_t)per_sm * sms_));
      const SeriesDesc* a_sd = d_sd;
      const Item* a_items = d_items + cls_start[c];
      int a_n = static_cast<int>(nit);
      int* a_queue = d_queue + c;
      void* args[] = {&a_sd, &a_items, &a_n, &a_queue};
      if ((e = cudaLaunchKernel(reinterpret_cast<const void*>(fn),
                                dim3(static_cast<unsigned>(grid)), dim3(32 * warps), args, smem,
                                cls_stream[c] >= 0 ? aux_[cls_stream[c]] : st)) != cudaSuccess)
        return cuda_fail(e, "tile kernel launch");
      ++launches;
      ctas_total += grid;
    }
    // per group, on its own stream after its tile kernels: the merges, then
    // one read-back of the group's histograms and counters
    for (int g = 0; g < ngrp; ++g) {
      cudaStream_t gs = nside ? aux_[g] : st;
      const Grp& gr = grp[g];
      if ((e = cudaEventRecordWithFlags(nside ? tiled_[g] : ev_[2], gs, evflags)) != cudaSuccess)
        return cuda_fail(e, "cudaEventRecord");
      if (gr.count > 0) {
        launches += launch_merges(d_sd + gr.first, gr.count, gr.max_n, gr.sym, gr.cross,
                                  gr.bands, sms_, gs, ngroups > 1);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "merge kernels launch");
        if ((e = cudaMemcpyAsync(host_ + h_hist + (gr.o_rb - o_hist0), arena_ + gr.o_rb,
                                 gr.rb_bytes, cudaMemcpyDeviceToHost, gs)) != cudaSuccess)
          return cuda_fail(e, "cudaMemcpyAsync(histograms)");
      }
      if ((e = cudaEventRecordWithFlags(done_[g], gs, evflags)) != cudaSuccess)
        return cuda_fail(e, "cudaEventRecord");
    }
    for (int k = 0; k < nside; ++k) {
      if ((e = cudaEventRecord(join_[k], aux_[k])) != cudaSuccess)
        return cuda_fail(e, "cudaEventRecord");
      if ((e = cudaStreamWaitEvent(st, join_[k], 0)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamWaitEvent");
    }
    if ((e = cudaEventRecordWithFlags(ev_[3], st, evflags)) != cudaSuccess)
      return cuda_fail(e, "cudaEventRecord");
    return RQA_OK;
  };

  // A caller's device series, with no stream given: the entry points order
  // the run on the legacy default stream, so the engine's own (non-blocking)
  // stream first waits for the work queued there (the series may still be
  // being written by it).  Outside any capture: a replay needs it as well.
  if (!stream) {
    bool dev_in = false;
    for (const auto& x : in) dev_in = dev_in || x.dev || x.dev2 || x.bits_dev;
    if (dev_in) {
      cudaError_t e = cudaEventRecord(order_, cudaStreamLegacy);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st, order_, 0);
      if (e != cudaSuccess) return cuda_fail(e, "ordering after the legacy default stream");
    }
  }

  if (use_graph) {
    if (!replay) {
      if (graph_) {
        cudaGraphExecDestroy(graph_);
        graph_ = nullptr;
      }
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
      rc = enqueue();
      e = cudaStreamEndCapture(st, &g);
      if (rc != RQA_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&graph_, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        graph_ = nullptr;
        return cuda_fail(e, "cudaGraphInstantiate");
      }
      graph_key_ = key;
      graph_launches_ = launches;
      graph_ctas_ = ctas_total;
    } else {
      launches = graph_launches_;  // the kernels the replayed graph launches
      ctas_total = graph_ctas_;
    }
    cudaError_t e = cudaGraphLaunch(graph_, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  } else {
    rc = enqueue();
    if (rc != RQA_OK) return rc;
  }
  tp[3] = clk::now();
  // ---- results: the measures of each series as soon as its group's
  // read-back has landed, the groups in the order their streams should finish
  std::vector<int> grp_order(ngrp);
  for (int g = 0; g < ngrp; ++g) grp_order[g] = g;
  std::stable_sort(grp_order.begin(), grp_order.end(),
                   [&](int a, int b) { return grp[a].work < grp[b].work; });
  std::vector<int> work_list;
  work_list.reserve(nrun);
  for (int g : grp_order)
    for (int i = grp[g].first; i < grp[g].first + grp[g].count; ++i) work_list.push_back(order[i]);
  std::atomic<bool> wait_failed{false};
  parallel_for(nrun, 8, [&](int i) {
    const int q = work_list[i];
    const P& p = plan[q];
    SeriesResult& r = results[q];
    thread_local int current_dev = -1;  // a worker thread waits on this device's events
    if (current_dev != dev_) {
      cudaSetDevice(dev_);
      current_dev = dev_;
    }
    if (cudaEventSynchronize(done_[grp_of(q)]) != cudaSuccess) {
      wait_failed = true;
      return;
    }
    const uint64_t* cnt = reinterpret_cast<const uint64_t*>(host_ + h_hist + (p.o_cnt - o_hist0));
    const SeriesDesc& d = hsd[dev_idx[q]];
    r.n = p.z.n;
    r.n2 = p.z.n2;
    r.hl = p.z.hl;
    r.status = static_cast<int>(cnt[CNT_STATUS]);
    if (r.status == RQA_OK) {
      const uint64_t* h = reinterpret_cast<const uint64_t*>(host_ + h_hist + (p.o_hist - o_hist0));
      const int64_t L1 = p.z.hl + 1;
      r.hist = h;
      int64_t last[3];
      for (int t = 0; t < 3; ++t)
        last[t] = std::min<int64_t>(static_cast<int64_t>(cnt[CNT_LAST + t]), p.z.hl);
      measures_from_histograms_last(h, h + L1, h + 2 * L1, last, p.z.n, p.z.n2,
                                    in[q].st.l_min, in[q].st.v_min, in[q].st.w_min, &r.meas);
    }
    rqa_stats_t& s = r.stats;
    s.n_vec = p.z.n;
    s.n_cols = p.z.n2;
    s.mode = p.z.matrix ? 2 : p.z.cross ? 1 : 0;
    s.pairs = p.z.cross ? cross_cell_count(p.z.n, p.z.n2, std::min<int64_t>(in[q].st.theiler, p.z.hl))
                        : pair_count(p.z.n, in[q].st.theiler);
    s.rechecks = static_cast<int64_t>(cnt[CNT_RECHECKS]);
    s.precision_used = p.z.matrix ? RQA_PREC_AUTO : p.z.f64 ? RQA_PREC_FP64 : RQA_PREC_FP32_RECHECK;
    s.band = p.z.f64 ? 0.0 : d.band_rel;
    s.band_bound = p.z.f64 ? 0.0 : d.bound_rel;
    s.exact = (p.z.f64 || p.z.matrix || d.band_rel >= d.bound_rel) ? 1 : 0;
    s.strip_width = 32 * p.z.tc.warps * p.z.tc.cols;
    s.band_rows = p.z.nbands > 1 ? p.z.band_h : 0;
    s.desc_bytes = static_cast<int64_t>(p.z.desc + p.z.carry);
    s.desc_bytes_all_strips = static_cast<int64_t>(p.z.desc_full);
    s.strip_groups = static_cast<int32_t>(p.z.ngroups);
    s.strips_per_group = static_cast<int32_t>(p.z.gstrips > 0 ? p.z.gstrips : p.z.nstrips);
    s.warps_per_cta = p.z.tc.warps;
    s.cols_per_lane = p.z.tc.cols;
    s.h2d_bytes = static_cast<int64_t>((o_zero - o_sd) + series_bytes);
    s.d2h_bytes = static_cast<int64_t>(hist_bytes + cnt_bytes + sizeof(SeriesDesc) * nrun);
    s.launches = launches;
    s.ctas = static_cast<int32_t>(ctas_total);
  });
  ce = cudaStreamSynchronize(st);
  tp[4] = clk::now();
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamSynchronize");
  if (wait_failed) return fail(RQA_ECUDA, "waiting for a group's read-back failed");
  if (nside) {  // tiles: from the fork to the last group's tile kernels
    tile_ms_ = 0.f;
    for (int g = 0; g < ngrp; ++g) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev_[1], tiled_[g]);
      tile_ms_ = std::max(tile_ms_, ms);
    }
  } else {
    cudaEventElapsedTime(&tile_ms_, ev_[1], ev_[2]);
  }
  cudaEventElapsedTime(&total_ms_, ev_[0], ev_[3]);
  for (int q : order) {
    results[q].stats.kernel_ms = tile_ms_;
    results[q].stats.total_ms = total_ms_;
  }
  last_sd_ = d_sd;
  last_f64_ = plan[0].run && plan[0].z.f64;
  last_matrix_ = plan[0].run && plan[0].z.matrix;
  last_stream_ = st;
  int first_err = RQA_OK;
  for (int q = 0; q < count && first_err == RQA_OK; ++q) {
    const SeriesResult& r = results[q];
    if (r.status == RQA_OK) continue;
    first_err = r.status;
    if (plan[q].run)
      err_ = r.status == RQA_ENAN       ? "series contains NaN or infinite values"
             : r.status == RQA_ETIMEOUT ? "a bounded device-side wait gave up"
                                        : "internal error: a line length outside 1..n";
  }
  if (tracing) {
    tp[5] = clk::now();
    auto ms = [&](int a, int b) {
      return std::chrono::duration<double, std::milli>(tp[b] - tp[a]).count();
    };
    std::fprintf(stderr,
                 "rqa trace: series=%d classes=%d plan=%.3f staging=%.3f enqueue=%.3f "
                 "device+results=%.3f finish=%.3f ms; device total=%.3f tile=%.3f ms%s\n",
                 count, ncls, ms(0, 1), ms(1, 2), ms(2, 3), ms(3, 4), ms(4, 5), total_ms_,
                 tile_ms_, use_graph ? (replay ? " (graph replay)" : " (graph capture)") : "");
  }
  return first_err;
}

int Engine::sample(const int64_t* i, const int64_t* j, int64_t count, uint8_t* out) {
  if (!last_sd_) return fail(RQA_EINVAL, "no run to sample from");
  if (last_matrix_) return fail(RQA_EINVAL, "a precomputed matrix has no decisions to sample");
  if (count <= 0) return RQA_OK;
  if (count > (int64_t(1) << 32)) return fail(RQA_EINVAL, "more than 2^32 decisions in one call");
  cudaError_t e = cudaSetDevice(dev_);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  void* buf = nullptr;
  const size_t bytes = count * (2 * sizeof(int64_t) + 1);
  if ((e = cudaMalloc(&buf, bytes)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(sample)");
  int64_t* di = static_cast<int64_t*>(buf);
  int64_t* dj = di + count;
  uint8_t* dout = reinterpret_cast<uint8_t*>(dj + count);
  cudaStream_t st = own_;
  int rc = RQA_OK;
  if ((e = cudaMemcpyAsync(di, i, count * sizeof(int64_t), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(dj, j, count * sizeof(int64_t), cudaMemcpyHostToDevice, st)) != cudaSuccess) {
    rc = cuda_fail(e, "cudaMemcpyAsync(sample)");
  } else {
    launch_sample(last_sd_, di, dj, count, dout, last_f64_ ? 1 : 0, st);
    if ((e = cudaMemcpyAsync(out, dout, count, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      rc = cuda_fail(e, "sample kernel");
  }
  cudaFree(buf);
  return rc;
}

}  // namespace rqa
