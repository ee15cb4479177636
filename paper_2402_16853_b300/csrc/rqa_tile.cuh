// rqa_tile.cuh -- the fused RQA tile kernel for sm_103a.
//
// One persistent CTA processes one CTA strip at a time: SW = warps * 32 * C
// consecutive columns of the upper triangle of the recurrence matrix (the
// matrix is symmetric, Sect. 4.2 notes the halved degree of parallelism of
// operator II for it).  Strips are taken from a work queue, longest first.
// Inside a strip, warp w owns 32*C columns (lane l owns columns
// col0 + l for C sub-blocks) and walks its rows bottom-up in blocks of 32.
//
// Per 32 x 32 sub-block the warp fuses the paper's three operators
// (Sect. 4.2):
//   I   create_recurrence_matrix -> FP32 distance per pair, the decision
//       packed by its sign bit into one 32-bit column word per lane; pairs in
//       the proven FP32 error band are re-decided in FP64;
//   II  detect_diagonal_lines     -> diagonal words from a bit-reverse,
//       rotate and 32x32 transpose of the column words, scanned for runs;
//   III detect_vertical_lines     -> the column words (upper part of full
//       column j) and the transposed row words (the part of full column i
//       below the line of identity, by symmetry), scanned for black and
//       white runs.
// Lines that cross sub-block borders are carried in registers (down a
// column, along a diagonal) or passed to the next warp through a shared-
// memory ring (rows and diagonals leaving the warp to the left).  Runs that
// touch the strip's own left or right edge are not counted here: their
// lengths go to small boundary descriptors that the merge kernels join
// across strips ("carryover buffers", Sect. 4.1).  The run of each full
// column that touches the line of identity is stored apart and joined by the
// finalize kernel.  Counts go to shared-memory histograms that are flushed
// once per strip.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "rqa_internal.h"

namespace rqa {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int HB = 1024;     // shared-memory histogram bins per line type
constexpr int RING = 8;      // slots of the warp-to-warp carry ring
constexpr long long SPIN_CYCLES = 4000000000LL;  // ~2 s at 2 GHz

// Run state words.  Two-colour state (rows, columns): length in bits 0..27,
// colour in bit 28, flag in bit 29 (the run touches the strip's right edge
// for rows, it is the column's first run for columns), done in bit 30.
// Diagonal state: black length in bits 0..27, edge flag in bit 28.
constexpr uint32_t ST_LEN = 0x0FFFFFFFu;
constexpr uint32_t ST_COLOUR = 1u << 28;
constexpr uint32_t ST_FLAG = 1u << 29;
constexpr uint32_t ST_DONE = 1u << 30;
constexpr uint32_t DG_EDGE = 1u << 28;

__device__ __forceinline__ uint32_t lowmask(int k) {
  return k >= 32 ? FULL : (k <= 0 ? 0u : ((1u << k) - 1u));
}

__device__ __forceinline__ int clamp32(int64_t v) {
  return v < 0 ? 0 : (v > 32 ? 32 : (int)v);
}

// 32 x 32 bit transpose across a warp: lane r holds row r (bit c = A[r][c]);
// on return lane c holds bit r = A[r][c].  Five shuffle stages, each swapping
// the off-diagonal blocks of 2j x 2j blocks.
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
#pragma unroll
  for (int j = 16; j >= 1; j >>= 1) {
    const uint32_t m = j == 16 ? 0x0000FFFFu
                     : j == 8  ? 0x00FF00FFu
                     : j == 4  ? 0x0F0F0F0Fu
                     : j == 2  ? 0x33333333u
                               : 0x55555555u;
    const uint32_t y = __shfl_xor_sync(FULL, x, j);
    x = (lane & j) ? ((x & ~m) | ((y >> j) & m)) : ((x & m) | ((y << j) & ~m));
  }
  return x;
}

// Status word value for an internal inconsistency (a line length outside
// 1..n); the entry point reports it as RQA_ECUDA.
constexpr unsigned long long STATUS_INTERNAL = 5ull;

// Shared-memory histogram with a global fallback for long lines.  A length
// outside 1..n is never written; it marks the series as failed instead.
struct HistSink {
  uint32_t* sh;              // [3][HB]
  unsigned long long* gl;    // [3][n+1]
  int64_t stride;            // n + 1
  unsigned long long* status;
  __device__ __forceinline__ void add(int type, uint32_t len) const {
    if (len < (uint32_t)HB && len > 0)
      atomicAdd(&sh[type * HB + len], 1u);
    else if (len > 0 && (int64_t)len < stride)
      atomicAdd(&gl[type * stride + len], 1ull);
    else
      atomicExch(status, STATUS_INTERNAL);
  }
};

// Scan cells hi..lo (descending bit index) of word x with two colours,
// continuing run state st.  close(colour, len, flag) is called for each run
// that ends inside the range; the open run is returned.
template <class F>
__device__ __forceinline__ uint32_t scan2(uint32_t x, int hi, int lo, uint32_t st,
                                          F&& close) {
  uint32_t col = (x >> hi) & 1u;
  uint32_t len = st & ST_LEN;
  uint32_t flag = (st & ST_FLAG) ? 1u : 0u;
  if (len != 0 && (((st & ST_COLOUR) ? 1u : 0u) != col)) {
    close((st & ST_COLOUR) ? 1u : 0u, len, flag);
    len = 0;
    flag = 0;
  }
  uint32_t T = (x ^ (x << 1)) & lowmask(hi + 1) & ~lowmask(lo + 1);
  int top = hi;
  while (T) {
    const int p = 31 - __clz(T);
    len += (uint32_t)(top - p + 1);
    close(col, len, flag);
    flag = 0;
    len = 0;
    col ^= 1u;
    top = p - 1;
    T &= lowmask(p);
  }
  len += (uint32_t)(top - lo + 1);
  return len | (col ? ST_COLOUR : 0u) | (flag ? ST_FLAG : 0u);
}

// Scan the black runs of cells hi..lo (descending) of x, continuing diagonal
// state st.  first(len) is called when the run that touches the strip's edge
// ends (len may be 0), emit(len) for every other run that ends inside.
template <class FA, class FE>
__device__ __forceinline__ uint32_t scan_black(uint32_t x, int hi, int lo, uint32_t st,
                                               FA&& first, FE&& emit) {
  const uint32_t seg = lowmask(hi + 1) & ~lowmask(lo);
  const uint32_t z = ~x & seg;
  uint32_t len = st & ST_LEN;
  const bool edge = (st & DG_EDGE) != 0;
  if (z == 0) return (len + (uint32_t)(hi - lo + 1)) | (edge ? DG_EDGE : 0u);
  const int ptop = 31 - __clz(z);
  const uint32_t fl = len + (uint32_t)(hi - ptop);
  if (edge)
    first(fl);
  else if (fl)
    emit(fl);
  const int pbot = __ffs(z) - 1;
  uint32_t mid = x & seg & lowmask(ptop) & ~lowmask(pbot + 1);
  while (mid) {
    const int h = 31 - __clz(mid);
    const int zz = 31 - __clz(z & lowmask(h));
    emit((uint32_t)(h - zz));
    mid &= lowmask(zz);
  }
  return (uint32_t)(pbot - lo);
}

// ---------------------------------------------------------------- distances
// FP32 margin of a pair: thr - d (L1, max) or thr - d^2 (L2), thr the scaled
// radius (squared for L2).  Non-negative <=> recurrent in FP32.  Explicit
// round-to-nearest intrinsics pin every operation (the error band is proven
// for exactly this sequence).
template <int M, int NORM>
__device__ __forceinline__ float pair_margin(const float* xr, const float* xc, float thr) {
  if (NORM == 1) {  // L2
    float acc = thr;
#pragma unroll
    for (int k = 0; k < M; ++k) {
      const float d = __fsub_rn(xr[k], xc[k]);
      acc = __fmaf_rn(-d, d, acc);
    }
    return acc;
  } else if (NORM == 2) {  // L1
    float acc = thr;
#pragma unroll
    for (int k = 0; k < M; ++k) acc = __fsub_rn(acc, fabsf(__fsub_rn(xr[k], xc[k])));
    return acc;
  } else {  // max
    float mx = 0.f;
#pragma unroll
    for (int k = 0; k < M; ++k) mx = fmaxf(mx, fabsf(__fsub_rn(xr[k], xc[k])));
    return __fsub_rn(thr, mx);
  }
}

// Exact FP64 decision, in the operation order of the specification (no
// fused multiply-add).
template <int NORM>
__device__ __forceinline__ bool exact_decision(const double* __restrict__ s, int64_t i,
                                               int64_t j, int m, int tau, double eps) {
  double acc = 0.0;
  for (int k = 0; k < m; ++k) {
    const double diff = __dsub_rn(s[i + (int64_t)k * tau], s[j + (int64_t)k * tau]);
    if (NORM == 0) {
      const double ad = fabs(diff);
      if (ad > acc) acc = ad;
    } else if (NORM == 2) {
      acc = __dadd_rn(acc, fabs(diff));
    } else {
      acc = __dadd_rn(acc, __dmul_rn(diff, diff));
    }
  }
  if (NORM == 1) acc = __dsqrt_rn(acc);
  return acc <= eps;
}

// Same decision with both vectors already in registers (FP64 path).
template <int M, int NORM>
__device__ __forceinline__ bool exact_decision_regs(const double* xr, const double* xc,
                                                    double eps) {
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < M; ++k) {
    const double diff = __dsub_rn(xr[k], xc[k]);
    if (NORM == 0) {
      const double ad = fabs(diff);
      if (ad > acc) acc = ad;
    } else if (NORM == 2) {
      acc = __dadd_rn(acc, fabs(diff));
    } else {
      acc = __dadd_rn(acc, __dmul_rn(diff, diff));
    }
  }
  if (NORM == 1) acc = __dsqrt_rn(acc);
  return acc <= eps;
}

// Bounded spin on a shared-memory counter.  Returns false (and raises the
// CTA abort flag) if the wait gave up or another warp already aborted.
__device__ __forceinline__ bool spin_until_ge(volatile int* ctr, int target,
                                              volatile int* abort_flag) {
  const long long t0 = clock64();
  while (*ctr < target) {
    if (*abort_flag) return false;
    if (clock64() - t0 > SPIN_CYCLES) {
      *abort_flag = 1;
      return false;
    }
    __nanosleep(32);
  }
  return true;
}

// Shared-memory bytes of the tile kernel.
template <int M, bool F64>
__host__ __device__ constexpr int tile_row_floats() {
  return F64 ? M : ((M + 3) / 4) * 4;
}
inline size_t tile_smem_bytes(int warps, int row_elems, int elem_bytes) {
  return (size_t)3 * HB * 4 + (size_t)warps * 32 * row_elems * elem_bytes +
         (size_t)(warps > 1 ? warps - 1 : 0) * RING * 64 * 4 + (size_t)2 * warps * 4 + 16;
}

// ------------------------------------------------------------------ kernel
template <int M, int NORM, int C, bool F64>
__global__ void __launch_bounds__(256)
tile_kernel(const SeriesDesc* __restrict__ sd, const Item* __restrict__ items, int nitems,
            int* __restrict__ queue) {
  using T = typename std::conditional<F64, double, float>::type;
  constexpr int MP = tile_row_floats<M, F64>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NW = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  uint32_t* sh_hist = reinterpret_cast<uint32_t*>(smem_raw);
  T* rowbuf = reinterpret_cast<T*>(sh_hist + 3 * HB) + warp * 32 * MP;
  T* rowbuf_end = reinterpret_cast<T*>(sh_hist + 3 * HB) + NW * 32 * MP;
  uint32_t* ring = reinterpret_cast<uint32_t*>(rowbuf_end);
  volatile int* prod = reinterpret_cast<volatile int*>(ring + (NW > 1 ? NW - 1 : 0) * RING * 64);
  volatile int* cons = prod + NW;
  __shared__ int s_item;
  __shared__ int s_skip;
  __shared__ volatile int s_abort;

  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const int it0 = atomicAdd(queue, 1);
      s_item = it0;
      s_skip = it0 < nitems
                   ? (int)((volatile unsigned long long*)sd[items[it0].series].counters)[CNT_STATUS]
                   : 0;
      s_abort = 0;
    }
    for (int q = threadIdx.x; q < 3 * HB; q += blockDim.x) sh_hist[q] = 0;
    if (threadIdx.x < 2 * NW) prod[threadIdx.x] = 0;
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) break;
    if (s_skip) continue;  // the series already failed (non-finite input or timeout)
    unsigned long long rechecks = 0;
    const Item wi = items[it];
    const SeriesDesc& S = sd[wi.series];
    const int64_t n = S.n;
    const int64_t SW = S.sw;
    const int64_t J1 = n - (int64_t)wi.strip * SW;             // strip: [J1-SW, J1)
    const int64_t off = strip_offset(n, SW, wi.strip);
    const int64_t jw1 = J1 - (int64_t)warp * 32 * C;           // warp: [jw0, jw1)
    const int64_t jw0 = jw1 - 32 * C;
    const int64_t wl_geo = (J1 - 2) / (32 * C);
    const int wlast = (int)(wl_geo < NW - 1 ? wl_geo : NW - 1);
    const HistSink hs{sh_hist, S.hist, n + 1, &S.counters[CNT_STATUS]};
    const int wtheiler = S.w;

    if (warp <= wlast) {
      const bool leftmost = warp == wlast;
      const int64_t jmax = jw1 - 1;
      const int bhi = (int)((jmax - 1) >> 5);
      const int bhi_left = leftmost ? -1 : (int)((jmax - 32 * C - 1) >> 5);
      uint32_t* ring_in = warp > 0 ? ring + (warp - 1) * RING * 64 : nullptr;
      uint32_t* ring_out = !leftmost ? ring + warp * RING * 64 : nullptr;
      int seq_in = 0, seq_out = 0;

      // Column vectors of this lane's C columns stay in registers for the strip.
      T xc[C][M];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int64_t j = jw0 + 32 * c + lane;
#pragma unroll
        for (int k = 0; k < M; ++k) {
          if constexpr (F64)
            xc[c][k] = j >= 0 ? (T)S.s[j + (int64_t)k * S.tau] : (T)0;
          else
            xc[c][k] = j >= 0 ? (T)S.xe[j * S.mp + k] : (T)0;
        }
      }
      uint32_t cst[C];   // column run state (first-run flag set)
      uint32_t dU[C];    // diagonal run leaving each sub-block upwards
#pragma unroll
      for (int c = 0; c < C; ++c) {
        cst[c] = ST_FLAG;
        dU[c] = 0;
      }
      const float thr = S.thr;
      const float band = S.band;
      bool ok = true;

      for (int b = bhi; b >= 0 && ok; --b) {
        const int64_t r0 = (int64_t)b << 5;
        {  // row vectors of rows r0 .. r0+31 into this warp's buffer
          const int64_t i = r0 + lane;
#pragma unroll
          for (int k = 0; k < MP; ++k) {
            T v = (T)0;
            if (i < n && k < M) {
              if constexpr (F64)
                v = S.s[i + (int64_t)k * S.tau];
              else
                v = S.xe[i * S.mp + k];
            }
            rowbuf[lane * MP + k] = v;
          }
        }
        __syncwarp();

        // ---- operator I: recurrence words (bit t = row r0 + t) per column
        uint32_t Rw[C];
        if constexpr (!F64) {
          uint32_t Nw[C];
          float mn[C];
#pragma unroll
          for (int c = 0; c < C; ++c) {
            Nw[c] = 0;
            mn[c] = __int_as_float(0x7f800000);
          }
#pragma unroll 4
          for (int t = 31; t >= 0; --t) {
            float xr[MP];
#pragma unroll
            for (int k = 0; k < MP; k += 4) {
              const float4 v = *reinterpret_cast<const float4*>(
                  reinterpret_cast<const float*>(rowbuf) + t * MP + k);
              xr[k] = v.x;
              if (k + 1 < MP) xr[k + 1] = v.y;
              if (k + 2 < MP) xr[k + 2] = v.z;
              if (k + 3 < MP) xr[k + 3] = v.w;
            }
#pragma unroll
            for (int c = 0; c < C; ++c) {
              const float acc = pair_margin<M, NORM>(xr, (const float*)xc[c], thr);
              Nw[c] = __funnelshift_l(__float_as_uint(acc), Nw[c], 1);
              mn[c] = fminf(mn[c], fabsf(acc));
            }
          }
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const int64_t j = jw0 + 32 * c + lane;
            const uint32_t live = j < 0 ? 0u
                                        : lowmask(clamp32(j - r0)) &
                                              lowmask(clamp32(j - wtheiler - r0 + 1));
            uint32_t R = ~Nw[c] & live;
            if (mn[c] <= band && live) {
              // near-radius pairs: re-decide in FP64 with the exact order
              uint32_t todo = live;
              while (todo) {
                const int t = __ffs(todo) - 1;
                todo &= todo - 1;
                float xr[M];
#pragma unroll
                for (int k = 0; k < M; ++k)
                  xr[k] = reinterpret_cast<const float*>(rowbuf)[t * MP + k];
                const float acc = pair_margin<M, NORM>(xr, (const float*)xc[c], thr);
                if (fabsf(acc) <= band) {
                  const bool r = exact_decision<NORM>(S.s, r0 + t, j, M, S.tau, S.eps);
                  R = r ? (R | (1u << t)) : (R & ~(1u << t));
                  ++rechecks;
                }
              }
            }
            Rw[c] = R;
          }
        } else {
#pragma unroll
          for (int c = 0; c < C; ++c) Rw[c] = 0;
          for (int t = 31; t >= 0; --t) {
            double xr[M];
#pragma unroll
            for (int k = 0; k < M; ++k) xr[k] = reinterpret_cast<const double*>(rowbuf)[t * MP + k];
#pragma unroll
            for (int c = 0; c < C; ++c) {
              const bool r = exact_decision_regs<M, NORM>(xr, (const double*)xc[c], S.eps);
              Rw[c] = (Rw[c] << 1) | (r ? 1u : 0u);
            }
          }
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const int64_t j = jw0 + 32 * c + lane;
            const uint32_t live = j < 0 ? 0u
                                        : lowmask(clamp32(j - r0)) &
                                              lowmask(clamp32(j - wtheiler - r0 + 1));
            Rw[c] &= live;
          }
        }
        __syncwarp();

        // ---- carries entering from the right (CTA edge or previous warp)
        uint32_t rst;   // row r0 + lane
        uint32_t dL;    // diagonal entering sub-block C-1's upper segment, lane d
        if (warp == 0) {
          rst = ST_FLAG;
          dL = DG_EDGE;
        } else {
          if (lane == 0) ok = spin_until_ge(prod + (warp - 1), seq_in + 1, &s_abort);
          ok = __shfl_sync(FULL, ok, 0);
          if (!ok) break;
          __threadfence_block();
          const volatile uint32_t* slot = ring_in + (seq_in % RING) * 64;
          rst = slot[lane];
          dL = slot[32 + lane];
          __syncwarp();
          if (lane == 0) cons[warp] = seq_in + 1;
          ++seq_in;
        }

        const int64_t irow = r0 + lane;
#pragma unroll
        for (int c = C - 1; c >= 0; --c) {
          const int64_t col0 = jw0 + 32 * c;
          const int64_t j = col0 + lane;
          const uint32_t R = Rw[c];

          // ---- operator III, upper part of full column j (rows < j)
          {
            const int vt = j < 0 ? 0 : clamp32(j - r0);
            if (vt > 0) {
              cst[c] = scan2(R, vt - 1, 0, cst[c], [&](uint32_t col, uint32_t len, uint32_t first) {
                if (first)
                  S.colend[j] = len | (col << 31);
                else
                  hs.add(col ? HIST_VERT : HIST_WHITE, len);
              });
            }
          }

          // ---- operator III, lower part of full column irow = upper row irow
          {
            const uint32_t RW = transpose32(R, lane);
            const int64_t lo = irow + 1 - col0;  // first valid bit of the row
            if (lo <= 31 && !(rst & ST_DONE) && irow <= J1 - 2) {
              const int lo_c = lo < 0 ? 0 : (int)lo;
              rst = scan2(RW, 31, lo_c, rst, [&](uint32_t col, uint32_t len, uint32_t edge) {
                if (edge)
                  S.row_a[off + irow] = (uint16_t)((len << 1) | col);
                else
                  hs.add(col ? HIST_VERT : HIST_WHITE, len);
              });
              if (lo >= 0) {  // the row ends here, at column irow + 1
                const uint32_t len = rst & ST_LEN, col = (rst & ST_COLOUR) ? 1u : 0u;
                const uint32_t same = (rst & ST_FLAG) ? 1u : 0u;
                S.row_z[off + irow] = (uint16_t)((len << 2) | (same << 1) | col);
                if (same) S.row_a[off + irow] = 0;
                rst = ST_DONE;
              }
            }
          }

          // ---- operator II, diagonal segments (lane d)
          {
            uint32_t Rr = __brev(R);
            Rr = __funnelshift_r(Rr, Rr, 31 - lane);
            const uint32_t D = transpose32(Rr, lane);
            const int d = lane;
            // lower segment: bits d-1..0, diagonal k = col0 - r0 + d - 32,
            // continues the upper segment of the block below (dU[c]).
            const int64_t klo = col0 - r0 + d - 32;
            uint32_t Lnext = dU[c];
            if (d > 0) {
              Lnext = scan_black(
                  D, d - 1, 0, dU[c],
                  [&](uint32_t len) {
                    if (klo >= 1) S.dia_a[off + klo - 1] = (uint16_t)len;
                  },
                  [&](uint32_t len) { hs.add(HIST_DIAG, len); });
            }
            // upper segment: bits 31..d, diagonal k = col0 - r0 + d, continues
            // the lower segment of the sub-block to the right (dL).
            const int64_t kup = col0 - r0 + d;
            dU[c] = scan_black(
                D, 31, d, dL,
                [&](uint32_t len) {
                  if (kup >= 1) S.dia_a[off + kup - 1] = (uint16_t)len;
                },
                [&](uint32_t len) { hs.add(HIST_DIAG, len); });
            dL = Lnext;
          }
        }

        // ---- carries leaving to the left
        if (leftmost) {
          if (!(rst & ST_DONE) && irow <= J1 - 2) {
            const uint32_t len = rst & ST_LEN, col = (rst & ST_COLOUR) ? 1u : 0u;
            const uint32_t same = (rst & ST_FLAG) ? 1u : 0u;
            if (len > 0) {
              S.row_z[off + irow] = (uint16_t)((len << 2) | (same << 1) | col);
              if (same) S.row_a[off + irow] = 0;
            }
          }
          const int64_t kx = jw0 - r0 + lane - 32;  // diagonal leaving through the left edge
          if (kx >= 1) {
            S.dia_z[off + kx - 1] = (uint16_t)((dL & ST_LEN) | ((dL & DG_EDGE) ? 0x8000u : 0u));
          }
        } else if (b <= bhi_left) {
          if (lane == 0) ok = spin_until_ge(cons + (warp + 1), seq_out - RING + 1, &s_abort);
          ok = __shfl_sync(FULL, ok, 0);
          if (!ok) break;
          uint32_t* slot = ring_out + (seq_out % RING) * 64;
          slot[lane] = rst;
          slot[32 + lane] = dL;
          __syncwarp();
          __threadfence_block();
          if (lane == 0) prod[warp] = seq_out + 1;
          ++seq_out;
        }
      }

      if (ok) {
        // ---- top border: close column runs, record diagonal ends (row 0)
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const int64_t j = jw0 + 32 * c + lane;
          if (j >= 1) {
            const uint32_t st = cst[c];
            const uint32_t len = st & ST_LEN, col = (st & ST_COLOUR) ? 1u : 0u;
            if (len > 0) {
              if (st & ST_FLAG)
                S.colend[j] = len | (col << 31);
              else
                hs.add(col ? HIST_VERT : HIST_WHITE, len);
            }
            // diagonal k = j ends at (0, j)
            S.dia_z[off + j - 1] =
                (uint16_t)((dU[c] & ST_LEN) | ((dU[c] & DG_EDGE) ? 0x8000u : 0u));
          }
        }
      }
    }
    __syncthreads();
    if (s_abort && threadIdx.x == 0)
      atomicExch(&S.counters[CNT_STATUS], 6ull /* RQA_ETIMEOUT */);
    // flush the strip's histograms
    const int64_t stride = n + 1;
    for (int q = threadIdx.x; q < 3 * HB; q += blockDim.x) {
      const uint32_t v = sh_hist[q];
      if (v) atomicAdd(&S.hist[(q / HB) * stride + (q % HB)], (unsigned long long)v);
    }
    // rechecks of this strip: one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rechecks += __shfl_xor_sync(FULL, rechecks, o);
    if (lane == 0 && rechecks) atomicAdd(&S.counters[CNT_RECHECKS], rechecks);
  }
}

}  // namespace rqa
