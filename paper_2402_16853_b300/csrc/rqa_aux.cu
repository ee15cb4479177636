// rqa_aux.cu -- the kernels around the fused tile kernel:
//   prepare   per series: min / max / non-finite check, centring and power-
//             of-two scaling for the FP32 copy, FP32 radius and the proven
//             FP32 recheck band;
//   embed     time-delay embedding (Sect. 2, Sect. 7.2) into FP32 vectors;
//   merge     join the boundary descriptors of the CTA strips along every
//             row and every diagonal (the carryover buffers of Sect. 4.1),
//             for cross recurrence along the diagonals of the rectangle;
//   finalize  join the runs of each full column at the line of identity and
//             form the full diagonal histogram from the upper triangle;
//   sample    individual decisions R_ij for spot checks.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "rqa_internal.h"
#include "rqa_kernels.h"
#include "rqa_tile.cuh"

namespace rqa {

// ----------------------------------------------------------------- prepare
// A double as an unsigned integer with the same order (finite values).
__device__ __forceinline__ unsigned long long ordered_bits(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double from_ordered_bits(unsigned long long o) {
  return __longlong_as_double((long long)((o >> 63) ? (o & 0x7FFFFFFFFFFFFFFFull) : ~o));
}

// Minimum, maximum and non-finite check of series blockIdx.y (and, for cross
// recurrence, of the second series), blockIdx.x taking a grid-stride share:
// min and max are order-independent, so combining the blocks by atomic
// maxima of the encoded values is deterministic.
__global__ void prepare_scan_kernel(SeriesDesc* __restrict__ sd) {
  SeriesDesc& S = sd[blockIdx.y];
  if (S.n <= 0 || !S.s || !S.counters) return;  // nothing to prepare
  __shared__ double s_mn[32], s_mx[32];
  __shared__ int s_bad[32];
  double mn = INFINITY, mx = -INFINITY;
  int bad = 0;
  // cross recurrence: both series share one centre and scale, so FP32
  // differences of a row and a column vector are differences of the values
  const int64_t total = S.cross ? S.N + S.N2 : S.N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = i < S.N ? S.s[i] : S.s2[i - S.N];
    if (!isfinite(v)) {
      bad = 1;
    } else {
      mn = fmin(mn, v);
      mx = fmax(mx, v);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    mn = fmin(mn, __shfl_xor_sync(FULL, mn, o));
    mx = fmax(mx, __shfl_xor_sync(FULL, mx, o));
    bad |= __shfl_xor_sync(FULL, bad, o);
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0) {
    s_mn[wid] = mn;
    s_mx[wid] = mx;
    s_bad[wid] = bad;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 1; w < nw; ++w) {
    mn = fmin(mn, s_mn[w]);
    mx = fmax(mx, s_mx[w]);
    bad |= s_bad[w];
  }
  if (bad) atomicCAS(&S.counters[CNT_STATUS], 0ull, 3ull /* RQA_ENAN */);
  if (mn <= mx) {  // the block saw a finite value
    atomicMax(&S.counters[CNT_LO], ~ordered_bits(mn));
    atomicMax(&S.counters[CNT_HI], ordered_bits(mx));
  }
}

// Centre, scale, FP32 radius and proven error band of each series, from the
// minimum and maximum prepare_scan_kernel gathered (one thread per series).
__global__ void prepare_kernel(SeriesDesc* __restrict__ sd, int count) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  SeriesDesc& S = sd[q];
  if (S.n <= 0 || !S.s || !S.counters) return;
  if (S.counters[CNT_STATUS] == 3ull) return;  // non-finite input
  const double mn = from_ordered_bits(~S.counters[CNT_LO]);
  const double mx = from_ordered_bits(S.counters[CNT_HI]);
  // Centre on the mid-range (minimises max |s - c|) and scale by a power of
  // two so the FP32 copies lie in [-1, 1].
  const double center = 0.5 * mn + 0.5 * mx;
  const double dev = fmax(mx - center, center - mn) * (1.0 + 0x1p-50);
  double scale = 1.0;
  if (dev > 0.0) scale = ldexp(1.0, -ilogb(dev) - 1);
  double E = S.eps * scale;
  if (!(E <= 0x1p20)) E = 0x1p20;  // every pair recurs by a huge margin
  const double Ms = dev * scale;
  const double u = 0x1p-24, m = (double)S.m, sm = sqrt(m);
  double unit, bound;
  // Bounds on |FP32 margin - exact margin| for the operation sequences of
  // pair_margin(), from the rounding of the FP32 copies (<= u Ms each), of
  // each subtraction, accumulation and of the radius, plus the rounding of
  // the FP64 decision itself; doubled for the first-order terms' neglected
  // higher orders.
  if (S.norm == 1) {
    const double a = 2.0 * u * Ms + u * E;
    unit = E * E;
    bound = 2.02 * ((3.0 + m + 2.0 * sm) * u * E * E + 2.0 * a * sm * E + m * a * a) +
            (m + 3.0) * 0x1p-52 * E * E;
  } else if (S.norm == 2) {
    unit = E;
    bound = 2.02 * ((1.0 + 2.0 * m) * u * E + 2.0 * m * u * Ms) + (m + 3.0) * 0x1p-52 * E;
  } else {
    unit = E;
    bound = 2.02 * (3.0 * u * E + 2.0 * u * Ms) + 4.0 * 0x1p-52 * E;
  }
  double band = fmax(1e-5 * unit, bound);
  // The FP64 definition itself leaves the normal range when the squares or
  // sums of the differences (at most 2 dev each) overflow, or when squares or
  // sums of radius-sized differences underflow; there the scaled FP32 test
  // could decide a pair differently from it, so every pair is re-decided.
  const double span = 2.0 * dev;
  const bool fp64_range = S.norm == 1   ? (span > 1e150 / sm || S.eps < 1e-140)
                          : S.norm == 2 ? (span * m > 1e300 || S.eps < 1e-290)
                                        : span > 1e300;
  if (S.band_override >= 0.0)
    band = S.band_override * unit;
  else if (bound >= 0.25 * unit || fp64_range)
    band = INFINITY;  // the FP32 test would decide almost nothing: re-decide all
  float thr;
  if (S.norm == 1) {
    const float e32 = __double2float_rn(E);
    thr = __fmul_rn(e32, e32);
  } else {
    thr = __double2float_rn(E);
  }
  S.center = center;
  S.scale = scale;
  S.thr = thr;
  S.band = __double2float_ru(band);
  S.band_rel = band / unit;
  S.bound_rel = bound / unit;
}

// ------------------------------------------------------------------- embed
// Rows' vectors into xe; for cross recurrence the columns' into xe2 after.
__global__ void embed_kernel(SeriesDesc* __restrict__ sd) {
  const SeriesDesc& S = sd[blockIdx.y];
  if (S.n <= 0 || !S.xe || !S.s) return;
  const int64_t rows = S.n * S.mp;
  const int64_t total = S.cross ? rows + S.n2 * S.mp : rows;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const bool second = q >= rows;
    const int64_t qq = second ? q - rows : q;
    const double* src = second ? S.s2 : S.s;
    const int64_t i = qq / S.mp;
    const int k = (int)(qq - i * S.mp);
    float v = 0.f;
    if (k < S.m)
      v = __double2float_rn(__dmul_rn(__dsub_rn(src[i + (int64_t)k * S.tau], S.center), S.scale));
    (second ? S.xe2 : S.xe)[qq] = v;
  }
}

// ------------------------------------------------- block-level histograms
struct BlockHist {
  uint32_t* sh;   // [3][HB]
  __device__ void init() {
    for (int q = threadIdx.x; q < 3 * HB; q += blockDim.x) sh[q] = 0;
    __syncthreads();
  }
  __device__ void add(const SeriesDesc& S, int type, uint64_t len) {
    if (len < (uint64_t)HB && len > 0)
      atomicAdd(&sh[type * HB + len], 1u);
    else if (len > 0 && len <= (uint64_t)S.hl)
      atomicAdd(&S.hist[type * (S.hl + 1) + len], 1ull);
    else
      atomicCAS(&S.counters[CNT_STATUS], 0ull, STATUS_INTERNAL);  // the first error stays
  }
  __device__ void flush(const SeriesDesc& S) {
    __syncthreads();
    for (int q = threadIdx.x; q < 3 * HB; q += blockDim.x) {
      const uint32_t v = sh[q];
      if (v) atomicAdd(&S.hist[(q / HB) * (S.hl + 1) + (q % HB)], (unsigned long long)v);
    }
  }
};

__device__ __forceinline__ void emit2(BlockHist& h, const SeriesDesc& S, uint32_t col,
                                      uint64_t len) {
  if (len) h.add(S, col ? HIST_VERT : HIST_WHITE, len);
}

// ------------------------------------------------------------ merge: rows
// Row i (cells (i, j), j > i) crosses strips Q = 0 .. (n-2-i)/sw from right
// to left.  Each strip left a descriptor: the run touching its right edge
// (a) and the run touching its left end (z), or one run over the whole
// segment.  Join them in order; the run left open at column i+1 is the row's
// end run for the line-of-identity join.
// Descriptors are read MERGE_AHEAD strips (items) at a time, all loads of
// a group issued before any is used: the walk along a row or diagonal is
// sequential, but its addresses follow from the geometry alone, so the
// loads need not wait on each other.
constexpr int MERGE_AHEAD = 8;

// Strips q0 .. q1 of a series that runs in strip groups (q1 < 0: all strips
// at once).  A row or diagonal that continues past the group's left edge
// leaves its open run in rcarry / dcarry, and the next group starts from it;
// the descriptors of strip Q sit at strip_offset(Q) - strip_offset(q0).
__device__ void merge_rows_body(uint32_t* sh, SeriesDesc* __restrict__ sd, int64_t q0, int64_t q1) {
  const SeriesDesc& S = sd[blockIdx.y];
  if (S.n <= 0 || !S.hist || S.cross) return;
  BlockHist h{sh};
  h.init();
  const int64_t n = S.n, sw = S.sw;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n - 1;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t qrow = (n - 2 - i) / sw;   // the row's last strip
    if (qrow < q0) continue;                 // it ended in an earlier group
    const int64_t qlast = q1 >= 0 && q1 < qrow ? q1 : qrow;
    uint32_t ocol = 0;
    uint64_t olen = 0;
    if (q0 > 0) {
      const uint32_t c = S.rcarry[i];
      olen = c & 0x7FFFFFFFu;
      ocol = c >> 31;
    }
    int64_t off = i;  // strip_offset(n, sw, Q) - strip_offset(n, sw, q0) + i
    for (int64_t Q0 = q0; Q0 <= qlast; Q0 += MERGE_AHEAD) {
      uint32_t zs[MERGE_AHEAD], as[MERGE_AHEAD];
#pragma unroll
      for (int u = 0; u < MERGE_AHEAD; ++u) {
        const int64_t Q = Q0 + u;
        zs[u] = 0;
        as[u] = 0;
        if (Q <= qlast) {
          zs[u] = S.row_z[off];
          as[u] = S.row_a[off];
          off += n - 1 - Q * sw;  // strip Q holds J1(Q) - 1 = n - Q sw - 1 entries
        }
      }
#pragma unroll
      for (int u = 0; u < MERGE_AHEAD; ++u) {
        if (Q0 + u > qlast) break;
        const uint32_t z = zs[u];
        const uint32_t zlen = z >> 2, zcol = z & 1u;
        if (z & 2u) {  // one run over the whole segment
          if (olen && ocol == zcol) {
            olen += zlen;
          } else {
            emit2(h, S, ocol, olen);
            ocol = zcol;
            olen = zlen;
          }
        } else {
          const uint32_t a = as[u];
          const uint32_t alen = a >> 1, acol = a & 1u;
          if (olen && ocol == acol) {
            emit2(h, S, acol, olen + alen);
          } else {
            emit2(h, S, ocol, olen);
            emit2(h, S, acol, alen);
          }
          ocol = zcol;
          olen = zlen;
        }
      }
    }
    if (qlast == qrow)
      S.rowend[i] = (uint32_t)olen | (ocol << 31);
    else
      S.rcarry[i] = (uint32_t)olen | (ocol << 31);
  }
  h.flush(S);
}

// ------------------------------------------------------- merge: diagonals
// Diagonal k >= 1 (cells (i, i+k)) starts at (n-1-k, n-1) and ends at (0, k).
// Walked in that order it crosses the items (strip Q, band g) one after the
// other: it leaves an item through its left edge (column J0) or its top edge
// (row R0), at row max(R0, J0 - k), and continues at the next cell up-left.
// Each item left the black run touching the diagonal's entry (a), the black
// run touching its exit (z), or an all-black flag.  With one band the items
// are the strips, Q = 0 .. (n-1-k)/sw.
__device__ void merge_diags_body(uint32_t* sh, SeriesDesc* __restrict__ sd, int64_t q0, int64_t q1) {
  const SeriesDesc& S = sd[blockIdx.y];
  if (S.n <= 0 || !S.hist || S.cross) return;
  BlockHist h{sh};
  h.init();
  const int64_t n = S.n, sw = S.sw;
  const bool banded = S.nbands > 1;
  const int64_t H = banded ? S.band_h : n;
  for (int64_t k = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    // entry row of the next item (-1: the walk is done); diagonal k enters
    // strip Q at row n - 1 - k - Q sw
    int64_t i = n - 1 - k - q0 * sw;
    if (i < 0) continue;  // the diagonal ended in an earlier group
    uint64_t L = q0 > 0 ? S.dcarry[k] : 0;
    if (!banded) {
      // one band: the items are the strips Q = q0, q0 + 1, ... in order (the
      // diagonal leaves strip Q through its left edge J0 into strip Q + 1)
      // and band_klo is 1, so no division is needed
      int64_t Q = q0, off = 0;  // off = strip_offset(n, sw, Q) - strip_offset(n, sw, q0)
      while (i >= 0 && (q1 < 0 || Q <= q1)) {
        int64_t os[MERGE_AHEAD];
        int cnt = 0;
#pragma unroll
        for (int u = 0; u < MERGE_AHEAD; ++u) {
          os[u] = -1;
          if (i >= 0 && (q1 < 0 || Q <= q1)) {
            os[u] = off + k - 1;
            ++cnt;
            const int64_t ie = n - (Q + 1) * sw - k;  // J0 - k, the top cell's row
            off += n - 1 - Q * sw;
            ++Q;
            i = ie > 0 ? ie - 1 : -1;
          }
        }
        uint32_t zs[MERGE_AHEAD], as[MERGE_AHEAD];
#pragma unroll
        for (int u = 0; u < MERGE_AHEAD; ++u) {
          zs[u] = os[u] >= 0 ? S.dia_z[os[u]] : 0u;
          as[u] = os[u] >= 0 ? S.dia_a[os[u]] : 0u;
        }
#pragma unroll
        for (int u = 0; u < MERGE_AHEAD; ++u) {
          if (u >= cnt) break;
          const uint32_t z = zs[u];
          if (z & 0x8000u) {
            L += (z & 0x7FFFu);
          } else {
            const uint64_t first = L + as[u];
            if (first) h.add(S, HIST_DIAG, first);
            L = z & 0x7FFFu;
          }
        }
      }
    }
    while (banded && i >= 0) {
      // the next items' descriptor positions, from the geometry alone
      int64_t os[MERGE_AHEAD];
      int cnt = 0;
#pragma unroll
      for (int u = 0; u < MERGE_AHEAD; ++u) {
        os[u] = -1;
        if (i >= 0) {
          const int64_t Q = (n - 1 - (i + k)) / sw;
          const int64_t J1 = n - Q * sw, J0 = J1 - sw;
          const int64_t g = banded ? i / H : 0;
          const int64_t R0 = g * H, R1 = R0 + H < n ? R0 + H : n;
          const int64_t off = banded ? S.dia_off[Q * S.nbands + g] : strip_offset(n, sw, Q);
          os[u] = off + k - band_klo(J1, sw, R1);
          ++cnt;
          const int64_t ie = R0 > J0 - k ? R0 : J0 - k;  // the diagonal's top cell in the item
          i = ie > 0 ? ie - 1 : -1;
        }
      }
      uint32_t zs[MERGE_AHEAD], as[MERGE_AHEAD];
#pragma unroll
      for (int u = 0; u < MERGE_AHEAD; ++u) {
        zs[u] = os[u] >= 0 ? S.dia_z[os[u]] : 0u;
        as[u] = os[u] >= 0 ? S.dia_a[os[u]] : 0u;
      }
#pragma unroll
      for (int u = 0; u < MERGE_AHEAD; ++u) {
        if (u >= cnt) break;
        const uint32_t z = zs[u];
        if (z & 0x8000u) {
          L += (z & 0x7FFFu);
        } else {
          const uint64_t first = L + as[u];
          if (first) h.add(S, HIST_DIAG, first);
          L = z & 0x7FFFu;
        }
      }
    }
    if (i >= 0 && q1 >= 0)
      S.dcarry[k] = (uint32_t)L;  // continues in the next group
    else if (L)
      h.add(S, HIST_DIAG, L);
  }
  h.flush(S);
}

// ------------------------------------------------------ merge: columns
// Row bands only.  Column j (rows 0 .. j-1 of the upper triangle) crosses
// bands gb = (j-1)/H down to 0.  Every band holds the column's first run in
// col_a -- in band gb the run touching row j-1, above it the run touching
// the band's bottom edge -- unless the column's segment there is one run, and
// its top run in col_z (with a flag when the segment is one run); band 0
// closed its top run itself unless it is one run or touches row j-1.  Join
// them bottom-up; the final run touching row j-1 goes to colend for the
// line-of-identity join.
__device__ void merge_cols_body(uint32_t* sh, SeriesDesc* __restrict__ sd) {
  const SeriesDesc& S = sd[blockIdx.y];
  if (S.n <= 0 || !S.hist || S.cross || S.nbands <= 1) return;
  BlockHist h{sh};
  h.init();
  const int64_t n = S.n, H = S.band_h;
  constexpr uint32_t LEN = 0x3FFFFFFFu, WHOLE = 1u << 30;
  for (int64_t j = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t gb = (j - 1) / H;
    if (gb == 0) {  // one band: its first (or only) run is final
      S.colend[j] = S.col_a[j];
      continue;
    }
    const uint32_t zb = S.col_z[gb * n + j];
    bool loi_open;
    uint64_t loi_len, olen = 0;
    uint32_t loi_col, ocol = 0;
    if (zb & WHOLE) {
      loi_open = true;
      loi_len = zb & LEN;
      loi_col = zb >> 31;
    } else {
      loi_open = false;
      const uint32_t ce = S.col_a[gb * n + j];
      loi_len = ce & 0x7FFFFFFFu;
      loi_col = ce >> 31;
      ocol = zb >> 31;
      olen = zb & LEN;
    }
    // the bands' descriptors read MERGE_AHEAD at a time (their addresses
    // follow from g alone, so the loads need not wait on each other), then
    // joined in order
    for (int64_t g0 = gb - 1; g0 >= 0; g0 -= MERGE_AHEAD) {
      uint32_t zs[MERGE_AHEAD], as[MERGE_AHEAD];
#pragma unroll
      for (int v = 0; v < MERGE_AHEAD; ++v) {
        const int64_t gv = g0 - v;
        zs[v] = gv >= 0 ? S.col_z[gv * n + j] : 0u;
        as[v] = gv >= 0 ? S.col_a[gv * n + j] : 0u;
      }
#pragma unroll
      for (int v = 0; v < MERGE_AHEAD; ++v) {
        const int64_t g = g0 - v;
        if (g < 0) break;
        const uint32_t z = zs[v];
        if (z & WHOLE) {
          const uint32_t zc = z >> 31;
          const uint64_t zl = z & LEN;
          if (loi_open) {
            if (loi_col == zc) {
              loi_len += zl;
            } else {
              loi_open = false;
              ocol = zc;
              olen = zl;
            }
          } else if (olen && ocol == zc) {
            olen += zl;
          } else {
            emit2(h, S, ocol, olen);
            ocol = zc;
            olen = zl;
          }
        } else {
          const uint32_t a = as[v];
          const uint32_t ac = a >> 31;
          const uint64_t al = a & 0x7FFFFFFFu;
          if (loi_open) {
            if (loi_col == ac) loi_len += al; else emit2(h, S, ac, al);
            loi_open = false;
          } else if (olen && ocol == ac) {
            emit2(h, S, ocol, olen + al);
          } else {
            emit2(h, S, ocol, olen);
            emit2(h, S, ac, al);
          }
          ocol = z >> 31;
          olen = g > 0 ? (z & LEN) : 0;  // band 0 closed its own top run
        }
      }
    }
    emit2(h, S, ocol, olen);  // the open run touching row 0
    S.colend[j] = (uint32_t)loi_len | (loi_col << 31);
  }
  h.flush(S);
}

// ------------------------------------------------ merge: cross diagonals
// Cross recurrence: diagonal k (cells (i, i+k), -(n1-1) <= k <= n2-1) runs
// from its bottom-right end, (min(n1-1, n2-1-k), ...), to its top-left end
// at row max(0, -k), through items (strip Q, band g): strip Q covers
// columns [n2 - (Q+1) sw, n2 - Q sw), band g rows [g H, (g+1) H) (one band:
// all rows); the diagonal leaves an item at row max(R0, J0 - k).  The
// descriptors mean what they mean for RQA; runs touching the matrix border
// were closed in the tile kernel or are closed here at the diagonal's ends.
__device__ void merge_cross_diags_body(uint32_t* sh, SeriesDesc* __restrict__ sd) {
  const SeriesDesc& S = sd[blockIdx.y];
  if (S.n <= 0 || !S.hist || !S.cross) return;
  BlockHist h{sh};
  h.init();
  const int64_t n1 = S.n, n2 = S.n2, sw = S.sw, nd = cross_strip_diags(n1, sw);
  const bool banded = S.nbands > 1;
  const int64_t H = banded ? S.band_h : n1;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n1 + n2 - 1;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = t - (n1 - 1);
    int64_t i = n1 - 1 < n2 - 1 - k ? n1 - 1 : n2 - 1 - k;  // bottom-right end
    const int64_t itop = k >= 0 ? 0 : -k;                   // top-left end
    uint64_t L = 0;
    for (;;) {
      const int64_t Q = (n2 - 1 - (i + k)) / sw;
      const int64_t J1 = n2 - Q * sw, J0 = J1 - sw;
      const int64_t g = banded ? i / H : 0;
      const int64_t R0 = g * H, R1 = R0 + H < n1 ? R0 + H : n1;
      const int64_t off = banded ? S.dia_off[Q * S.nbands + g] : Q * nd;
      const int64_t o = off + (k - (J0 - (R1 - 1)));
      const uint32_t z = S.dia_z[o];
      if (z & 0x8000u) {
        L += (z & 0x7FFFu);
      } else {
        const uint64_t first = L + S.dia_a[o];
        if (first) h.add(S, HIST_DIAG, first);
        L = z & 0x7FFFu;
      }
      const int64_t ie = R0 > J0 - k ? R0 : J0 - k;
      if (ie <= itop) break;
      i = ie - 1;
    }
    if (L) h.add(S, HIST_DIAG, L);
  }
  h.flush(S);
}

// ------------------------------------------------ merge: cross columns
// Cross recurrence in row bands: column j crosses bands nbands-1 .. 0.  The
// last band closed its first run at the matrix border; every other band
// holds its first run (col_a, touching its bottom edge) unless the column's
// segment there is one run, and every band but 0 its top run (col_z, with a
// whole-segment flag; band 0 records it only when whole).  Join bottom-up.
__device__ void merge_cross_cols_body(uint32_t* sh, SeriesDesc* __restrict__ sd) {
  const SeriesDesc& S = sd[blockIdx.y];
  if (S.n <= 0 || !S.hist || !S.cross || S.nbands <= 1) return;
  BlockHist h{sh};
  h.init();
  const int64_t n2 = S.n2, nb = S.nbands;
  constexpr uint32_t LEN = 0x3FFFFFFFu, WHOLE = 1u << 30;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n2;
       j += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t zl = S.col_z[(nb - 1) * n2 + j];
    uint32_t ocol = zl >> 31;
    uint64_t olen = zl & LEN;
    for (int64_t g0 = nb - 2; g0 >= 0; g0 -= MERGE_AHEAD) {  // eight bands' loads at a time
      uint32_t zs[MERGE_AHEAD], as[MERGE_AHEAD];
#pragma unroll
      for (int v = 0; v < MERGE_AHEAD; ++v) {
        const int64_t gv = g0 - v;
        zs[v] = gv >= 0 ? S.col_z[gv * n2 + j] : 0u;
        as[v] = gv >= 0 ? S.col_a[gv * n2 + j] : 0u;
      }
#pragma unroll
      for (int v = 0; v < MERGE_AHEAD; ++v) {
        const int64_t g = g0 - v;
        if (g < 0) break;
        const uint32_t z = zs[v];
        if (z & WHOLE) {
          if (olen && ocol == (z >> 31)) {
            olen += z & LEN;
          } else {
            emit2(h, S, ocol, olen);
            ocol = z >> 31;
            olen = z & LEN;
          }
        } else {
          const uint32_t a = as[v];
          const uint32_t ac = a >> 31;
          const uint64_t al = a & 0x7FFFFFFFu;
          if (olen && ocol == ac) {
            emit2(h, S, ocol, olen + al);
          } else {
            emit2(h, S, ocol, olen);
            emit2(h, S, ac, al);
          }
          ocol = z >> 31;
          olen = g > 0 ? (z & LEN) : 0;  // band 0 closed its own top run
        }
      }
    }
    emit2(h, S, ocol, olen);
  }
  h.flush(S);
}

// The merges as kernels of their own (strip groups walk rows and diagonals
// group by group), and fused: the walks of one series touch disjoint
// outputs (rowend, colend) and add to the histograms by atomics, so they need
// no order among themselves, and one launch (blockIdx.z: the walk) lets their
// latency-bound loads overlap.
// (Every body takes the block's shared bins from its kernel, so that the
// fused kernels hold one set, not one per walk: the walks are latency-bound
// and need the occupancy.)
__global__ void merge_rows_kernel(SeriesDesc* __restrict__ sd, int64_t q0, int64_t q1) {
  __shared__ uint32_t sh[3 * HB];
  merge_rows_body(sh, sd, q0, q1);
}
__global__ void merge_diags_kernel(SeriesDesc* __restrict__ sd, int64_t q0, int64_t q1) {
  __shared__ uint32_t sh[3 * HB];
  merge_diags_body(sh, sd, q0, q1);
}
__global__ void merge_cols_kernel(SeriesDesc* __restrict__ sd) {
  __shared__ uint32_t sh[3 * HB];
  merge_cols_body(sh, sd);
}
__global__ void merge_cross_diags_kernel(SeriesDesc* __restrict__ sd) {
  __shared__ uint32_t sh[3 * HB];
  merge_cross_diags_body(sh, sd);
}
__global__ void merge_cross_cols_kernel(SeriesDesc* __restrict__ sd) {
  __shared__ uint32_t sh[3 * HB];
  merge_cross_cols_body(sh, sd);
}
// z = 0 rows, 1 diagonals, 2 columns (row bands only)
__global__ void merge_sym_kernel(SeriesDesc* __restrict__ sd) {
  __shared__ uint32_t sh[3 * HB];
  if (blockIdx.z == 0)
    merge_rows_body(sh, sd, 0, -1);
  else if (blockIdx.z == 1)
    merge_diags_body(sh, sd, 0, -1);
  else
    merge_cols_body(sh, sd);
}
// z = 0 diagonals, 1 columns (row bands only)
__global__ void merge_cross_kernel(SeriesDesc* __restrict__ sd) {
  __shared__ uint32_t sh[3 * HB];
  if (blockIdx.z == 0)
    merge_cross_diags_body(sh, sd);
  else
    merge_cross_cols_body(sh, sd);
}

// ----------------------------------------------------------------- finalize
// Full column j = upper column j (rows < j), the line-of-identity cell, and
// upper row j (by symmetry).  The cell (j, j) is black iff w = 0.
__global__ void join_loi_kernel(SeriesDesc* __restrict__ sd) {
  const SeriesDesc& S = sd[blockIdx.y];
  if (S.n <= 0 || !S.hist || S.cross) return;
  __shared__ uint32_t sh[3 * HB];
  BlockHist h{sh};
  h.init();
  const uint32_t cd = S.w == 0 ? 1u : 0u;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < S.n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t up = S.colend[j], rt = S.rowend[j];
    uint64_t L = 1;
    const uint32_t ulen = up & 0x7FFFFFFFu, ucol = up >> 31;
    const uint32_t rlen = rt & 0x7FFFFFFFu, rcol = rt >> 31;
    if (ulen) {
      if (ucol == cd) L += ulen; else emit2(h, S, ucol, ulen);
    }
    if (rlen) {
      if (rcol == cd) L += rlen; else emit2(h, S, rcol, rlen);
    }
    emit2(h, S, cd, L);
  }
  h.flush(S);
}

// Full diagonal histogram: both triangles (symmetric) plus the line of
// identity, one line of length n when w = 0.
__global__ void diag_full_kernel(SeriesDesc* __restrict__ sd) {
  const SeriesDesc& S = sd[blockIdx.y];
  if (S.n <= 0 || !S.hist || S.cross) return;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l <= S.n;
       l += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long v = 2ull * S.hist[HIST_DIAG * (S.n + 1) + l];
    if (S.w == 0 && l == S.n) v += 1ull;
    S.hist[HIST_DIAG * (S.n + 1) + l] = v;
  }
}

// ------------------------------------------------------------------ sample
// R_ij with the tile kernel's decision code: row vector i (of s), column
// vector j (of s2 for cross recurrence; RQA takes the pair as i < j).
template <int NORM>
__device__ bool sample_one(const SeriesDesc& S, int64_t i, int64_t j, bool f64) {
  if (!S.cross && i > j) {
    const int64_t t = i;
    i = j;
    j = t;
  }
  if ((i > j ? i - j : j - i) < S.w) return false;
  const double* s2 = S.cross ? S.s2 : S.s;
  const float* xe2 = S.cross ? S.xe2 : S.xe;
  if (f64) return exact_decision2<NORM>(S.s, s2, i, j, S.m, S.tau, S.eps);
  // FP32 margin in the tile kernel's order (row vector i, column vector j)
  float acc;
  if (NORM == 1) {
    acc = S.thr;
    for (int k = 0; k < S.m; ++k) {
      const float d = __fsub_rn(S.xe[i * S.mp + k], xe2[j * S.mp + k]);
      acc = __fmaf_rn(-d, d, acc);
    }
  } else if (NORM == 2) {
    acc = S.thr;
    for (int k = 0; k < S.m; ++k)
      acc = __fsub_rn(acc, fabsf(__fsub_rn(S.xe[i * S.mp + k], xe2[j * S.mp + k])));
  } else {
    float mx = 0.f;
    for (int k = 0; k < S.m; ++k)
      mx = fmaxf(mx, fabsf(__fsub_rn(S.xe[i * S.mp + k], xe2[j * S.mp + k])));
    acc = __fsub_rn(S.thr, mx);
  }
  if (fabsf(acc) <= S.band) return exact_decision2<NORM>(S.s, s2, i, j, S.m, S.tau, S.eps);
  return !(__float_as_uint(acc) >> 31);
}

__global__ void sample_kernel(const SeriesDesc* __restrict__ sd, const int64_t* __restrict__ ii,
                              const int64_t* __restrict__ jj, int64_t count, uint8_t* out,
                              int f64) {
  const SeriesDesc& S = sd[0];
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < count;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = ii[q], j = jj[q];
    bool r = false;
    if (i >= 0 && j >= 0 && i < S.n && j < S.n2) {
      if (S.norm == 1) r = sample_one<1>(S, i, j, f64);
      else if (S.norm == 2) r = sample_one<2>(S, i, j, f64);
      else r = sample_one<0>(S, i, j, f64);
    }
    out[q] = r ? 1 : 0;
  }
}

// -------------------------------------------------------- recurrence plot
// One thread per 32-bit word of the bit-packed plot: word w of plot row r
// holds R(i0 + r, j0 + 32 w + b) in bit b (0 outside the matrix).
__global__ void plot_kernel(const SeriesDesc* __restrict__ sd, int64_t i0, int64_t j0,
                            int64_t rows, int64_t cols, uint32_t* __restrict__ out, int f64) {
  const SeriesDesc& S = sd[0];
  const int64_t wpr = (cols + 31) / 32;
  const int64_t total = rows * wpr;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = q / wpr, w = q - r * wpr;
    const int64_t i = i0 + r;
    uint32_t word = 0;
    for (int b = 0; b < 32; ++b) {
      const int64_t c = w * 32 + b, j = j0 + c;
      if (c >= cols || i < 0 || j < 0 || i >= S.n || j >= S.n2) continue;
      bool rr;
      if (S.norm == 1) rr = sample_one<1>(S, i, j, f64);
      else if (S.norm == 2) rr = sample_one<2>(S, i, j, f64);
      else rr = sample_one<0>(S, i, j, f64);
      word |= (rr ? 1u : 0u) << b;
    }
    out[q] = word;
  }
}

// Bits [0, k) set, k clamped to [0, 32].
__device__ __forceinline__ uint32_t lowmask64(int64_t k) {
  return k <= 0 ? 0u : k >= 32 ? FULL : ((1u << k) - 1u);
}

// The FP32 path of the plot, one warp per 32 x 32 tile of the window: lane l
// holds column j0 + 32 w + l's vector, row t's vector is broadcast from lane
// t, the margins (in sample_one()'s operation order, so the recheck band
// holds) give one column word per lane, pairs inside the band are re-decided
// in FP64, and a warp transpose turns the column words into the plot's row
// words (lane t writes row t's word w).
template <int M, int NORM>
__global__ void plot_tile_kernel(const SeriesDesc* __restrict__ sd, int64_t i0, int64_t j0,
                                 int64_t rows, int64_t cols, uint32_t* __restrict__ out) {
  const SeriesDesc& S = sd[0];
  const int lane = threadIdx.x & 31;
  const int64_t wpr = (cols + 31) / 32, tr = (rows + 31) / 32;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float* xe2 = S.cross ? S.xe2 : S.xe;
  const double* s2 = S.cross ? S.s2 : S.s;
  for (int64_t tile = warp0; tile < tr * wpr; tile += nwarps) {
    const int64_t rb = (tile / wpr) * 32, w = tile % wpr;
    const int64_t j = j0 + w * 32 + lane;       // this lane's column
    const int64_t ir = i0 + rb + lane;          // the row this lane broadcasts
    const bool jok = w * 32 + lane < cols && j >= 0 && j < S.n2;
    const bool iok = rb + lane < rows && ir >= 0 && ir < S.n;
    float xc[M], xr[M];
#pragma unroll
    for (int k = 0; k < M; ++k) {
      xc[k] = jok ? xe2[j * S.mp + k] : 0.f;
      xr[k] = iok ? S.xe[ir * S.mp + k] : 0.f;
    }
    uint32_t word = 0, near = 0;
#pragma unroll 4
    for (int t = 0; t < 32; ++t) {
      float acc;
      if (NORM == 1) {
        acc = S.thr;
#pragma unroll
        for (int k = 0; k < M; ++k) {
          const float d = __fsub_rn(__shfl_sync(FULL, xr[k], t), xc[k]);
          acc = __fmaf_rn(-d, d, acc);
        }
      } else if (NORM == 2) {
        acc = S.thr;
#pragma unroll
        for (int k = 0; k < M; ++k)
          acc = __fsub_rn(acc, fabsf(__fsub_rn(__shfl_sync(FULL, xr[k], t), xc[k])));
      } else {
        float mx = 0.f;
#pragma unroll
        for (int k = 0; k < M; ++k)
          mx = fmaxf(mx, fabsf(__fsub_rn(__shfl_sync(FULL, xr[k], t), xc[k])));
        acc = __fsub_rn(S.thr, mx);
      }
      word |= (uint32_t)(!(__float_as_uint(acc) >> 31)) << t;
      near |= (uint32_t)(fabsf(acc) <= S.band) << t;
    }
    // rows outside the window or the matrix, and the Theiler window: the rows
    // i = base + t with |i - j| < w are t in [j - w + 1 - base, j + w - base)
    const int64_t base = i0 + rb;
    const int64_t rlim = rows - rb < S.n - base ? rows - rb : S.n - base;
    uint32_t live = jok ? lowmask64(rlim) : 0u;
    if (S.w > 0) live &= ~(lowmask64(j + S.w - base) & ~lowmask64(j - S.w + 1 - base));
    word &= live;
    near &= live;
    while (near) {  // rare: re-decide in FP64 with the definition's order
      const int t = __ffs(near) - 1;
      near &= near - 1;
      const bool r = exact_decision2<NORM>(S.s, s2, i0 + rb + t, j, M, S.tau, S.eps);
      word = r ? (word | (1u << t)) : (word & ~(1u << t));
    }
    const uint32_t rw = transpose32(word, lane);  // lane t: row rb + t, bit l = column l
    if (rb + lane < rows) out[(rb + lane) * wpr + w] = rw;
  }
}

template <int NORM>
static void launch_plot_tile(int m, const SeriesDesc* d_sd, int64_t i0, int64_t j0,
                             int64_t rows, int64_t cols, uint32_t* out, unsigned blocks,
                             cudaStream_t st) {
  switch (m) {
#define RQA_PLOT_CASE(MM) \
  case MM: plot_tile_kernel<MM, NORM><<<blocks, 256, 0, st>>>(d_sd, i0, j0, rows, cols, out); break;
    RQA_PLOT_CASE(1) RQA_PLOT_CASE(2) RQA_PLOT_CASE(3) RQA_PLOT_CASE(4) RQA_PLOT_CASE(5)
    RQA_PLOT_CASE(6) RQA_PLOT_CASE(7) RQA_PLOT_CASE(8) RQA_PLOT_CASE(9) RQA_PLOT_CASE(10)
#undef RQA_PLOT_CASE
    default: break;
  }
}

void launch_plot(const SeriesDesc* d_sd, int64_t i0, int64_t j0, int64_t rows, int64_t cols,
                 uint32_t* out, int f64, int m, int norm, int sms, cudaStream_t st) {
  if (!f64) {  // one warp per 32 x 32 tile
    const int64_t tiles = ((rows + 31) / 32) * ((cols + 31) / 32);
    int64_t blocks = (tiles + 7) / 8;
    if (blocks > 16 * (int64_t)sms) blocks = 16 * (int64_t)sms;
    if (blocks < 1) blocks = 1;
    if (norm == 1)
      launch_plot_tile<1>(m, d_sd, i0, j0, rows, cols, out, (unsigned)blocks, st);
    else if (norm == 2)
      launch_plot_tile<2>(m, d_sd, i0, j0, rows, cols, out, (unsigned)blocks, st);
    else
      launch_plot_tile<0>(m, d_sd, i0, j0, rows, cols, out, (unsigned)blocks, st);
    return;
  }
  const int64_t total = rows * ((cols + 31) / 32);
  int64_t blocks = (total + 255) / 256;
  if (blocks > 16 * (int64_t)sms) blocks = 16 * (int64_t)sms;
  if (blocks < 1) blocks = 1;
  plot_kernel<<<(unsigned)blocks, 256, 0, st>>>(d_sd, i0, j0, rows, cols, out, f64);
}

// ------------------------------------------------------ bounded-wait test
// Failure detection without a fault: warp 1 waits, with the tile kernel's
// own bounded spin, for a counter that warp 0 never raises.  The wait must
// give up after SPIN_CYCLES, raise the abort flag and report RQA_ETIMEOUT
// (status[0]) with the cycles it waited (status[1]); the context stays usable.
__global__ void wait_selftest_kernel(unsigned long long* status) {
  __shared__ volatile int ctr;
  __shared__ volatile int abort_flag;
  if (threadIdx.x == 0) {
    ctr = 0;
    abort_flag = 0;
  }
  __syncthreads();
  if (threadIdx.x == 32) {
    const long long t0 = clock64();
    const bool ok = spin_until_ge(&ctr, 1, &abort_flag);
    status[0] = ok ? 0ull : 6ull /* RQA_ETIMEOUT */;
    status[1] = (unsigned long long)(clock64() - t0);
    status[2] = abort_flag ? 1ull : 0ull;
  }
}

void launch_wait_selftest(unsigned long long* status, cudaStream_t st) {
  wait_selftest_kernel<<<1, 64, 0, st>>>(status);
}

// ------------------------------------------------------------ host launch
void launch_prepare(SeriesDesc* d_sd, int count, int64_t max_len, int sms, cudaStream_t st) {
  int64_t blocks = (max_len + 8191) / 8192;  // 32 values per thread
  if (blocks > 4 * sms) blocks = 4 * sms;
  if (blocks < 1) blocks = 1;
  prepare_scan_kernel<<<dim3((unsigned)blocks, count), 256, 0, st>>>(d_sd);
  prepare_kernel<<<(count + 127) / 128, 128, 0, st>>>(d_sd, count);
}
void launch_embed(SeriesDesc* d_sd, int count, int64_t max_n_mp, int sms, cudaStream_t st) {
  int64_t blocks = (max_n_mp + 255) / 256;
  if (blocks > 8 * sms) blocks = 8 * sms;
  if (blocks < 1) blocks = 1;
  embed_kernel<<<dim3((unsigned)blocks, count), 256, 0, st>>>(d_sd);
}
// Longest length with a non-zero count in histogram blockIdx.z of series
// blockIdx.y (0 if the histogram is empty), into counters[CNT_LAST + z]:
// each block takes a grid-stride share of the bins and one atomic max.
__global__ void last_bin_kernel(SeriesDesc* sd) {
  SeriesDesc& S = sd[blockIdx.y];
  const int64_t hl = S.hl;
  const unsigned long long* __restrict__ h = S.hist + (int64_t)blockIdx.z * (hl + 1);
  unsigned long long best = 0;
  for (int64_t l = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l <= hl;
       l += (int64_t)gridDim.x * blockDim.x)
    if (h[l]) best = (unsigned long long)l;
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
    best = v > best ? v : best;
  }
  if ((threadIdx.x & 31) == 0 && best) atomicMax(&S.counters[CNT_LAST + blockIdx.z], best);
}

int preload_aux_kernels() {
  const void* fns[] = {
      reinterpret_cast<const void*>(prepare_scan_kernel),
      reinterpret_cast<const void*>(prepare_kernel),
      reinterpret_cast<const void*>(embed_kernel),
      reinterpret_cast<const void*>(merge_rows_kernel),
      reinterpret_cast<const void*>(merge_diags_kernel),
      reinterpret_cast<const void*>(merge_cols_kernel),
      reinterpret_cast<const void*>(merge_cross_diags_kernel),
      reinterpret_cast<const void*>(merge_cross_cols_kernel),
      reinterpret_cast<const void*>(merge_sym_kernel),
      reinterpret_cast<const void*>(merge_cross_kernel),
      reinterpret_cast<const void*>(join_loi_kernel),
      reinterpret_cast<const void*>(diag_full_kernel),
      reinterpret_cast<const void*>(last_bin_kernel),
  };
  cudaFuncAttributes a;
  for (const void* f : fns)
    if (cudaFuncGetAttributes(&a, f) != cudaSuccess) return -1;
  return static_cast<int>(sizeof(fns) / sizeof(fns[0]));
}

int launch_group_merges(SeriesDesc* d_sd, int64_t n, int64_t q0, int64_t q1, int sms,
                        cudaStream_t st) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4 * sms) blocks = 4 * sms;
  if (blocks < 1) blocks = 1;
  merge_rows_kernel<<<dim3((unsigned)blocks, 1), 256, 0, st>>>(d_sd, q0, q1);
  merge_diags_kernel<<<dim3((unsigned)blocks, 1), 256, 0, st>>>(d_sd, q0, q1);
  return 2;
}

int launch_merges(SeriesDesc* d_sd, int count, int64_t max_n, bool sym, bool cross, bool bands,
                  int sms, cudaStream_t st, bool grouped) {
  int64_t blocks = (max_n + 255) / 256;
  if (blocks > 4 * sms) blocks = 4 * sms;
  if (blocks < 1) blocks = 1;
  int launched = 0;
  // Small sets: rows, diagonals and (bands) columns in one launch, their
  // latency-bound walks overlapping (2,000 points: 0.134 -> 0.112 ms per
  // run).  Separate launches from 2^17 vectors on (1M points: 4.5 against
  // 6.1 ms, the concurrent walks over gigabytes of descriptors in each
  // other's way) and for sets of many series (the 4,096-series batch: 309
  // against 314 ms of device time).
  const bool fuse = max_n <= (int64_t(1) << 17) && count <= 8;
  if (sym && !grouped && fuse) {
    merge_sym_kernel<<<dim3((unsigned)blocks, count, bands ? 3 : 2), 256, 0, st>>>(d_sd);
    ++launched;
  } else {
    if (sym && !grouped) {
      merge_rows_kernel<<<dim3((unsigned)blocks, count), 256, 0, st>>>(d_sd, 0, -1);
      merge_diags_kernel<<<dim3((unsigned)blocks, count), 256, 0, st>>>(d_sd, 0, -1);
      launched += 2;
    }
    if (sym && bands) {  // (strip groups merged their rows and diagonals already)
      merge_cols_kernel<<<dim3((unsigned)blocks, count), 256, 0, st>>>(d_sd);
      ++launched;
    }
  }
  if (sym) {
    join_loi_kernel<<<dim3((unsigned)blocks, count), 256, 0, st>>>(d_sd);
    diag_full_kernel<<<dim3((unsigned)blocks, count), 256, 0, st>>>(d_sd);
    launched += 2;
  }
  if (cross && fuse) {  // diagonals and (bands) columns in one launch
    merge_cross_kernel<<<dim3((unsigned)blocks, count, bands ? 2 : 1), 256, 0, st>>>(d_sd);
    ++launched;
  } else if (cross) {
    merge_cross_diags_kernel<<<dim3((unsigned)blocks, count), 256, 0, st>>>(d_sd);
    ++launched;
    if (bands) {
      merge_cross_cols_kernel<<<dim3((unsigned)blocks, count), 256, 0, st>>>(d_sd);
      ++launched;
    }
  }
  // after every histogram update: the last non-zero bins (the merges above
  // add the lines that cross strip borders)
  int64_t lb_blocks = (max_n + 4095) / 4096;  // about 16 bins per thread
  if (lb_blocks > blocks) lb_blocks = blocks;
  if (lb_blocks < 1) lb_blocks = 1;
  last_bin_kernel<<<dim3((unsigned)lb_blocks, count, 3), 256, 0, st>>>(d_sd);
  return launched + 1;
}
void launch_sample(const SeriesDesc* d_sd, const int64_t* ii, const int64_t* jj, int64_t count,
                   uint8_t* out, int f64, cudaStream_t st) {
  int64_t blocks = (count + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  sample_kernel<<<(unsigned)blocks, 256, 0, st>>>(d_sd, ii, jj, count, out, f64);
}

}  // namespace rqa
