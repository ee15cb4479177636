// rqa_tile.cuh -- the fused RQA tile kernel for sm_103a.
//
// One persistent CTA processes one CTA strip at a time: SW = warps * 32 * C
// consecutive columns of the upper triangle of the recurrence matrix (the
// matrix is symmetric, Sect. 4.2 notes the halved degree of parallelism of
// operator II for it).  Strips are taken from a work queue, longest first.
// Inside a strip, warp w owns 32*C columns (lane l owns columns col0 + l of
// C sub-blocks) and walks its rows bottom-up in blocks of 32.
//
// Per 32 x 32 sub-block the warp fuses the paper's three operators
// (Sect. 4.2):
//   I   create_recurrence_matrix -> FP32 distance margin per pair, the
//       decision taken from its sign bit and packed by a funnel shift into
//       one 32-bit column word per lane; pairs inside the proven FP32 error
//       band are re-decided in FP64;
//   II  detect_diagonal_lines     -> diagonal words from a bit reverse, a
//       rotate and a 32x32 transpose of the column words, scanned for runs;
//   III detect_vertical_lines     -> the column words (upper part of full
//       column j) and the transposed row words (the part of full column i
//       below the line of identity, by symmetry), scanned for black and
//       white runs.
// Lines that cross sub-block borders are carried in per-warp shared state
// (down a column, along a diagonal) or passed to the next warp through a
// shared-memory ring (rows and diagonals leaving the warp to the left).  Runs
// that touch the strip's own left or right edge are not counted here: their
// lengths go to boundary descriptors that the merge kernels join across
// strips (the carryover buffers of Sect. 4.1).  The run of each full column
// that touches the line of identity is stored apart and joined by the
// finalize kernel.  Counts go to shared-memory histograms flushed once per
// strip.
//
// Template flags select the variants built from this one body:
//   XR  cross recurrence (Sect. 3.3): rows from one series, columns from
//       another, every strip spans all rows, no row scans and no
//       line-of-identity join, a two-sided Theiler window;
//   MX  a precomputed matrix (Sect. 9): the recurrence words are read from
//       the caller's bits instead of computed (with XR);
//   BD  row bands: a work item is (strip, band of rows), so series whose
//       strips alone cannot fill the GPU still do; column runs and diagonals
//       that cross a band edge get their own descriptors.  A separate
//       instantiation, so the unbanded kernel keeps its registers.
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
// The test instantiation's limit (~0.5 ms): its test withholds a hand-over
// on purpose, so the wait must give up quickly; far above a block's time.
constexpr long long TEST_SPIN_CYCLES = 1000000LL;

// Run state words.  Two-colour state (rows, columns): length in bits 0..27,
// colour in bit 28, flag in bit 29 (the run touches the strip's right edge
// for rows, it is the column's first run for columns), done in bit 30.
// Diagonal state: black length in bits 0..27, edge flag in bit 28.
constexpr uint32_t ST_LEN = 0x0FFFFFFFu;
constexpr uint32_t ST_COLOUR = 1u << 28;
constexpr uint32_t ST_FLAG = 1u << 29;
constexpr uint32_t ST_DONE = 1u << 30;
constexpr uint32_t DG_EDGE = 1u << 28;

// Status word value for an internal inconsistency (a line length outside
// 1..n); the entry point reports it as RQA_ECUDA.
constexpr unsigned long long STATUS_INTERNAL = 5ull;

// Bits [0, k) set, k clamped to [0, 32] (one BMSK instruction).
__device__ __forceinline__ uint32_t lowmask(int k) {
  uint32_t r;
  asm("bmsk.clamp.b32 %0, %1, %2;" : "=r"(r) : "r"(0), "r"(k < 0 ? 0 : k));
  return r;
}

__device__ __forceinline__ int clamp32(int v) { return v < 0 ? 0 : (v > 32 ? 32 : v); }

// Position of the highest set bit (x != 0).
__device__ __forceinline__ int msb(uint32_t x) { return 31 - __clz(x); }

// Position of the lowest set bit (x != 0): the highest set bit of the
// isolated lowest bit, one bfind instead of a bit reverse and a find.
__device__ __forceinline__ uint32_t lowbit_index(uint32_t x) {
  uint32_t r;
  asm("bfind.u32 %0, %1;" : "=r"(r) : "r"(x & (0u - x)));
  return r;
}

// 32 x 32 bit transpose across a warp: lane r holds row r (bit c = A[r][c]);
// on return lane c holds bit r = A[r][c].  Five stages; each swaps the
// off-diagonal j x j blocks of every 2j x 2j block with one shuffle and, for
// j = 16 and 8, one byte permute, else one rotate and one three-input logic
// operation.
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
#pragma unroll
  for (int j = 16; j >= 1; j >>= 1) {
    const uint32_t m = j == 16 ? 0x0000FFFFu
                     : j == 8  ? 0x00FF00FFu
                     : j == 4  ? 0x0F0F0F0Fu
                     : j == 2  ? 0x33333333u
                               : 0x55555555u;
    const bool hi = (lane & j) != 0;
    const uint32_t keep = hi ? ~m : m;
    const uint32_t y = __shfl_xor_sync(FULL, x, j);
    if (j >= 8) {  // whole bytes move: one byte permute of x and y
      x = __byte_perm(x, y, j == 16 ? (hi ? 0x3276u : 0x5410u) : (hi ? 0x3715u : 0x6240u));
    } else {
      const uint32_t rot = __funnelshift_l(y, y, hi ? 32 - j : j);
      x = (x & keep) | (rot & ~keep);
    }
  }
  return x;
}

// Two independent transposes with their stages interleaved, so the shuffle
// latencies of the two chains overlap.
__device__ __forceinline__ void transpose32x2(uint32_t& x, uint32_t& z, int lane) {
#pragma unroll
  for (int j = 16; j >= 1; j >>= 1) {
    const uint32_t m = j == 16 ? 0x0000FFFFu
                     : j == 8  ? 0x00FF00FFu
                     : j == 4  ? 0x0F0F0F0Fu
                     : j == 2  ? 0x33333333u
                               : 0x55555555u;
    const bool hi = (lane & j) != 0;
    const uint32_t keep = hi ? ~m : m;
    const uint32_t y = __shfl_xor_sync(FULL, x, j);
    const uint32_t w = __shfl_xor_sync(FULL, z, j);
    if (j >= 8) {
      const uint32_t sel = j == 16 ? (hi ? 0x3276u : 0x5410u) : (hi ? 0x3715u : 0x6240u);
      x = __byte_perm(x, y, sel);
      z = __byte_perm(z, w, sel);
    } else {
      const uint32_t ry = __funnelshift_l(y, y, hi ? 32 - j : j);
      const uint32_t rw = __funnelshift_l(w, w, hi ? 32 - j : j);
      x = (x & keep) | (ry & ~keep);
      z = (z & keep) | (rw & ~keep);
    }
  }
}

// Histogram sink: shared-memory bins for short lines; longer ones (and any
// length outside 1..HB-1) go to a per-warp queue in shared memory, q[0] the
// count and q[1..OVF] the entries (type << 30 | length), which drain() moves
// to the global histograms.  The hot path thus holds no call and no 64-bit
// address arithmetic.  A warp adds at most three queued lengths per lane
// between two drains (one per scan of a sub-block; lengths <= RQA_MAX_N <
// 2^28), so 96 < OVF entries; a count above OVF is still caught by drain()
// and reported, never written.  A length outside 1..n is never counted; it
// marks the series as failed instead.
constexpr int OVF = 128;
// Values of the current item that the hot loop uses rarely or once per row
// block (descriptor pointers, the global histograms, the radius and band,
// the recheck's FP64 inputs): one copy per CTA in shared memory, read at
// each use with a volatile load so that the compiler keeps none of them in
// registers across the loop.  At three CTAs per SM (80 registers a thread)
// this leaves registers to the scans and the distance loop: 2.5 % faster on
// the 1M-point L2 series than holding them in registers.
struct StripCtx {
  unsigned long long* gl;      // [3][nh+1]
  unsigned long long* status;
  uint32_t* colfirst;
  uint16_t* rowA;              // row_a + the strip's row offset
  uint16_t* rowZ;
  uint16_t* dia_a;
  uint16_t* dia_z;
  int64_t dbase;               // descriptor of diagonal k: dbase + k (k >= klo)
  const float* xe;
  const double* sser;
  const double* sser2;         // cross recurrence: the column series
  double eps;
  float thr, band;
  int tau;
  uint32_t nh;
  int klo;
  int mp;
  const SeriesDesc* sp;
};
template <class V>
__device__ __forceinline__ V ldv(const V& r) { return *reinterpret_cast<const volatile V*>(&r); }
struct HistSink {
  uint32_t* sh;              // [3][HB]
  const StripCtx* cx;
  uint32_t* q;               // this warp's queue: [1 + OVF]
  __device__ __forceinline__ void add(int type, uint32_t len) const {
    if (len - 1u < (uint32_t)(HB - 1)) {
      atomicAdd(&sh[type * HB + len], 1u);
    } else {
      const uint32_t k = atomicAdd(q, 1u);
      if (k < (uint32_t)OVF) q[1 + k] = ((uint32_t)type << 30) | len;
    }
  }
  // Warp-collective: move the queued lengths to the global histograms.
  __device__ __forceinline__ void drain(int lane) const {
    __syncwarp();
    const uint32_t cnt = *reinterpret_cast<volatile uint32_t*>(q);
    if (cnt == 0) return;  // the same value in every lane
    const uint32_t m = cnt < (uint32_t)OVF ? cnt : (uint32_t)OVF;
    unsigned long long* const gl = ldv(cx->gl);
    unsigned long long* const status = ldv(cx->status);
    const uint32_t n = ldv(cx->nh);
    for (uint32_t k = lane; k < m; k += 32) {
      const uint32_t v = q[1 + k], type = v >> 30, len = v & 0x3FFFFFFFu;
      if (len > 0 && len <= n)
        atomicAdd(&gl[(size_t)type * (n + 1) + len], 1ull);
      else
        atomicCAS(status, 0ull, STATUS_INTERNAL);  // the first error stays
    }
    if (cnt > (uint32_t)OVF && lane == 0) atomicCAS(status, 0ull, STATUS_INTERNAL);
    __syncwarp();
    if (lane == 0) *q = 0;
    __syncwarp();
  }
  // vertical (black, colour 1) or white vertical (colour 0)
  __device__ __forceinline__ void add2(uint32_t colour, uint32_t len) const {
    add(colour ? HIST_VERT : HIST_WHITE, len);
  }
  // A run that lies inside one full 32-bit word of valid cells: 1 <= len <=
  // 30 <= n, so its shared bin always exists and no range check is needed.
  __device__ __forceinline__ void add_in(int type, uint32_t len) const {
    atomicAdd(&sh[type * HB + len], 1u);
  }
};

// Scan the two-colour cells hi..lo (descending bit index) of x, continuing
// run state st.  first(colour, len) receives the first run that ends here if
// st carries the flag, emit(colour, len) every other run that ends here; the
// run left open at lo is returned.  Interior runs (cells hi..lo are valid)
// go straight to the shared bins.
template <class E, class F>
__device__ __forceinline__ uint32_t scan2(uint32_t x, int hi, int lo, uint32_t st,
                                          const HistSink& hs, E&& emit, F&& first) {
  uint32_t cl = st & ST_LEN;
  const uint32_t cc = (st >> 28) & 1u;
  uint32_t fl = (st >> 29) & 1u;
  uint32_t col = (x >> hi) & 1u;
  if (cl != 0 && cc != col) {  // the carried run ends before cell hi
    if (fl) first(cc, cl); else emit(cc, cl);
    fl = 0;
    cl = 0;
  }
  uint32_t T = (x ^ (x << 1)) & lowmask(hi + 1) & ~lowmask(lo + 1);
  int top = hi;
  if (T) {
    int p = msb(T);
    const uint32_t len = cl + (uint32_t)(top - p + 1);
    if (fl) first(col, len); else emit(col, len);
    fl = 0;
    cl = 0;
    col ^= 1u;
    top = p - 1;
    T ^= 1u << p;
    while (T) {
      p = msb(T);
      hs.add_in(col ? HIST_VERT : HIST_WHITE, (uint32_t)(top - p + 1));
      col ^= 1u;
      top = p - 1;
      T ^= 1u << p;
    }
  }
  return (cl + (uint32_t)(top - lo + 1)) | (col << 28) | (fl << 29);
}

// Lines of length 1..3 are counted without emitting them one by one: 16-bit
// fields packed two per register, added to the histograms every
// FLUSH_BLOCKS blocks.  The two-colour fields count black runs and runs of
// both colours (white = both - black at the flush): a 32-cell word holds at
// most 30 interior runs of one length, a block at most 8 two-colour words,
// so a field gains at most 240 per block and 61,440 < 2^16 between flushes.
struct ShortCounts {
  uint32_t v12;   // vertical black: length 1 | length 2 << 16
  uint32_t v3w1;  // vertical black length 3 | both colours length 1 << 16
  uint32_t w23;   // both colours: length 2 | length 3 << 16
  uint32_t d12;   // diagonal: length 1 | length 2 << 16
  uint32_t d3;    // diagonal: length 3
};
constexpr int FLUSH_BLOCKS = 256;

// Two-colour scan of a full word (cells 31 .. 0 in scan order), same
// contract as scan2(x, 31, 0, ...).  Runs that touch neither cell 31 nor
// cell 0 are interior: with T the transition mask, an interior run starts
// (lowest cell q) at every transition below the topmost one and its length
// is the distance to the next transition above q, so the interior runs of
// length 1, 2 and 3 are popcounts of T against T shifted by 1, 2 and 3.
// Only longer interior runs and the two runs touching the word's ends are
// passed to emit / first individually.
template <class E, class F>
__device__ __forceinline__ uint32_t scan2_full(uint32_t x, uint32_t st, ShortCounts& sc,
                                               const HistSink& hs, E&& emit, F&& first) {
  const uint32_t T = (x ^ (x << 1)) & 0xFFFFFFFEu;
  uint32_t cl = st & ST_LEN;
  const uint32_t cc = (st >> 28) & 1u;
  uint32_t fl = (st >> 29) & 1u;
  const uint32_t ctop = x >> 31;
  if (cl != 0 && cc != ctop) {
    if (fl) first(cc, cl); else emit(cc, cl);
    fl = 0;
    cl = 0;
  }
  if (T == 0) return (cl + 32u) | (ctop << 28) | (fl << 29);
  const int ptop = msb(T);
  const uint32_t toplen = cl + (uint32_t)(32 - ptop);
  if (fl) first(ctop, toplen); else emit(ctop, toplen);
  {  // unconditional: with no interior run every count below is zero
    // interior runs start (lowest cell) at every transition but the top
    // one, which the masks below never select (no transition lies above it)
    const uint32_t t1 = T >> 1, t2 = T >> 2, t3 = T >> 3;
    const uint32_t l1 = T & t1;
    const uint32_t l2 = T & t2 & ~t1;
    const uint32_t l3 = T & t3 & ~(t1 | t2);
    sc.v12 += __popc(l1 & x) + (__popc(l2 & x) << 16);
    sc.v3w1 += __popc(l3 & x) + (__popc(l1) << 16);
    sc.w23 += __popc(l2) + (__popc(l3) << 16);
    uint32_t lg = T & ~(t1 | t2 | t3);  // and the top transition, never taken
    while (lg & (lg - 1u)) {
      // lowest cell q of a run of length >= 4 whose upper end is a transition
      // below bit 32: in the word of the run's colour as ones, adding 2^q
      // carries through the run and stops at that transition, so the bits
      // that change are the run plus one
      const uint32_t bq = lg & (0u - lg);
      lg ^= bq;
      const bool black = (x & bq) != 0u;
      const uint32_t y = black ? x : ~x;
      hs.add_in(black ? HIST_VERT : HIST_WHITE, (uint32_t)__popc((y + bq) ^ y) - 1u);
    }
  }
  return lowbit_index(T) | ((x & 1u) << 28);
}

// Black-run scan of a full word (cells 31 .. 0), continuing diagonal state
// st.  first(len) receives the run that touches the strip's edge when it
// ends (len may be 0), emit(len) every other run that ends at the word's
// top; interior runs of length 1..3 are counted by popcounts as in
// scan2_full, longer ones go straight to the shared bins.  The black run
// left open at cell 0 is returned.  A segment of a word (cells hi..lo) is
// scanned as a full word whose cells outside the segment are black: they
// extend only the run left open at the bottom, whose length the caller
// shortens by their number (the cells below the segment; those above it are
// moved out by a shift first).
template <class E, class F>
__device__ __forceinline__ uint32_t scanb_full(uint32_t x, uint32_t st, ShortCounts& sc,
                                               const HistSink& hs, E&& emit, F&& first) {
  const uint32_t cl = st & ST_LEN;
  if (x == FULL) return (cl + 32u) | (st & DG_EDGE);
  const int zt = msb(~x);  // highest white cell
  const uint32_t f = cl + (uint32_t)(31 - zt);
  if (st & DG_EDGE)
    first(f);
  else if (f)
    emit(f);
  const uint32_t T = (x ^ (x << 1)) & 0xFFFFFFFEu;
  const uint32_t Sb = T & x & lowmask(zt);  // lowest cells of interior black runs
  {  // unconditional, as in scan2_full
    const uint32_t t1 = T >> 1, t2 = T >> 2, t3 = T >> 3;
    sc.d12 += __popc(Sb & t1) + (__popc(Sb & t2 & ~t1) << 16);
    sc.d3 += __popc(Sb & t3 & ~(t1 | t2));
    uint32_t lg = Sb & ~(t1 | t2 | t3);
    while (lg) {  // as in scan2_full: the carry from bit q runs through the black run
      const uint32_t bq = lg & (0u - lg);
      lg ^= bq;
      hs.add_in(HIST_DIAG, (uint32_t)__popc((x + bq) ^ x) - 1u);
    }
  }
  return lowbit_index(~x);
}

// Add a warp's short-line counters to the CTA's shared bins and clear them.
__device__ __forceinline__ void flush_one(uint32_t x, uint32_t* dst, int lane) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
  if (lane == 0 && x) atomicAdd(dst, x);
}
__device__ __forceinline__ void flush_short(ShortCounts& sc, uint32_t* sh_hist, int lane) {
  flush_one(sc.v12 & 0xFFFFu, sh_hist + HIST_VERT * HB + 1, lane);
  flush_one(sc.v12 >> 16, sh_hist + HIST_VERT * HB + 2, lane);
  flush_one(sc.v3w1 & 0xFFFFu, sh_hist + HIST_VERT * HB + 3, lane);
  flush_one((sc.v3w1 >> 16) - (sc.v12 & 0xFFFFu), sh_hist + HIST_WHITE * HB + 1, lane);
  flush_one((sc.w23 & 0xFFFFu) - (sc.v12 >> 16), sh_hist + HIST_WHITE * HB + 2, lane);
  flush_one((sc.w23 >> 16) - (sc.v3w1 & 0xFFFFu), sh_hist + HIST_WHITE * HB + 3, lane);
  flush_one(sc.d12 & 0xFFFFu, sh_hist + HIST_DIAG * HB + 1, lane);
  flush_one(sc.d12 >> 16, sh_hist + HIST_DIAG * HB + 2, lane);
  flush_one(sc.d3, sh_hist + HIST_DIAG * HB + 3, lane);
  sc = ShortCounts{0, 0, 0, 0, 0};
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

// The packed paths use the sm_100 float2 arithmetic (__fadd2_rn, __ffma2_rn):
// one instruction for two columns, each lane rounded as its scalar form.

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

// The same decision for a row vector of series a and a column vector of
// series b (cross recurrence).
template <int NORM>
__device__ __forceinline__ bool exact_decision2(const double* __restrict__ a,
                                                const double* __restrict__ b, int64_t i,
                                                int64_t j, int m, int tau, double eps) {
  double acc = 0.0;
  for (int k = 0; k < m; ++k) {
    const double diff = __dsub_rn(a[i + (int64_t)k * tau], b[j + (int64_t)k * tau]);
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
                                              volatile int* abort_flag,
                                              long long limit = SPIN_CYCLES) {
  const long long t0 = clock64();
  while (*ctr < target) {
    if (*abort_flag) return false;
    if (clock64() - t0 > limit) {
      *abort_flag = 1;
      return false;
    }
    __nanosleep(32);
  }
  return true;
}

// Cells of column j, rows r0 .. r0+31, that can recur: RQA keeps the rows
// above the line of identity outside the Theiler window (i <= j - w); cross
// recurrence keeps the rows below n outside |i - j| < w.
template <bool XR>
__device__ __forceinline__ uint32_t live_mask(int j, int r0, int n, int w) {
  if (j < 0) return 0u;
  if constexpr (XR)
    return lowmask(n - r0) & ~(lowmask(j + w - r0) & ~lowmask(j - w + 1 - r0));
  else
    return lowmask(j - r0) & lowmask(j - w - r0 + 1);
}

// Row buffer layout: FP32 rows hold each coordinate twice (x0 x0 x1 x1 ...)
// for the packed paths (every norm); FP64 rows hold m doubles.
template <int M, int NORM, bool F64>
__host__ __device__ constexpr int tile_row_elems() {
  return F64 ? M : ((2 * M + 3) / 4) * 4;
}

// Shared-memory bytes of the tile kernel for a launch shape.
inline size_t tile_smem_bytes(int warps, int row_elems, int elem_bytes, int cols) {
  return (size_t)3 * HB * 4                                    // histograms
         + (size_t)warps * 32 * row_elems * elem_bytes          // row vectors
         + (size_t)warps * 4 * cols * 32 * 4                    // per-warp column state
         + (size_t)(warps > 1 ? warps - 1 : 0) * RING * 64 * 4  // carry rings
         + (size_t)2 * warps * 4                                 // ring counters
         + (size_t)warps * (OVF + 1) * 4 + 16;                  // long-line queues
}

// ------------------------------------------------------------------ kernel
// TW: the test instantiation of the bounded waits (TEST_SPIN_CYCLES, and
// the series' withhold_warp / withhold_seq honoured).
template <int M, int NORM, int C, bool F64, bool XR, bool MX = false, bool BD = false,
          bool TW = false>
__global__ void __launch_bounds__(256, 3)
tile_kernel(const SeriesDesc* __restrict__ sd, const Item* __restrict__ items, int nitems,
            int* __restrict__ queue) {
  constexpr long long spin_limit = TW ? TEST_SPIN_CYCLES : SPIN_CYCLES;
  static_assert(C <= 4, "the short-run counters are flushed for at most 8 two-colour words a block");
  using T = typename std::conditional<F64, double, float>::type;
  constexpr int RE = tile_row_elems<M, NORM, F64>();
  constexpr bool PACKED = !F64 && (C % 2 == 0);  // two columns per packed operation
  // the packed L2 and L-infinity margins are negated (sign bit 1 = recurrent),
  // the packed L1 one and the scalar ones are not (sign bit 1 = no recurrence)
  constexpr bool SIGN_REC = PACKED && NORM != 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NW = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  uint32_t* sh_hist = reinterpret_cast<uint32_t*>(smem_raw);
  T* rowbuf = reinterpret_cast<T*>(sh_hist + 3 * HB) + warp * 32 * RE;
  uint32_t* wstate =
      reinterpret_cast<uint32_t*>(reinterpret_cast<T*>(sh_hist + 3 * HB) + NW * 32 * RE);
  uint32_t* Rw_s = wstate + warp * 4 * C * 32;   // recurrence words  [C][32]
  uint32_t* cst_s = Rw_s + C * 32;               // column run state  [C][32]
  uint32_t* dU_s = cst_s + C * 32;               // diagonal up carry [2][C][32]
  uint32_t* ring = wstate + NW * 4 * C * 32;
  volatile int* prod = reinterpret_cast<volatile int*>(ring + (NW > 1 ? NW - 1 : 0) * RING * 64);
  volatile int* cons = prod + NW;
  uint32_t* ovfq = reinterpret_cast<uint32_t*>(const_cast<int*>(cons) + NW) + warp * (OVF + 1);
  __shared__ int s_item;
  __shared__ int s_skip;
  __shared__ volatile int s_abort;
  __shared__ StripCtx s_ctx;

  // per-lane diagonal segment masks (lane d: lower segment bits d-1..0)
  const uint32_t segL = lowmask(lane);
  const uint32_t segU = ~segL;
  if (lane == 0) ovfq[0] = 0;

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
    uint32_t rechecks = 0;  // per lane: at most C columns x n rows < 2^25 pairs
    const Item wi = items[it];
    const SeriesDesc* Sp = sd + wi.series;
    const int n = (int)Sp->n;                    // rows
    const int ncol = XR ? (int)Sp->n2 : n;       // columns
    const int SW = Sp->sw;
    const int tau = Sp->tau;
    const int wtheiler = Sp->w;
    const double* __restrict__ sser = Sp->s;
    const float* __restrict__ xe = Sp->xe;
    const double* __restrict__ sser2 = XR ? Sp->s2 : Sp->s;   // column series
    const float* __restrict__ xe2 = XR ? Sp->xe2 : Sp->xe;
    const int mp = Sp->mp;
    const double eps = Sp->eps;
    uint32_t* __restrict__ colend = Sp->colend;
    uint16_t* __restrict__ row_a = Sp->row_a;
    uint16_t* __restrict__ row_z = Sp->row_z;
    uint16_t* __restrict__ dia_a = Sp->dia_a;
    uint16_t* __restrict__ dia_z = Sp->dia_z;
    const int J1 = ncol - wi.strip * SW;              // strip: [J1-SW, J1)
    // Row band g: rows [R0, R1) of the strip (one band: all rows); the banded
    // code is a separate instantiation so the unbanded one stays lean
    constexpr bool banded = BD;
    const int g = banded ? wi.band : 0;
    const int R0 = banded ? g * Sp->band_h : 0;
    const int R1 = banded ? min(R0 + Sp->band_h, n) : n;
    // descriptors of diagonal k sit at off + k - klo (RQA: k >= 1 in a
    // strip-triangular layout; cross: the n + SW - 1 diagonals of the strip;
    // banded: per item, from the series' item table)
    const int64_t off = banded ? Sp->dia_off[(int64_t)wi.strip * Sp->nbands + g]
                        : XR   ? (int64_t)wi.strip * cross_strip_diags(n, SW)
                               : strip_offset(n, SW, wi.strip) - strip_offset(n, SW, wi.base);
    const int klo = XR ? J1 - SW - (R1 - 1) : banded ? (int)band_klo(J1, SW, R1) : 1;
    // row descriptors keep the strip-triangular layout (rows never cross bands)
    const int64_t roff = (banded && !XR) ? strip_offset(n, SW, wi.strip) : off;
    const int jw1 = J1 - warp * 32 * C;              // warp: [jw0, jw1)
    const int jw0 = jw1 - 32 * C;
    const int wl_geo = XR ? (J1 - 1) / (32 * C) : (J1 - 2 - R0) / (32 * C);
    const int wlast = wl_geo < NW - 1 ? wl_geo : NW - 1;
    const int nh = XR ? (int)Sp->hl : n;             // longest possible line
    if (threadIdx.x == 0) {
      s_ctx.gl = Sp->hist;
      s_ctx.status = &Sp->counters[CNT_STATUS];
      s_ctx.colfirst = banded ? Sp->col_a + (int64_t)g * (XR ? ncol : n) : colend;
      s_ctx.rowA = row_a + roff;
      s_ctx.rowZ = row_z + roff;
      s_ctx.dia_a = dia_a;
      s_ctx.dia_z = dia_z;
      s_ctx.dbase = off - klo;
      s_ctx.xe = xe;
      s_ctx.sser = sser;
      s_ctx.sser2 = sser2;
      s_ctx.nh = (uint32_t)nh;
      s_ctx.klo = klo;
      s_ctx.eps = eps;
      s_ctx.thr = Sp->thr;
      s_ctx.band = Sp->band;
      s_ctx.tau = tau;
      s_ctx.mp = mp;
      s_ctx.sp = Sp;
    }
    __syncthreads();
    const HistSink hs{sh_hist, &s_ctx, ovfq};

    if (warp <= wlast) {
      const bool leftmost = warp == wlast;
      const int jmax = jw1 - 1;
      // RQA: rows above the line of identity (within the band); cross: all n rows
      const int bhi = XR       ? (R1 - 1) >> 5
                      : banded ? min((jmax - 1) >> 5, (R1 - 1) >> 5)
                               : (jmax - 1) >> 5;
      const int bhi_left = leftmost ? -1
                           : XR     ? bhi
                           : banded ? min((jmax - 32 * C - 1) >> 5, (R1 - 1) >> 5)
                                    : (jmax - 32 * C - 1) >> 5;
      const int blo = R0 >> 5;
      // the band cuts this warp's triangle (cross: the rectangle) so diagonals
      // continue below its bottom
      const bool cut_below =
          banded && (XR ? R1 < n : ((jmax - 1) >> 5) > ((R1 - 1) >> 5));
      // first run of each column: next to the line of identity (colend), or
      // per band [nbands][columns], touching the band's bottom edge (or, for
      // RQA, the line of identity)
      uint32_t* ring_in = warp > 0 ? ring + (warp - 1) * RING * 64 : nullptr;
      uint32_t* ring_out = !leftmost ? ring + warp * RING * 64 : nullptr;
      int seq_in = 0, seq_out = 0;

      // Column vectors of this lane's C columns stay in registers (packed in
      // pairs of columns on the L2 path).
      constexpr int CX = PACKED ? 1 : C;
      constexpr int CP = PACKED ? C / 2 : 1;
      T xc[CX][M];
      // packed paths: columns j - 32 and j of a pair, negated (exact), so that
      // the packed add x_r + (-x_c) rounds exactly as x_r - x_c
      float2 xn2[CP][M];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int j = jw0 + 32 * c + lane;
#pragma unroll
        for (int k = 0; k < (MX ? 0 : M); ++k) {
          if constexpr (F64) {
            xc[c][k] = j >= 0 ? sser2[j + k * tau] : 0.0;
          } else if constexpr (PACKED) {
            if (c % 2 == 1) {
              const int j0 = j - 32;
              xn2[c / 2][k] = make_float2(j0 >= 0 ? -xe2[(int64_t)j0 * mp + k] : 0.f,
                                          j >= 0 ? -xe2[(int64_t)j * mp + k] : 0.f);
            }
          } else {
            xc[c][k] = j >= 0 ? xe2[(int64_t)j * mp + k] : 0.f;
          }
        }
        cst_s[c * 32 + lane] = ST_FLAG;
        // carry from below the first block: a run touching the band's bottom
        // edge where the diagonal continues there (cell (R1, j) exists)
        dU_s[c * 32 + lane] = (cut_below && (XR ? j >= 0 : j > R1)) ? DG_EDGE : 0u;
      }
      int bufo = 0;  // which half of dU_s holds the carries of the block below
      ShortCounts sc{0, 0, 0, 0, 0};
      int since_flush = 0;
      bool ok = true;

      for (int b = bhi; b >= blo && ok; --b) {
        const int r0 = b << 5;
        const float thr = ldv(s_ctx.thr);
        const float band = ldv(s_ctx.band);
        if constexpr (!MX) {  // row vectors of rows r0 .. r0+31 into this warp's buffer
          const int i = r0 + lane;
          if constexpr (!F64) {
            // 16-byte loads of the padded FP32 vector (mp is a multiple of 4)
            // and 16-byte stores; the layout holds each coordinate twice.
            // Slots past the m coordinates are never read.
            const float4* src = reinterpret_cast<const float4*>(ldv(s_ctx.xe) + (int64_t)i * ldv(s_ctx.mp));
            float4* dst = reinterpret_cast<float4*>(reinterpret_cast<float*>(rowbuf) + lane * RE);
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int p = 0; p < (RE / 4 + 1) / 2; ++p) {
              const float4 v = i < n ? src[p] : z4;
              dst[2 * p] = make_float4(v.x, v.x, v.y, v.y);
              if (2 * p + 1 < RE / 4) dst[2 * p + 1] = make_float4(v.z, v.z, v.w, v.w);
            }
          } else {
#pragma unroll
            for (int k = 0; k < RE; ++k) {
              T v = (T)0;
              if (i < n && k < M) v = sser[i + k * tau];
              rowbuf[lane * RE + k] = v;
            }
          }
        }
        __syncwarp();

        // ---- operator I: recurrence words (bit t = row r0 + t) per column
        if constexpr (MX) {
          // precomputed matrix: lane l reads row r0 + l's 32 cells of columns
          // col0 .. col0+31 (two words and a funnel shift when col0 is not a
          // word boundary; col0 < 0 only in a ragged last strip), and the
          // warp transpose turns the 32 row words into column words
          const uint32_t* __restrict__ bits = Sp->bits;
          const int64_t wpr = Sp->wpr;
          const int i = r0 + lane;
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const int col0 = jw0 + 32 * c;
            uint32_t rw = 0;
            if (i < n && col0 > -32) {
              const uint32_t* rowp = bits + (int64_t)i * wpr;
              if (col0 >= 0) {
                const int wi = col0 >> 5, sh = col0 & 31;
                const uint32_t lo = rowp[wi];
                const uint32_t hi = (sh != 0 && wi + 1 < wpr) ? rowp[wi + 1] : 0u;
                rw = __funnelshift_r(lo, hi, sh);
              } else {
                rw = rowp[0] << (-col0);
              }
            }
            Rw_s[c * 32 + lane] =
                transpose32(rw, lane) & live_mask<true>(col0 + lane, r0, n, wtheiler);
          }
        } else if constexpr (!F64) {
          uint32_t Nw[C];
          float mn[C];
#pragma unroll
          for (int c = 0; c < C; ++c) {
            Nw[c] = 0;
            mn[c] = __int_as_float(0x7f800000);
          }
          if constexpr (PACKED && NORM == 1) {
            // L2, two columns per packed op.  Accumulate -thr + sum d^2, the
            // exact negation of pair_margin() (round-to-nearest is symmetric),
            // whose sign bit is 1 for a recurrence.  An exact zero (a tie) is
            // inside the band and re-decided below.
            const float2 nthr2 = make_float2(-thr, -thr);
#pragma unroll 4
            for (int t = 31; t >= 0; --t) {
              float2 xr2[2 * (RE / 4)];
              const float4* rb = reinterpret_cast<const float4*>(rowbuf) + t * (RE / 4);
#pragma unroll
              for (int p = 0; p < RE / 4; ++p) {  // 16-byte loads: two coordinates each
                const float4 v = rb[p];
                xr2[2 * p] = make_float2(v.x, v.y);
                xr2[2 * p + 1] = make_float2(v.z, v.w);
              }
#pragma unroll
              for (int c = 0; c < C / 2; ++c) {
                float2 acc = nthr2;
#pragma unroll
                for (int k = 0; k < M; ++k) {
                  const float2 d = __fadd2_rn(xr2[k], xn2[c][k]);
                  acc = __ffma2_rn(d, d, acc);
                }
                Nw[2 * c] = __funnelshift_l(__float_as_uint(acc.x), Nw[2 * c], 1);
                Nw[2 * c + 1] = __funnelshift_l(__float_as_uint(acc.y), Nw[2 * c + 1], 1);
                mn[2 * c] = fminf(mn[2 * c], fminf(fabsf(acc.x), fabsf(acc.y)));
              }
            }
#pragma unroll
            for (int c = 0; c < C / 2; ++c) mn[2 * c + 1] = mn[2 * c];
          } else if constexpr (PACKED && NORM == 2) {
            // L1, two columns per packed subtraction, then thr minus each |d_k|
            // in pair_margin()'s order (x_r + (-x_c) rounds exactly as
            // x_r - x_c), so every margin is the scalar one; its sign bit is 1
            // for a pair that does not recur.
#pragma unroll 4
            for (int t = 31; t >= 0; --t) {
              float2 xr2[2 * (RE / 4)];
              const float4* rb = reinterpret_cast<const float4*>(rowbuf) + t * (RE / 4);
#pragma unroll
              for (int p = 0; p < RE / 4; ++p) {  // 16-byte loads: two coordinates each
                const float4 v = rb[p];
                xr2[2 * p] = make_float2(v.x, v.y);
                xr2[2 * p + 1] = make_float2(v.z, v.w);
              }
#pragma unroll
              for (int c = 0; c < C / 2; ++c) {
                float a0 = thr, a1 = thr;
#pragma unroll
                for (int k = 0; k < M; ++k) {
                  const float2 dd = __fadd2_rn(xr2[k], xn2[c][k]);
                  a0 = __fsub_rn(a0, fabsf(dd.x));
                  a1 = __fsub_rn(a1, fabsf(dd.y));
                }
                Nw[2 * c] = __funnelshift_l(__float_as_uint(a0), Nw[2 * c], 1);
                Nw[2 * c + 1] = __funnelshift_l(__float_as_uint(a1), Nw[2 * c + 1], 1);
                mn[2 * c] = fminf(mn[2 * c], fminf(fabsf(a0), fabsf(a1)));
              }
            }
#pragma unroll
            for (int c = 0; c < C / 2; ++c) mn[2 * c + 1] = mn[2 * c];
          } else if constexpr (PACKED) {
            // L-infinity, two columns per packed subtraction: the exact
            // maximum of |d_k| per column, then mx - thr, the exact negation
            // of pair_margin()'s thr - mx, whose sign bit is 1 for a
            // recurrence.  An exact zero (a tie) is inside the band.
            const float2 nthr2 = make_float2(-thr, -thr);
#pragma unroll 4
            for (int t = 31; t >= 0; --t) {
              float2 xr2[2 * (RE / 4)];
              const float4* rb = reinterpret_cast<const float4*>(rowbuf) + t * (RE / 4);
#pragma unroll
              for (int p = 0; p < RE / 4; ++p) {  // 16-byte loads: two coordinates each
                const float4 v = rb[p];
                xr2[2 * p] = make_float2(v.x, v.y);
                xr2[2 * p + 1] = make_float2(v.z, v.w);
              }
#pragma unroll
              for (int c = 0; c < C / 2; ++c) {
                float m0 = 0.f, m1 = 0.f;
#pragma unroll
                for (int k = 0; k < M; ++k) {
                  const float2 d = __fadd2_rn(xr2[k], xn2[c][k]);
                  m0 = fmaxf(m0, fabsf(d.x));
                  m1 = fmaxf(m1, fabsf(d.y));
                }
                const float2 acc = __fadd2_rn(make_float2(m0, m1), nthr2);
                Nw[2 * c] = __funnelshift_l(__float_as_uint(acc.x), Nw[2 * c], 1);
                Nw[2 * c + 1] = __funnelshift_l(__float_as_uint(acc.y), Nw[2 * c + 1], 1);
                mn[2 * c] = fminf(mn[2 * c], fminf(fabsf(acc.x), fabsf(acc.y)));
              }
            }
#pragma unroll
            for (int c = 0; c < C / 2; ++c) mn[2 * c + 1] = mn[2 * c];
          } else {
#pragma unroll 4
            for (int t = 31; t >= 0; --t) {
              float xr[M];
              const float* rb = reinterpret_cast<const float*>(rowbuf) + t * RE;
#pragma unroll
              for (int k = 0; k < M; ++k) xr[k] = rb[2 * k];
#pragma unroll
              for (int c = 0; c < C; ++c) {
                const float acc = pair_margin<M, NORM>(xr, (const float*)xc[c], thr);
                Nw[c] = __funnelshift_l(__float_as_uint(acc), Nw[c], 1);
                mn[c] = fminf(mn[c], fabsf(acc));
              }
            }
          }
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const int j = jw0 + 32 * c + lane;
            const uint32_t live = live_mask<XR>(j, r0, n, wtheiler);
            // packed L2 / L-infinity: sign bit = recurrent; else not recurrent
            uint32_t R = (SIGN_REC ? Nw[c] : ~Nw[c]) & live;
            if (mn[c] <= band && live) {
              // near-radius pairs: re-decide in FP64 with the exact order
              uint32_t todo = live;
              while (todo) {
                const int t = __ffs(todo) - 1;
                todo &= todo - 1;
                float xr[M], xcc[M];
                const float* rb = reinterpret_cast<const float*>(rowbuf) + t * RE;
#pragma unroll
                for (int k = 0; k < M; ++k) {
                  xr[k] = rb[2 * k];
                  if constexpr (PACKED) {
                    xcc[k] = -((c % 2) ? xn2[c / 2][k].y : xn2[c / 2][k].x);
                  } else {
                    xcc[k] = (float)xc[c][k];
                  }
                }
                const float acc = pair_margin<M, NORM>(xr, xcc, thr);
                if (fabsf(acc) <= band) {
                  bool r;
                  if constexpr (XR)
                    r = exact_decision2<NORM>(ldv(s_ctx.sser), ldv(s_ctx.sser2), r0 + t, j, M, ldv(s_ctx.tau),
                                             ldv(s_ctx.eps));
                  else
                    r = exact_decision<NORM>(ldv(s_ctx.sser), r0 + t, j, M, ldv(s_ctx.tau), ldv(s_ctx.eps));
                  R = r ? (R | (1u << t)) : (R & ~(1u << t));
                  ++rechecks;
                }
              }
            }
            Rw_s[c * 32 + lane] = R;
          }
        } else {
          uint32_t Rf[C];
#pragma unroll
          for (int c = 0; c < C; ++c) Rf[c] = 0;
          for (int t = 31; t >= 0; --t) {
            double xr[M];
#pragma unroll
            for (int k = 0; k < M; ++k) xr[k] = reinterpret_cast<const double*>(rowbuf)[t * RE + k];
#pragma unroll
            for (int c = 0; c < C; ++c) {
              const bool r = exact_decision_regs<M, NORM>(xr, (const double*)xc[c], eps);
              Rf[c] = (Rf[c] << 1) | (r ? 1u : 0u);
            }
          }
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const int j = jw0 + 32 * c + lane;
            const uint32_t live = live_mask<XR>(j, r0, n, wtheiler);
            Rw_s[c * 32 + lane] = Rf[c] & live;
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
          if (lane == 0)
            ok = spin_until_ge(prod + (warp - 1), seq_in + 1, &s_abort, spin_limit);
          ok = __shfl_sync(FULL, ok, 0);
          if (!ok) break;
          __threadfence_block();
          const volatile uint32_t* slot = ring_in + (seq_in % RING) * 64;
          if constexpr (!XR) rst = slot[lane];
          dL = slot[32 + lane];
          __syncwarp();
          if (lane == 0) cons[warp] = seq_in + 1;
          ++seq_in;
        }

        const int irow = r0 + lane;
        const bool row_valid = irow <= J1 - 2;
        const int d = lane;
        uint32_t* dU_old = dU_s + bufo * C * 32;
        uint32_t* dU_new = dU_s + (bufo ^ 1) * C * 32;
        uint32_t Dprev = 0;
#pragma unroll 1
        for (int c = C - 1; c >= 0; --c) {
          const int col0 = jw0 + 32 * c;
          const int j = col0 + lane;
          const uint32_t R = Rw_s[c * 32 + lane];
          // row words (lane = row) and diagonal words (lane = diagonal: a bit
          // reverse and a lane rotate of the column words, then a transpose)
          uint32_t RW = R, D;
          {
            const uint32_t rb = __brev(R);
            D = __funnelshift_r(rb, rb, 31 - lane);
            if constexpr (!XR)
              transpose32x2(RW, D, lane);
            else
              D = transpose32(D, lane);
          }
          if constexpr (XR && !MX) {
            // cross recurrence, a block below the top row block with no
            // column left of the matrix: every column word is full
            if (r0 + 32 <= n && col0 >= 0) {
              auto emit2 = [&](uint32_t col, uint32_t len) { hs.add2(col, len); };
              cst_s[c * 32 + lane] = scan2_full(
                  R, cst_s[c * 32 + lane], sc, hs, emit2, [&](uint32_t col, uint32_t len) {
                    if (banded && R1 < n)  // touches the band's bottom edge: join later
                      ldv(s_ctx.colfirst)[j] = len | (col << 31);
                    else if (len)
                      hs.add2(col, len);
                  });
              const int k = col0 - r0 + d;
              auto emitd = [&](uint32_t len) { hs.add(HIST_DIAG, len); };
              auto firstd = [&](uint32_t len) {
                if (k >= ldv(s_ctx.klo)) ldv(s_ctx.dia_a)[ldv(s_ctx.dbase) + k] = (uint16_t)len;
              };
              if (c == C - 1) {
                dU_new[c * 32 + lane] =
                    scanb_full(D | segL, dL, sc, hs, emitd, firstd) - (uint32_t)d;
              } else {
                const uint32_t w = (Dprev & segL) | (D & segU);
                dU_new[c * 32 + lane] = scanb_full(__funnelshift_r(w, w, d),
                                                   dU_old[(c + 1) * 32 + lane], sc, hs, emitd, firstd);
              }
              Dprev = D;
              hs.drain(lane);
              continue;
            }
          }
          if constexpr (!XR && !MX) {
            // two or more blocks right of the diagonal (almost every
            // sub-block): every column and row word is full, no row ends
            // here, so the per-lane geometry below is not needed (5 % of the
            // 1M-point kernel's time)
            if (col0 - r0 >= 64) {
              auto emit2 = [&](uint32_t col, uint32_t len) { hs.add2(col, len); };
              cst_s[c * 32 + lane] = scan2_full(
                  R, cst_s[c * 32 + lane], sc, hs, emit2,
                  [&](uint32_t col, uint32_t len) { ldv(s_ctx.colfirst)[j] = len | (col << 31); });
              rst = scan2_full(RW, rst, sc, hs, emit2, [&](uint32_t col, uint32_t len) {
                ldv(s_ctx.rowA)[irow] = (uint16_t)((len << 1) | col);
              });
              const int k = col0 - r0 + d;
              auto emitd = [&](uint32_t len) { hs.add(HIST_DIAG, len); };
              auto firstd = [&](uint32_t len) {
                if (k >= ldv(s_ctx.klo)) ldv(s_ctx.dia_a)[ldv(s_ctx.dbase) + k] = (uint16_t)len;
              };
              if (c == C - 1) {
                dU_new[c * 32 + lane] =
                    scanb_full(D | segL, dL, sc, hs, emitd, firstd) - (uint32_t)d;
              } else {
                const uint32_t w = (Dprev & segL) | (D & segU);
                dU_new[c * 32 + lane] = scanb_full(__funnelshift_r(w, w, d),
                                                   dU_old[(c + 1) * 32 + lane], sc, hs, emitd, firstd);
              }
              Dprev = D;
              hs.drain(lane);
              continue;
            }
          }

          // ---- operator III, upper part of full column j (rows < j); cross:
          // the whole column, whose first run ends at the bottom border
          {
            const int vt = j < 0 ? 0 : clamp32((XR ? n : j) - r0);
            auto emitc = [&](uint32_t col, uint32_t len) { hs.add2(col, len); };
            auto firstc = [&](uint32_t col, uint32_t len) {
              if constexpr (XR) {
                if (banded && R1 < n)  // touches the band's bottom edge: join later
                  ldv(s_ctx.colfirst)[j] = len | (col << 31);
                else if (len)
                  hs.add2(col, len);
              } else {
                ldv(s_ctx.colfirst)[j] = len | (col << 31);
              }
            };
            if (vt == 32)
              cst_s[c * 32 + lane] = scan2_full(R, cst_s[c * 32 + lane], sc, hs, emitc, firstc);
            else if (vt > 0)
              cst_s[c * 32 + lane] = scan2(R, vt - 1, 0, cst_s[c * 32 + lane], hs, emitc, firstc);
          }

          // ---- operator III, lower part of full column irow = upper row irow
          if constexpr (!XR) {
            const int lo = irow + 1 - col0;  // first valid bit of the row
            if (lo <= 31 && !(rst & ST_DONE) && row_valid) {
              auto emitr = [&](uint32_t col, uint32_t len) { hs.add2(col, len); };
              auto firstr = [&](uint32_t col, uint32_t len) {
                ldv(s_ctx.rowA)[irow] = (uint16_t)((len << 1) | col);
              };
              if (lo <= 0)
                rst = scan2_full(RW, rst, sc, hs, emitr, firstr);
              else
                rst = scan2(RW, 31, lo, rst, hs, emitr, firstr);
              if (lo >= 0) {  // the row ends here, at column irow + 1
                const uint32_t len = rst & ST_LEN, col = (rst >> 28) & 1u;
                const uint32_t same = (rst >> 29) & 1u;
                ldv(s_ctx.rowZ)[irow] = (uint16_t)((len << 2) | (same << 1) | col);
                if (same) ldv(s_ctx.rowA)[irow] = 0;
                rst = ST_DONE;
              }
            }
          }

          // ---- operator II: diagonal pieces (lane d)
          {
            const int k = col0 - r0 + d;  // diagonal of this sub-block's upper segment
            auto emitd = [&](uint32_t len) { hs.add(HIST_DIAG, len); };
            auto firstd = [&](uint32_t len) {
              if (k >= ldv(s_ctx.klo)) ldv(s_ctx.dia_a)[ldv(s_ctx.dbase) + k] = (uint16_t)len;
            };
            if (c == C - 1) {
              // upper segment only (bits 31..d), entering from the right;
              // its d cells below count as black and are taken off again
              dU_new[c * 32 + lane] =
                  scanb_full(D | segL, dL, sc, hs, emitd, firstd) - (uint32_t)d;
            } else {
              // the lower segment of sub-block c+1 (bits d-1..0 of Dprev) and
              // the upper segment of c (bits 31..d of D) are one diagonal;
              // rotated by d its cells run from bit 31 down to bit 0
              const uint32_t w = (Dprev & segL) | (D & segU);
              const uint32_t y = __funnelshift_r(w, w, d);
              dU_new[c * 32 + lane] = scanb_full(y, dU_old[(c + 1) * 32 + lane], sc, hs, emitd, firstd);
            }
            Dprev = D;
          }
          hs.drain(lane);
        }
        {  // the lower segment of sub-block 0 (bits d-1..0) leaves to the left
          const int k = jw0 - r0 + d - 32;
          const uint32_t du = dU_old[lane];
          dL = du;
          if (d > 0)  // the segment shifted to the top, 32 - d black cells below it
            dL = scanb_full(
                     (Dprev << (32 - d)) | lowmask(32 - d), du, sc, hs,
                     [&](uint32_t len) { hs.add(HIST_DIAG, len); },
                     [&](uint32_t len) {
                       if (k >= ldv(s_ctx.klo)) ldv(s_ctx.dia_a)[ldv(s_ctx.dbase) + k] = (uint16_t)len;
                     }) -
                 (uint32_t)(32 - d);
          hs.drain(lane);
        }
        bufo ^= 1;
        if (++since_flush == FLUSH_BLOCKS) {
          flush_short(sc, sh_hist, lane);
          since_flush = 0;
        }

        // ---- carries leaving to the left
        if (leftmost) {
          if (!XR && !(rst & ST_DONE) && row_valid) {
            const uint32_t len = rst & ST_LEN, col = (rst >> 28) & 1u;
            const uint32_t same = (rst >> 29) & 1u;
            if (len > 0) {
              ldv(s_ctx.rowZ)[irow] = (uint16_t)((len << 2) | (same << 1) | col);
              if (same) ldv(s_ctx.rowA)[irow] = 0;
            }
          }
          const int kx = jw0 - r0 + lane - 32;  // diagonal leaving through the left edge
          if (kx >= ldv(s_ctx.klo))
            ldv(s_ctx.dia_z)[ldv(s_ctx.dbase) + kx] = (uint16_t)((dL & ST_LEN) | ((dL & DG_EDGE) ? 0x8000u : 0u));
        } else if (b <= bhi_left) {
          if (lane == 0)
            ok = spin_until_ge(cons + (warp + 1), seq_out - RING + 1, &s_abort, spin_limit);
          ok = __shfl_sync(FULL, ok, 0);
          if (!ok) break;
          uint32_t* slot = ring_out + (seq_out % RING) * 64;
          if constexpr (!XR) slot[lane] = rst;
          slot[32 + lane] = dL;
          __syncwarp();
          __threadfence_block();
          // test instantiation: from the chosen hand-over on, this warp stops
          // publishing, and the next warp's bounded wait gives up
          const bool withhold =
              TW && warp + 1 == ldv(s_ctx.sp)->withhold_warp && seq_out + 1 >= ldv(s_ctx.sp)->withhold_seq;
          if (lane == 0 && !withhold) prod[warp] = seq_out + 1;
          ++seq_out;
        }
      }

      if (ok) {
        // ---- top border (row R0): close or record column runs, record the
        // ends of the diagonals leaving through it (k = j - R0 at (R0, j))
#pragma unroll 1
        for (int c = 0; c < C; ++c) {
          const int j = jw0 + 32 * c + lane;
          if (j >= (XR ? 0 : R0 + 1)) {
            const uint32_t st = cst_s[c * 32 + lane];
            const uint32_t len = st & ST_LEN, col = (st >> 28) & 1u;
            const bool whole = (st & ST_FLAG) != 0;  // one run over the column's segment
            // the run continues in the band above, or below: record it
            const bool keep = banded && !(R0 == 0 && ((!XR && j <= R1) || !whole));
            if (!keep) {
              if (len > 0) {
                if (!XR && whole)
                  ldv(s_ctx.colfirst)[j] = len | (col << 31);
                else
                  hs.add2(col, len);
              }
            } else {
              ldv(s_ctx.sp)->col_z[(int64_t)g * (XR ? ncol : n) + j] =
                  len | (whole ? (1u << 30) : 0u) | (col << 31);
            }
            const uint32_t du = dU_s[bufo * C * 32 + c * 32 + lane];
            ldv(s_ctx.dia_z)[ldv(s_ctx.dbase) + (j - R0)] =
                (uint16_t)((du & ST_LEN) | ((du & DG_EDGE) ? 0x8000u : 0u));
          }
        }
      }
      hs.drain(lane);
      flush_short(sc, sh_hist, lane);
    }
    __syncthreads();
    const SeriesDesc* const Sq = ldv(s_ctx.sp);
    if (s_abort && threadIdx.x == 0)
      atomicCAS(&Sq->counters[CNT_STATUS], 0ull, 6ull /* RQA_ETIMEOUT */);
    // flush the strip's histograms
    const int64_t stride = (int64_t)(XR ? (int)Sq->hl : n) + 1;
    for (int q = threadIdx.x; q < 3 * HB; q += blockDim.x) {
      const uint32_t v = sh_hist[q];
      if (v) atomicAdd(&Sq->hist[(q / HB) * stride + (q % HB)], (unsigned long long)v);
    }
    // rechecks of this strip: one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rechecks += __shfl_xor_sync(FULL, rechecks, o);
    if (lane == 0 && rechecks) atomicAdd(&Sq->counters[CNT_RECHECKS], (unsigned long long)rechecks);
  }
}

}  // namespace rqa
