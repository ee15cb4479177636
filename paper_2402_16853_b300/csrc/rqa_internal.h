// rqa_internal.h -- structures shared by the host side and the CUDA kernels of
// librqa_b300.so.  Nothing here is part of the public C ABI (include/rqa.h).
#pragma once
#include <stdint.h>

namespace rqa {

// Per-series state in device memory.  The host fills the inputs and buffer
// pointers; the prepare kernel fills the FP32 constants.
struct SeriesDesc {
  // ---- inputs
  const double* s;      // FP64 series, N values (device)
  float* xe;            // embedded FP32 vectors, [n][mp] (device)
  int64_t N;            // series length
  int64_t n;            // embedded vectors, N - (m-1) tau
  int32_t m, tau, norm, w;
  int32_t mp;           // floats per stored vector (m rounded up to 4)
  int32_t sw;           // columns per CTA strip
  double eps;
  double band_override; // < 0: automatic
  // ---- cross recurrence (Sect. 3.3): the columns come from a second series
  const double* s2;     // FP64 column series (device); == s for RQA
  float* xe2;           // its embedded FP32 vectors; == xe for RQA
  int64_t N2, n2;       // its length and vector count; == N, n for RQA
  int64_t hl;           // longest possible line: n (RQA) or max(n, n2)
  int32_t cross;        // 1: rows from s, columns from s2, no symmetry
  // ---- precomputed matrix (Sect. 9): rows x n2 bits, row-major, bit b of
  // word w of a row is column 32 w + b; s, s2, xe, xe2 are unused
  const uint32_t* bits;
  int64_t wpr;          // words per row, ceil(n2 / 32)
  // ---- row bands (RQA only): with nbands > 1, CTA strip Q is split into
  // items (Q, g) of rows [g H, (g+1) H) so that series too small to fill the
  // GPU with strips alone still do; 0 / 1: one band of all rows
  int32_t band_h;       // H, a multiple of 32
  int32_t nbands;       // ceil(n / H)
  const int64_t* dia_off;  // [nstrips][nbands] diagonal-descriptor offset of item (Q, g)
  uint32_t* col_a;      // [nbands][n] first run of column j in band g (touches its bottom)
  uint32_t* col_z;      // [nbands][n] run of column j touching band g's top edge
  // ---- filled by the prepare kernel
  double center, scale; // x32 = fl32((s - center) * scale)
  float thr;            // FP32 threshold: eps*scale (L1, max) or its square (L2)
  float band;           // |acc| <= band -> re-decide in FP64
  double band_rel;      // band / eps (eps^2 for L2)
  double bound_rel;     // proven sufficient band, same units
  // ---- outputs (device)
  unsigned long long* hist;   // [3][hl+1]: upper diagonals, vertical, white vertical
  uint16_t* row_a;            // boundary descriptors, strip-triangular layout
  uint16_t* row_z;
  uint16_t* dia_a;
  uint16_t* dia_z;
  uint32_t* colend;           // [n] run of column j touching row j-1
  uint32_t* rowend;           // [n] run of row i touching column i+1
  // strip groups (Divide & Recombine, Sect. 4.1): a series whose boundary
  // descriptors would exceed the memory budget runs G strips at a time; the
  // run of each row and each diagonal left open at a group's left edge is
  // carried to the next group here (length | colour << 31; diagonals: length)
  uint32_t* rcarry;           // [n]
  uint32_t* dcarry;           // [n]
  unsigned long long* counters;  // [0] rechecks, [1] status (rqa_status)
  // ---- test of the bounded ring waits (read only by the test instantiation
  // of the tile kernel; 0 = off): warp withhold_warp - 1 of every CTA stops
  // publishing its carries from its withhold_seq-th hand-over on, so the
  // next warp's wait must give up
  int32_t withhold_warp;
  int32_t withhold_seq;
};

// Fill the column-series fields of an RQA (symmetric) descriptor: the
// columns are the rows' own vectors.
__host__ __device__ inline void desc_set_symmetric(SeriesDesc& d) {
  d.s2 = d.s;
  d.xe2 = d.xe;
  d.N2 = d.N;
  d.n2 = d.n;
  d.hl = d.n;
  d.cross = 0;
}

enum { HIST_DIAG = 0, HIST_VERT = 1, HIST_WHITE = 2 };
// Per-series counters: rechecks, status, (written after the merges) the
// longest length with a non-zero count in each of the three histograms, so
// the host reads each histogram only up to there, and the series' minimum
// and maximum in an order-preserving encoding (the minimum complemented),
// gathered by atomic maxima while the series is scanned.
enum {
  CNT_RECHECKS = 0,
  CNT_STATUS = 1,
  CNT_LAST = 2 /* [3] */,
  CNT_LO = 5,
  CNT_HI = 6,
  CNT_WORDS = 7
};

// Offset of strip Q's descriptors: strips hold J1(Q) - 1 entries each, with
// J1(Q) = n - Q*sw the exclusive right end of the strip.
__host__ __device__ inline int64_t strip_offset(int64_t n, int64_t sw, int64_t Q) {
  return Q * (n - 1) - sw * (Q * (Q - 1) / 2);
}
__host__ __device__ inline int64_t num_strips(int64_t n, int64_t sw) {
  return n >= 2 ? (n - 2) / sw + 1 : 0;
}

// Cross recurrence: every strip spans all n1 rows, so strip Q holds the
// n1 + sw - 1 diagonals k = J1(Q) - sw - (n1 - 1) .. J1(Q) - 1 that can
// cross it, with J1(Q) = n2 - Q*sw.
__host__ __device__ inline int64_t cross_strip_diags(int64_t n1, int64_t sw) {
  return n1 + sw - 1;
}
__host__ __device__ inline int64_t cross_num_strips(int64_t n2, int64_t sw) {
  return n2 >= 1 ? (n2 - 1) / sw + 1 : 0;
}

struct Item {
  int32_t series;
  int32_t strip;
  int32_t band;
  int32_t base;   // first strip of the item's strip group (0 unless the series
                  // runs in groups; its descriptors start at that strip's)
};

// Diagonals k >= 1 that can cross item (Q, g) of an RQA strip [J1 - sw, J1)
// and band rows [R0, R1): k from band_klo to J1 - 1 - R0.
__host__ __device__ inline int64_t band_klo(int64_t J1, int64_t sw, int64_t R1) {
  const int64_t k = J1 - sw - R1 + 1;
  return k > 1 ? k : 1;
}

struct TileConfig {
  int warps;       // warps per CTA (warps of one CTA strip, right to left)
  int cols;        // columns per lane (C): a warp covers 32*C columns
  int band_scale;  // row-band height: the size rule's (0), half (-1) or double (+1)
};

}  // namespace rqa
