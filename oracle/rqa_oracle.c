/*
 * rqa_oracle.c -- TEST INFRASTRUCTURE, not part of the product.
 *
 * A plain, slow, FP64 CPU statement of recurrence quantification analysis
 * (RQA) as the PyRQA paper states the problem:
 *   - time-delay embedding of a scalar series (Sect. 2; Sect. 7.2, the
 *     embedding_dimension / time_delay settings),
 *   - the pairwise distance under the L1, L2 or L-infinity norm (Sect. 7.2,
 *     "similarity measures") and the fixed-radius neighbourhood (Sect. 2,
 *     Sect. 7.2 FixedRadius), giving the binary recurrence matrix (Sect. 2),
 *   - the three line types -- diagonal and vertical lines of recurrence points
 *     and white vertical lines of non-recurrence points -- and their
 *     frequency distributions (Sect. 2, the enumerated list of line types),
 *   - the quantitative measures of Table 3, whose definitions the paper
 *     defers to Marwan et al. (2007) (Sect. 2).
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   R1  vectors are x_i = (s[i], s[i+tau], ..., s[i+(m-1)tau]), i = 0..n-1,
 *       n = N - (m-1)tau (0-based, as Fig. 1 numbers vectors x_0..x_10);
 *   R2  distances use a fixed left-to-right operation order:
 *       L1  d = ((|D0| + |D1|) + ...),   L2  d = sqrt(((D0*D0) + D1*D1) + ...),
 *       Linf d = max over k of |Dk| starting from 0, with Dk = x_i[k] - x_j[k];
 *   R3  R_ij = 1 iff d(x_i, x_j) <= eps and |i - j| >= w (Theiler window w;
 *       w = 0 keeps the line of identity, w = 1 removes only it);
 *   R4  lines are maximal runs along a diagonal or a column of the FULL n x n
 *       matrix (both triangles, line of identity included); runs cut by the
 *       matrix border count with their truncated length;
 *   R5  measures: see oracle_measures() below.
 *
 * This file shares no code with the CUDA library; it is built with
 * -ffp-contract=off so no multiply-add is fused.  Only tests/, the smoke
 * check of the graft entry point and the benchmark's CPU-baseline leg may
 * load it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_NORM_MAX 0
#define ORACLE_NORM_L2 1
#define ORACLE_NORM_L1 2

typedef struct {
  int32_t m;        /* embedding dimension (Sect. 7.2)                      */
  int32_t tau;      /* time delay (Sect. 7.2)                               */
  double eps;       /* fixed radius (Sect. 7.2, FixedRadius)                */
  int32_t norm;     /* ORACLE_NORM_*  (Sect. 7.2: L1, L2, L-infinity)       */
  int32_t theiler;  /* Theiler window w (reading R3)                        */
  int32_t l_min;    /* min_diagonal_line_length (Sect. 7.2)                 */
  int32_t v_min;    /* min_vertical_line_length (Sect. 7.2)                 */
  int32_t w_min;    /* min_white_vertical_line_length (Sect. 7.2)           */
} oracle_settings;

typedef struct {
  double rr, det, l, div, l_entr, lam, tt, v_entr, w, w_entr;
  int64_t l_max, v_max, w_max, n_vec, recurrence_points;
} oracle_measures_t;

/* Number of embedded vectors (reading R1). */
int64_t oracle_nvec(int64_t N, int32_t m, int32_t tau) {
  int64_t n = N - (int64_t)(m - 1) * (int64_t)tau;
  return n > 0 ? n : 0;
}

/* Distance between embedded vectors x_i and x_j (Sect. 7.2; reading R2). */
double oracle_distance(const double* s, int64_t i, int64_t j, int32_t m,
                       int32_t tau, int32_t norm) {
  double acc = 0.0;
  for (int32_t k = 0; k < m; ++k) {
    double a = s[i + (int64_t)k * tau];
    double b = s[j + (int64_t)k * tau];
    double diff = a - b;
    if (norm == ORACLE_NORM_MAX) {
      double ad = fabs(diff);
      if (ad > acc) acc = ad;
    } else if (norm == ORACLE_NORM_L1) {
      acc = acc + fabs(diff);
    } else {
      acc = acc + diff * diff;
    }
  }
  if (norm == ORACLE_NORM_L2) acc = sqrt(acc);
  return acc;
}

/* One element of the recurrence matrix (Sect. 2, fixed radius; reading R3). */
int oracle_recurrent(const double* s, int64_t i, int64_t j,
                     const oracle_settings* st) {
  int64_t gap = i > j ? i - j : j - i;
  if (gap < (int64_t)st->theiler) return 0;
  return oracle_distance(s, i, j, st->m, st->tau, st->norm) <= st->eps;
}

/* Materialise the full n x n recurrence matrix, row-major, one byte per cell.
 * Only for small n: the paper's point is that this is O(N^2) memory
 * (Sect. 1).  Returns the number of recurrence points. */
uint64_t oracle_matrix(const double* s, int64_t N, const oracle_settings* st,
                       uint8_t* R) {
  int64_t n = oracle_nvec(N, st->m, st->tau);
  uint64_t rp = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      uint8_t r = (uint8_t)oracle_recurrent(s, i, j, st);
      R[i * n + j] = r;
      rp += r;
    }
  return rp;
}

/* Close a run of `len` cells of value `v` into the histograms. */
static void close_run(uint64_t* hist_one, uint64_t* hist_zero, int v,
                      int64_t len) {
  if (len <= 0) return;
  if (v) {
    if (hist_one) hist_one[len] += 1;
  } else {
    if (hist_zero) hist_zero[len] += 1;
  }
}

/* Scan one line of cells (a diagonal or a column), given as a callback-free
 * pair of accessors, and add its maximal runs to the histograms.  The cells
 * are visited in order; a run ends where the value changes or the line ends
 * (reading R4: runs cut by the border keep their truncated length). */
typedef struct {
  const uint8_t* R;       /* materialised matrix, or NULL                    */
  const double* s;        /* series, when cells are computed on the fly      */
  const oracle_settings* st;
  int64_t n;
} cell_src;

static int cell_at(const cell_src* c, int64_t i, int64_t j) {
  if (c->R) return c->R[i * c->n + j];
  return oracle_recurrent(c->s, i, j, c->st);
}

/* Diagonal k of the full matrix: cells (i, i + k), k in (-(n-1), n-1).
 * Operator II of Sect. 4.2 ("the inspection of a single diagonal"). */
static void scan_diagonal(const cell_src* c, int64_t k, uint64_t* hd) {
  int64_t n = c->n;
  int64_t i0 = k >= 0 ? 0 : -k;
  int64_t len_line = n - (k >= 0 ? k : -k);
  int prev = -1;
  int64_t run = 0;
  for (int64_t t = 0; t < len_line; ++t) {
    int v = cell_at(c, i0 + t, i0 + t + k);
    if (v == prev) {
      run += 1;
    } else {
      if (prev >= 0) close_run(hd, NULL, prev, run);
      prev = v;
      run = 1;
    }
  }
  if (prev >= 0) close_run(hd, NULL, prev, run);
}

/* Column j of the full matrix: cells (i, j), i = 0..n-1.
 * Operator III of Sect. 4.2 ("the inspection of a single column regarding
 * vertical and white vertical lines"). */
static uint64_t scan_column(const cell_src* c, int64_t j, uint64_t* hv,
                            uint64_t* hw) {
  int64_t n = c->n;
  int prev = -1;
  int64_t run = 0;
  uint64_t ones = 0;
  for (int64_t i = 0; i < n; ++i) {
    int v = cell_at(c, i, j);
    ones += (uint64_t)v;
    if (v == prev) {
      run += 1;
    } else {
      if (prev >= 0) close_run(hv, hw, prev, run);
      prev = v;
      run = 1;
    }
  }
  if (prev >= 0) close_run(hv, hw, prev, run);
  return ones;
}

/* Histograms (index = line length, 0..n) from a materialised matrix.
 * hd: diagonal lines of 1s, hv: vertical lines of 1s, hw: vertical lines of
 * 0s.  Each array holds n + 1 entries and is overwritten. */
void oracle_histograms_from_matrix(const uint8_t* R, int64_t n, uint64_t* hd,
                                   uint64_t* hv, uint64_t* hw) {
  cell_src c = {R, NULL, NULL, n};
  memset(hd, 0, sizeof(uint64_t) * (size_t)(n + 1));
  memset(hv, 0, sizeof(uint64_t) * (size_t)(n + 1));
  memset(hw, 0, sizeof(uint64_t) * (size_t)(n + 1));
  for (int64_t k = -(n - 1); k <= n - 1; ++k) scan_diagonal(&c, k, hd);
  for (int64_t j = 0; j < n; ++j) scan_column(&c, j, hv, hw);
}

/* The same histograms with every cell computed on the fly (O(n) memory),
 * split over threads by diagonal and by column; per-thread histograms are
 * summed at the end (integer sums, so the order does not matter).
 *
 * To time a bounded sample, the caller may restrict the work to every
 * `stride`-th column and every `stride`-th diagonal (stride = 1: all of
 * them, the complete result).  Returns the number of cells visited and
 * stores in *rp the number of recurrence points met in the visited columns
 * (all of them when stride = 1). */
uint64_t oracle_histograms_streaming(const double* s, int64_t N,
                                     const oracle_settings* st, int32_t threads,
                                     int64_t stride, uint64_t* hd, uint64_t* hv,
                                     uint64_t* hw, uint64_t* rp) {
  int64_t n = oracle_nvec(N, st->m, st->tau);
  memset(hd, 0, sizeof(uint64_t) * (size_t)(n + 1));
  memset(hv, 0, sizeof(uint64_t) * (size_t)(n + 1));
  memset(hw, 0, sizeof(uint64_t) * (size_t)(n + 1));
  *rp = 0;
  if (n <= 0) return 0;
  if (stride < 1) stride = 1;
  cell_src c = {NULL, s, st, n};
  uint64_t visited = 0, ones = 0;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
#pragma omp parallel reduction(+ : visited, ones)
  {
    uint64_t* ld = (uint64_t*)calloc((size_t)(n + 1), sizeof(uint64_t));
    uint64_t* lv = (uint64_t*)calloc((size_t)(n + 1), sizeof(uint64_t));
    uint64_t* lw = (uint64_t*)calloc((size_t)(n + 1), sizeof(uint64_t));
    int64_t ndiag = 2 * n - 1;
#pragma omp for schedule(dynamic, 1) nowait
    for (int64_t q = 0; q < ndiag; q += stride) {
      int64_t k = q - (n - 1);
      scan_diagonal(&c, k, ld);
      visited += (uint64_t)(n - (k >= 0 ? k : -k));
    }
#pragma omp for schedule(dynamic, 1)
    for (int64_t j = 0; j < n; j += stride) {
      ones += scan_column(&c, j, lv, lw);
      visited += (uint64_t)n;
    }
#pragma omp critical
    {
      for (int64_t l = 0; l <= n; ++l) {
        hd[l] += ld[l];
        hv[l] += lv[l];
        hw[l] += lw[l];
      }
    }
    free(ld);
    free(lv);
    free(lw);
  }
  *rp = ones;
  return visited;
}

/* ------------------------------------------------------------------------
 * Cross recurrence (the non-symmetric matrix of two series, Sect. 4.2:
 * operator II's degree of parallelism 2N - 1 for non-symmetric matrices;
 * Sect. 3.3 describes cross recurrence quantification).  Rows are the
 * vectors x_i of series s1 (n1 of them), columns the vectors y_j of s2 (n2):
 *   C_ij = 1 iff d(x_i, y_j) <= eps and |i - j| >= w,
 * with the same distance and embedding readings R1-R3.  Lines are runs along
 * the n1 + n2 - 1 diagonals (i, i + k), k in (-(n1-1), n2-1), and along the
 * n2 columns of the n1 x n2 matrix (reading R4 on a rectangle).
 * ------------------------------------------------------------------------ */
double oracle_cross_distance(const double* s1, const double* s2, int64_t i, int64_t j,
                             int32_t m, int32_t tau, int32_t norm) {
  double acc = 0.0;
  for (int32_t k = 0; k < m; ++k) {
    double diff = s1[i + (int64_t)k * tau] - s2[j + (int64_t)k * tau];
    if (norm == ORACLE_NORM_MAX) {
      double ad = fabs(diff);
      if (ad > acc) acc = ad;
    } else if (norm == ORACLE_NORM_L1) {
      acc = acc + fabs(diff);
    } else {
      acc = acc + diff * diff;
    }
  }
  if (norm == ORACLE_NORM_L2) acc = sqrt(acc);
  return acc;
}

static int cross_cell(const double* s1, const double* s2, int64_t i, int64_t j,
                      const oracle_settings* st) {
  int64_t gap = i > j ? i - j : j - i;
  if (gap < (int64_t)st->theiler) return 0;
  return oracle_cross_distance(s1, s2, i, j, st->m, st->tau, st->norm) <= st->eps;
}

/* Histograms (length max(n1, n2) + 1) of the n1 x n2 cross matrix, cells
 * computed on the fly.  Returns the number of recurrence points. */
uint64_t oracle_cross_histograms(const double* s1, int64_t N1, const double* s2,
                                 int64_t N2, const oracle_settings* st,
                                 int32_t threads, uint64_t* hd, uint64_t* hv,
                                 uint64_t* hw) {
  int64_t n1 = oracle_nvec(N1, st->m, st->tau);
  int64_t n2 = oracle_nvec(N2, st->m, st->tau);
  int64_t L = n1 > n2 ? n1 : n2;
  memset(hd, 0, sizeof(uint64_t) * (size_t)(L + 1));
  memset(hv, 0, sizeof(uint64_t) * (size_t)(L + 1));
  memset(hw, 0, sizeof(uint64_t) * (size_t)(L + 1));
  if (n1 <= 0 || n2 <= 0) return 0;
  uint64_t ones = 0;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
#pragma omp parallel reduction(+ : ones)
  {
    uint64_t* ld = (uint64_t*)calloc((size_t)(L + 1), sizeof(uint64_t));
    uint64_t* lv = (uint64_t*)calloc((size_t)(L + 1), sizeof(uint64_t));
    uint64_t* lw = (uint64_t*)calloc((size_t)(L + 1), sizeof(uint64_t));
#pragma omp for schedule(dynamic, 1) nowait
    for (int64_t k = -(n1 - 1); k <= n2 - 1; ++k) {
      /* diagonal k: cells (i, i + k) inside the rectangle */
      int64_t i0 = k >= 0 ? 0 : -k;
      int prev = -1;
      int64_t run = 0;
      for (int64_t i = i0; i < n1 && i + k < n2; ++i) {
        int v = cross_cell(s1, s2, i, i + k, st);
        if (v == prev) {
          run += 1;
        } else {
          if (prev >= 0) close_run(ld, NULL, prev, run);
          prev = v;
          run = 1;
        }
      }
      if (prev >= 0) close_run(ld, NULL, prev, run);
    }
#pragma omp for schedule(dynamic, 1)
    for (int64_t j = 0; j < n2; ++j) {
      int prev = -1;
      int64_t run = 0;
      for (int64_t i = 0; i < n1; ++i) {
        int v = cross_cell(s1, s2, i, j, st);
        ones += (uint64_t)v;
        if (v == prev) {
          run += 1;
        } else {
          if (prev >= 0) close_run(lv, lw, prev, run);
          prev = v;
          run = 1;
        }
      }
      if (prev >= 0) close_run(lv, lw, prev, run);
    }
#pragma omp critical
    {
      for (int64_t l = 0; l <= L; ++l) {
        hd[l] += ld[l];
        hv[l] += lv[l];
        hw[l] += lw[l];
      }
    }
    free(ld);
    free(lv);
    free(lw);
  }
  return ones;
}

/* ------------------------------------------------------------------------
 * A precomputed binary matrix (Sect. 9 lists the quantitative analysis of
 * precomputed recurrence matrices as requested by users).  R holds rows x
 * cols cells (row-major, 0 or 1) and is taken as given, except that cells
 * with |i - j| < w count as 0, as for a computed matrix (reading R3).  Lines
 * are runs along the rows + cols - 1 diagonals and down the cols columns,
 * border-cut runs keeping their length (reading R4).  Histograms have
 * max(rows, cols) + 1 entries.  Returns the number of 1-cells counted.
 * ------------------------------------------------------------------------ */
static int rect_cell(const uint8_t* R, int64_t cols, int64_t i, int64_t j, int32_t w) {
  int64_t gap = i > j ? i - j : j - i;
  if (gap < (int64_t)w) return 0;
  return R[i * cols + j] != 0;
}

uint64_t oracle_histograms_from_rect(const uint8_t* R, int64_t rows, int64_t cols,
                                     int32_t w, uint64_t* hd, uint64_t* hv,
                                     uint64_t* hw) {
  int64_t L = rows > cols ? rows : cols;
  memset(hd, 0, sizeof(uint64_t) * (size_t)(L + 1));
  memset(hv, 0, sizeof(uint64_t) * (size_t)(L + 1));
  memset(hw, 0, sizeof(uint64_t) * (size_t)(L + 1));
  if (rows <= 0 || cols <= 0) return 0;
  for (int64_t k = -(rows - 1); k <= cols - 1; ++k) {
    int64_t i = k >= 0 ? 0 : -k;
    int prev = -1;
    int64_t run = 0;
    for (; i < rows && i + k < cols; ++i) {
      int v = rect_cell(R, cols, i, i + k, w);
      if (v == prev) {
        run += 1;
      } else {
        if (prev >= 0) close_run(hd, NULL, prev, run);
        prev = v;
        run = 1;
      }
    }
    if (prev >= 0) close_run(hd, NULL, prev, run);
  }
  uint64_t ones = 0;
  for (int64_t j = 0; j < cols; ++j) {
    int prev = -1;
    int64_t run = 0;
    for (int64_t i = 0; i < rows; ++i) {
      int v = rect_cell(R, cols, i, j, w);
      ones += (uint64_t)v;
      if (v == prev) {
        run += 1;
      } else {
        if (prev >= 0) close_run(hv, hw, prev, run);
        prev = v;
        run = 1;
      }
    }
    if (prev >= 0) close_run(hv, hw, prev, run);
  }
  return ones;
}

/* Sum over l >= lo of h[l] and of l * h[l], exactly in 64-bit integers. */
static void hist_sums(const uint64_t* h, int64_t n, int64_t lo, uint64_t* s0,
                      uint64_t* s1) {
  uint64_t a = 0, b = 0;
  if (lo < 1) lo = 1;
  for (int64_t l = lo; l <= n; ++l) {
    a += h[l];
    b += (uint64_t)l * h[l];
  }
  *s0 = a;
  *s1 = b;
}

/* Longest line of length >= lo, 0 if there is none. */
static int64_t hist_max(const uint64_t* h, int64_t n, int64_t lo) {
  if (lo < 1) lo = 1;
  for (int64_t l = n; l >= lo; --l)
    if (h[l] > 0) return l;
  return 0;
}

/* Shannon entropy (natural log) of the distribution of lines of length
 * >= lo: -sum p ln p with p = h[l] / (number of such lines), accumulated in
 * ascending l. */
static double hist_entropy(const uint64_t* h, int64_t n, int64_t lo,
                           uint64_t count) {
  double acc = 0.0;
  if (lo < 1) lo = 1;
  for (int64_t l = lo; l <= n; ++l) {
    if (h[l] == 0) continue;
    double p = (double)h[l] / (double)count;
    acc = acc + p * log(p);
  }
  return 0.0 - acc;
}

/* RQA measures from the three histograms (reading R5, Marwan et al. 2007 as
 * cited in Sect. 2; Table 3 lists RR, DET, L, Lmax, DIV, L_entr, LAM, TT,
 * Vmax, V_entr):
 *   RR     = RP / n^2, RP = number of recurrence points of the full matrix
 *   DET    = sum_{l>=l_min} l P_D(l) / sum_{l>=1} l P_D(l)
 *   L      = sum_{l>=l_min} l P_D(l) / sum_{l>=l_min} P_D(l)
 *   Lmax   = longest diagonal line of length >= l_min (0 if none);
 *            the line of identity counts when w = 0 (Table 3: Lmax = 732
 *            for 732 vectors)
 *   DIV    = 1 / Lmax
 *   L_entr = -sum_{l>=l_min} p(l) ln p(l), p(l) = P_D(l) / sum_{l>=l_min} P_D
 *   LAM, TT, Vmax, V_entr: the same four with P_V and v_min
 *   W, Wmax, W_entr: the same with P_W and w_min (white vertical lines)
 * Every division is a plain IEEE division (0/0 gives NaN, x/0 gives inf). */
void oracle_measures_rect(const uint64_t* hd, const uint64_t* hv,
                          const uint64_t* hw, int64_t n, int64_t rows, int64_t cols,
                          uint64_t rp, const oracle_settings* st,
                          oracle_measures_t* out);

void oracle_measures(const uint64_t* hd, const uint64_t* hv,
                     const uint64_t* hw, int64_t n, uint64_t rp,
                     const oracle_settings* st, oracle_measures_t* out) {
  oracle_measures_rect(hd, hv, hw, n, n, n, rp, st, out);
}

/* The same measures for an n-by-m (cross) matrix: histograms of length
 * n + 1 (n = the longer side), RR = RP / (rows * cols). */
void oracle_measures_rect(const uint64_t* hd, const uint64_t* hv,
                          const uint64_t* hw, int64_t n, int64_t rows, int64_t cols,
                          uint64_t rp, const oracle_settings* st,
                          oracle_measures_t* out) {
  uint64_t d0, d1, dall0, dall1, v0, v1, vall0, vall1, w0, w1;
  hist_sums(hd, n, st->l_min, &d0, &d1);
  hist_sums(hd, n, 1, &dall0, &dall1);
  hist_sums(hv, n, st->v_min, &v0, &v1);
  hist_sums(hv, n, 1, &vall0, &vall1);
  hist_sums(hw, n, st->w_min, &w0, &w1);
  (void)dall0;
  (void)vall0;
  out->n_vec = rows;
  out->recurrence_points = (int64_t)rp;
  out->rr = (double)rp / ((double)rows * (double)cols);
  out->det = (double)d1 / (double)dall1;
  out->l = (double)d1 / (double)d0;
  out->l_max = hist_max(hd, n, st->l_min);
  out->div = 1.0 / (double)out->l_max;
  out->l_entr = hist_entropy(hd, n, st->l_min, d0);
  out->lam = (double)v1 / (double)vall1;
  out->tt = (double)v1 / (double)v0;
  out->v_max = hist_max(hv, n, st->v_min);
  out->v_entr = hist_entropy(hv, n, st->v_min, v0);
  out->w = (double)w1 / (double)w0;
  out->w_max = hist_max(hw, n, st->w_min);
  out->w_entr = hist_entropy(hw, n, st->w_min, w0);
}
