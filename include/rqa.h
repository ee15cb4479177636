/*
 * rqa.h -- C ABI of the B300 (sm_103a) recurrence quantification analysis
 * library (librqa_b300.so).
 *
 * The library computes, for a scalar time series, what the PyRQA paper
 * describes as an RQA computation (Sect. 7, Listings 2-4):
 *   1. time-delay embedding with dimension m and delay tau (Sect. 2, Sect. 7.2),
 *   2. the binary recurrence matrix R_ij = [d(x_i, x_j) <= eps and |i-j| >= w]
 *      under the L-infinity, L2 or L1 norm with a fixed radius eps
 *      (Sect. 2, Sect. 7.2 "similarity measure" / FixedRadius) and a Theiler
 *      window w, never materialised,
 *   3. the frequency distributions of diagonal lines, vertical lines and white
 *      vertical lines over the full n x n matrix (Sect. 2, the three line
 *      types; Sect. 4.2, operators I-III), and
 *   4. the measures of Table 3 (RR, DET, L, Lmax, DIV, L_entr, LAM, TT, Vmax,
 *      V_entr) plus W, Wmax, W_entr for white vertical lines.
 * n = N - (m-1)*tau embedded vectors x_i = (s[i], s[i+tau], ..., s[i+(m-1)tau]).
 * Cross recurrence (rqa_run_cross) compares the vectors x_i of one series
 * with the vectors y_j of another (Sect. 3.3): the n1 x n2 matrix
 * C_ij = [d(x_i, y_j) <= eps and |i-j| >= w], with lines along its
 * n1 + n2 - 1 diagonals and down its n2 columns (Sect. 4.2, non-symmetric
 * matrix).
 *
 * Results are exact: every recurrence decision equals the FP64 decision
 * d <= eps computed in the order
 *   L1   d = ((|D0| + |D1|) + ...)      L2  d = sqrt(((D0*D0) + D1*D1) + ...)
 *   Linf d = max_k |Dk|                 Dk = s[i+k*tau] - s[j+k*tau]
 * with no fused multiply-add, so the histograms are integers that do not
 * depend on the hardware, and the measures are computed from them on the
 * host in a fixed order (see rqa_measures_t).
 *
 * Errors: every call returns an rqa_status (RQA_OK = 0); none aborts the
 * process.  rqa_strerror() names a code; rqa_last_error() gives the detail of
 * the last failure on a handle.  The library never falls back to the CPU:
 * without a usable CUDA device, rqa_create() returns RQA_ENODEV.
 *
 * Threading: a handle is used by one thread at a time.  Server handles
 * (rqa_server_*) are safe to call from several threads.
 */
#ifndef RQA_B300_H
#define RQA_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ codes */
typedef enum {
  RQA_OK = 0,
  RQA_EINVAL = 1,    /* invalid settings or arguments                      */
  RQA_ESHORT = 2,    /* fewer than one embedded vector (n < 1)             */
  RQA_ENAN = 3,      /* a series value is NaN or infinite                  */
  RQA_ENOMEM = 4,    /* device allocation failed or over the memory budget */
  RQA_ECUDA = 5,     /* a CUDA call failed; see rqa_last_error()           */
  RQA_ETIMEOUT = 6,  /* a bounded device-side wait gave up                 */
  RQA_PENDING = 7,   /* server: the request has not finished yet           */
  RQA_ENODEV = 8,    /* no CUDA device of compute capability 10.3          */
  RQA_ETOOBIG = 9,   /* n or m beyond the supported maximum                */
  RQA_ENOTFOUND = 10 /* server: unknown ticket                             */
} rqa_status;

typedef enum { RQA_NORM_MAX = 0, RQA_NORM_L2 = 1, RQA_NORM_L1 = 2 } rqa_norm;

/* How pair distances are evaluated on the GPU.  Both give the same, exact
 * result; they differ in speed.
 *   RQA_PREC_AUTO / RQA_PREC_FP32_RECHECK: FP32 distances on centred, scaled
 *     FP32 copies of the vectors; pairs whose FP32 margin |eps - d| (|eps^2 -
 *     d^2| for L2) is within a proven error band are re-decided in FP64 with
 *     the exact operation order above.
 *   RQA_PREC_FP64: every pair in FP64 (the plain comparison path). */
typedef enum {
  RQA_PREC_AUTO = 0,
  RQA_PREC_FP32_RECHECK = 1,
  RQA_PREC_FP64 = 2
} rqa_precision;

/* Analysis parameters: the paper's Settings (Sect. 7.2, Listing 2). */
typedef struct {
  int32_t m;        /* embedding_dimension, 1..RQA_MAX_M                     */
  int32_t tau;      /* time_delay, >= 1                                      */
  double eps;       /* FixedRadius radius, finite and > 0                    */
  int32_t norm;     /* rqa_norm (similarity_measure)                         */
  int32_t theiler;  /* Theiler window w >= 0: cells with |i-j| < w are 0     */
  int32_t l_min;    /* min_diagonal_line_length, >= 1                        */
  int32_t v_min;    /* min_vertical_line_length, >= 1                        */
  int32_t w_min;    /* min_white_vertical_line_length, >= 1                  */
  int32_t precision;     /* rqa_precision                                    */
  double band_override;  /* < 0: automatic band (exact).  >= 0: the FP32
                            recheck band as a fraction of eps (of eps^2 for
                            L2); +inf rechecks every pair.  A band below the
                            proven bound may give inexact results, which
                            rqa_stats_t.exact reports.                       */
} rqa_settings;

#define RQA_MAX_M 10
/* Largest series (embedded vectors).  A single series whose strip-boundary
 * descriptors would exceed a fifth of the device's memory (RQA_DESC_BUDGET
 * bytes if that variable is set) runs its CTA strips in groups, carrying the
 * open run of every row and diagonal from group to group (Sect. 4.1), so
 * that its descriptor memory is bounded by the budget rather than growing
 * as n^2; rqa_stats_t reports the groups and bytes. */
#define RQA_MAX_N ((int64_t)1 << 24)
/* Cross recurrence and precomputed matrices: rows and columns each (their
 * strips are not grouped). */
#define RQA_MAX_N_RECT ((int64_t)1 << 22)

/* Measures (the paper's RQAResult, Sect. 7.4, Table 3).  With P_D, P_V, P_W
 * the histograms of diagonal, vertical and white vertical line lengths over
 * the full matrix (line of identity included when w = 0) and RP the number
 * of recurrence points:
 *   rr = RP / (n*n)  (cross recurrence: RP / (n1*n2); n_vec = n1)
 *   det = sum_{l>=l_min} l P_D(l) / sum_{l>=1} l P_D(l)
 *   l = sum_{l>=l_min} l P_D(l) / sum_{l>=l_min} P_D(l)
 *   l_max = longest diagonal line >= l_min (0 if none), div = 1 / l_max
 *   l_entr = 0 - sum_{l>=l_min, P_D(l)>0} p ln p, p = P_D(l) / sum_{l>=l_min} P_D,
 *            accumulated in ascending l
 *   lam, tt, v_max, v_entr: the same with P_V and v_min
 *   w, w_max, w_entr: the same with P_W and w_min (no white analogue of det)
 * Integer sums are exact (uint64); each quotient is one IEEE division, so
 * 0/0 gives NaN and x/0 gives +inf.                                          */
typedef struct {
  double rr, det, l, div, l_entr, lam, tt, v_entr, w, w_entr;
  int64_t l_max, v_max, w_max, n_vec, recurrence_points;
} rqa_measures_t;

/* Diagnostics of the last run on a handle (not part of the result). */
typedef struct {
  int64_t n_vec;          /* rows: embedded vectors of the (first) series     */
  int64_t pairs;          /* unique off-window pairs i < j, j - i >= max(w,1);
                             cross recurrence: cells with |i - j| >= w        */
  int64_t rechecks;       /* pairs re-decided in FP64                         */
  double band;            /* recheck band used, in units of eps (eps^2 L2)    */
  double band_bound;      /* proven sufficient band, same units               */
  int32_t precision_used; /* rqa_precision actually run                       */
  int32_t exact;          /* 1 if band >= band_bound (or FP64 path)           */
  int32_t strip_width;    /* columns per CTA strip                            */
  int32_t warps_per_cta;
  int32_t cols_per_lane;
  int32_t ctas;           /* persistent CTAs launched                         */
  float kernel_ms;        /* device time of the tile kernel (events)          */
  float total_ms;         /* device time of all kernels of the run            */
  int64_t h2d_bytes;      /* host-to-device bytes copied by the run           */
  int64_t d2h_bytes;      /* device-to-host bytes copied by the run           */
  int32_t launches;       /* kernels launched by the run                      */
  int32_t mode;           /* 0 RQA, 1 cross recurrence, 2 precomputed matrix  */
  int64_t n_cols;         /* columns: n_vec for RQA, n2 for cross recurrence  */
  int64_t band_rows;      /* RQA: rows per band when strips were split into
                             row bands to fill the GPU (0: not split)         */
  int64_t desc_bytes;     /* device bytes of strip-boundary descriptors (and
                             group carries) the run held at once              */
  int64_t desc_bytes_all_strips; /* the same for all strips at once          */
  int32_t strip_groups;   /* 1, or the strip groups a long single series ran
                             in to keep desc_bytes within the budget          */
  int32_t strips_per_group;
} rqa_stats_t;

typedef struct rqa_handle rqa_handle;

/* Create a computation (RQAComputation.create, Sect. 7.3).  Validates the
 * settings (RQA_EINVAL) and selects the current CUDA device (RQA_ENODEV if
 * there is none of compute capability 10.3).  *out receives the handle. */
int rqa_create(const rqa_settings* settings, rqa_handle** out);

/* Replace the handle's analysis parameters (a new Settings object for the
 * same computation object, Sect. 7.2-7.3) without giving up its device
 * buffers, streams or loaded kernels, so that a sequence of series with
 * different parameters runs on one handle.  RQA_EINVAL (settings kept) if
 * they are invalid; the previous result is forgotten. */
int rqa_set_settings(rqa_handle* h, const rqa_settings* settings);

/* Run on a host series of n FP64 values (RQAComputation.run, Sect. 7.4).
 * The library copies the series to the device (pageable or pinned host
 * memory both work) and blocks until the result is ready.  Device buffers
 * are owned by the handle and reused by later runs of the same or smaller n. */
int rqa_run(rqa_handle* h, const double* host_series, int64_t n);

/* The run of Sect. 7.4 (RQAComputation.run) on a series already in device
 * memory (e.g. a torch CUDA tensor), ordered on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream).  The
 * caller keeps the series alive and unmodified until the call returns; the
 * call returns when the results are on the host.  dev_series must be 8-byte
 * aligned memory the handle's device can read (its own device memory,
 * managed memory or mapped pinned host memory); anything else, pageable
 * host memory included, is refused with RQA_EINVAL before a kernel runs.
 * The call waits for its results, so it must not be issued on a stream that
 * is being captured into a CUDA graph; from the second consecutive call with
 * the same series length, pointer and stream the library replays a graph of
 * its own, and the series' values, like the settings', are read anew by
 * every call. */
int rqa_run_device(rqa_handle* h, const double* dev_series, int64_t n,
                   void* cuda_stream);

/* Cross recurrence (Sect. 3.3; Sect. 4.2's non-symmetric matrix) of two host
 * series: rows are the n1 = n_x - (m-1)*tau vectors of x, columns the
 * n2 = n_y - (m-1)*tau vectors of y, cells with |i - j| < theiler are 0.
 * The handle's settings apply to both series, which share one FP32
 * centring and scaling so that the result is exact as for rqa_run.  After
 * the call rqa_measures, rqa_histogram (entries l = 0..max(n1, n2)),
 * rqa_stats and rqa_sample_decisions (i < n1, j < n2) describe the cross
 * matrix.  The same series twice gives the result of rqa_run. */
int rqa_run_cross(rqa_handle* h, const double* host_x, int64_t n_x,
                  const double* host_y, int64_t n_y);
/* The same with both series in device memory, ordered on cuda_stream. */
int rqa_run_cross_device(rqa_handle* h, const double* dev_x, int64_t n_x,
                         const double* dev_y, int64_t n_y, void* cuda_stream);
/* Lines and measures of a precomputed binary matrix (Sect. 9 lists the
 * analysis of precomputed recurrence matrices as a user request): `rows` x
 * `cols` cells, row-major and bit-packed as rqa_recurrence_plot writes them
 * (row r occupies ceil(cols/32) uint32 words, bit b of word w is column
 * 32 w + b; bits past the last column are ignored).  The matrix is taken as
 * given, except that cells with |i - j| < theiler count as 0; diagonal lines
 * run along all rows + cols - 1 diagonals and vertical / white lines down the
 * cols columns, as for cross recurrence, with RR = RP / (rows * cols) and
 * histograms of max(rows, cols) + 1 entries.  The handle's m, tau, eps, norm
 * and precision are not used.  rows, cols in 1..RQA_MAX_N_RECT; the library copies
 * the host bits (rows * ceil(cols/32) * 4 bytes) to the device. */
int rqa_run_matrix(rqa_handle* h, const uint32_t* host_bits, int64_t rows,
                   int64_t cols);
/* The same with the bits in device memory (4-byte aligned), ordered on
 * cuda_stream. */
int rqa_run_matrix_device(rqa_handle* h, const uint32_t* dev_bits, int64_t rows,
                          int64_t cols, void* cuda_stream);
/* Copy the measures of the last successful run: the members of the
 * paper's RQAResult object (Sect. 7.4, e.g. determinism; Table 3 lists
 * them), computed from the three line-length distributions as defined
 * above (the paper defers the definitions to Marwan et al. 2007, Sect. 2).
 * RQA_EINVAL if there is no successful run. */
int rqa_measures(const rqa_handle* h, rqa_measures_t* out);

/* Copy a histogram of the last run -- one of the frequency distributions of
 * the three line types that Sect. 2 names (diagonal lines and vertical lines
 * of recurrence points, white vertical lines of non-recurrence points):
 * kind 0 = diagonal lines, 1 = vertical lines, 2 = white vertical lines;
 * entry l = number of lines of length l,
 * l = 0..n (entry 0 is always 0; cross recurrence: l = 0..max(n1, n2)).
 * cap = capacity of `out` in entries; *len receives n + 1.  RQA_EINVAL if cap < n + 1 (then *len still says how
 * many entries are needed). */
int rqa_histogram(const rqa_handle* h, int32_t kind, uint64_t* out,
                  int64_t cap, int64_t* len);

/* Diagnostics of the last run (rqa_stats_t); the paper has no counterpart. */
int rqa_stats(const rqa_handle* h, rqa_stats_t* out);

/* Evaluate individual recurrence decisions R_ij of the last run's series
 * with the same device decision code as the tile kernel (FP32 test with the
 * FP64 recheck band, or FP64).  i, j, out: host arrays of `count` entries;
 * out[q] = R_{i[q], j[q]} (0 or 1).  For spot checks at sizes where the full
 * matrix cannot be enumerated on the CPU.  RQA_EINVAL after rqa_run_matrix,
 * whose cells are the caller's. */
int rqa_sample_decisions(rqa_handle* h, const int64_t* i, const int64_t* j,
                         int64_t count, uint8_t* out);

/* End a computation made by rqa_create (Sect. 7.3): frees its device
 * buffers and the handle.  NULL is ignored. */
void rqa_destroy(rqa_handle* h);

/* Failures are status codes here where PyRQA raises exceptions (Sect. 6:
 * an absent compute device makes its execution throw).  rqa_strerror()
 * names a code (a static string; "unknown status" for other values);
 * rqa_last_error() gives the detail of the last failure on a handle (valid
 * until the handle's next call). */
const char* rqa_strerror(int status);
const char* rqa_last_error(const rqa_handle* h);

/* ---------------------------------------------------- without allocation
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot let the library allocate device memory -- programs that hand the
 * whole GPU to their own memory pool, services that must keep a fixed device
 * footprint from start-up, or code paths where cudaMalloc's implicit
 * synchronisation of the device would stall unrelated streams.
 *
 * rqa_run_noalloc() computes the three histograms of one series exactly as
 * rqa_run_device() does, but keeps every intermediate buffer in one static
 * device array of RQA_NOALLOC_SCRATCH_BYTES that each GPU loading the library
 * holds until the process exits; it calls no cudaMalloc/cudaFree.
 *   settings    analysis parameters (validated as by rqa_create)
 *   dev_series  n_points FP64 values in device memory, read on cuda_stream
 *               (8-byte aligned and readable by the current device, as for
 *               rqa_run_device; else RQA_EINVAL before anything runs)
 *   dev_hist    device buffer of 3 * (n_vec + 1) uint64 (8-byte aligned) that receives the
 *               diagonal, vertical and white-vertical histograms, laid out
 *               like rqa_histogram (kind * (n_vec + 1) + length)
 *   cuda_stream cudaStream_t (NULL: legacy default stream); the call returns
 *               after the work on it has finished
 * Series of more than RQA_NOALLOC_MAX_N embedded vectors are rejected with
 * RQA_ETOOBIG before anything is launched.  All calls share the one array:
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race and must be serialised by the caller.  The call always blocks until
 * its work on cuda_stream has finished (it reads a status word back), so it
 * must not be called on a stream that is being captured into a CUDA graph.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress), which also loads the module holding the array if
 * CUDA's lazy loading has not yet done so; rqa_preload_kernels() performs
 * that look-up ahead of time.  settings->theiler at or above n acts as n
 * (every cell removed).  settings->band_override must be negative (the
 * automatic, exact band) or +inf (every pair re-decided in FP64); other
 * values are refused with RQA_EINVAL, since this call has no statistics
 * through which to report an inexact result.  rqa_noalloc_last_error()
 * describes the last failure of the calling thread. */
#define RQA_NOALLOC_MAX_N ((int64_t)32768)
#define RQA_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
int rqa_run_noalloc(const rqa_settings* settings, const double* dev_series,
                    int64_t n_points, uint64_t* dev_hist, void* cuda_stream);
const char* rqa_noalloc_last_error(void);

/* ------------------------------------------------------ recurrence plot
 * The paper's RecurrencePlotComputation (Sect. 7.3, Table 2): a window of the
 * recurrence matrix, rows [i0, i0 + rows) and columns [j0, j0 + cols), written
 * bit-packed to host memory: plot row r occupies ceil(cols / 32) uint32
 * words, bit b of word w is R(i0 + r, j0 + 32 w + b); cells outside the
 * n x n matrix are 0.  The decisions are exactly those of rqa_run (FP32 with
 * the FP64 recheck band, or FP64).  The buffer needs rows * ceil(cols/32) * 4
 * bytes (at most 4 GiB).  rqa_plot_last_error() describes the last failure
 * of the calling thread. */
int rqa_recurrence_plot(const rqa_settings* settings, const double* host_series,
                        int64_t n_points, int64_t i0, int64_t j0, int64_t rows,
                        int64_t cols, uint32_t* out_bits);
/* The same window of the cross-recurrence matrix of x (rows) and y
 * (columns); cells outside the n1 x n2 matrix are 0. */
int rqa_cross_recurrence_plot(const rqa_settings* settings, const double* host_x,
                              int64_t n_x, const double* host_y, int64_t n_y,
                              int64_t i0, int64_t j0, int64_t rows, int64_t cols,
                              uint32_t* out_bits);
const char* rqa_plot_last_error(void);

/* --------------------------------------------------------------- autotuner
 * Sect. 9 plans the automatic selection of the best-performing
 * implementation at runtime.  rqa_autotune() times whole runs (device time
 * from the first copy to the last) for each tile shape -- CTA-strip width
 * (1, 2, 4 and 8 warps), columns per lane (4, or 2 for FP32 distances) and
 * row-band height -- on one series
 * -- host_series of n_points values, or a built-in z-scored AR(1) series of
 * n_points values when host_series is NULL -- as RQA (cross = 0) or as the
 * cross recurrence of the series with itself (cross = 1), and records the
 * fastest shape for the class (RQA or cross, m, norm, FP64 or not,
 * ceil(log2 n)).  Every later run of that class in the process (single,
 * cross, batched, served) uses the recorded shape; results do not depend on
 * it.  *best_warps receives the width; ms_per_width (4 floats, may be NULL)
 * the best of two timed runs per width at four columns per lane.
 * rqa_autotune_clear() forgets every recorded shape.  The environment
 * variables RQA_TILE_WARPS (1..8) and RQA_TILE_COLS (2 or 4) override the
 * table.  rqa_autotune_last_error() describes the last failure of the
 * calling thread. */
int rqa_autotune(const rqa_settings* settings, const double* host_series,
                 int64_t n_points, int32_t cross, int32_t* best_warps,
                 float* ms_per_width);
/* The full tile-shape search for the same class: every strip width at four
 * and (FP32 distances only) two columns per lane, and, when the winner runs
 * in row bands, the band height of the size rule halved and doubled.  The
 * winner is recorded for the class as by rqa_autotune; *best_warps,
 * *best_cols (2 or 4), *best_band_scale (-1, 0, +1) and *best_ms (whole-run
 * device time) receive it (any pointer may be NULL).  rqa_autotune searches
 * this space too but reports only the width. */
int rqa_autotune_shape(const rqa_settings* settings, const double* host_series,
                       int64_t n_points, int32_t cross, int32_t* best_warps,
                       int32_t* best_cols, int32_t* best_band_scale, float* best_ms);
/* Write the recorded choices to a text file (one class per line: kind m norm
 * f64 log2n warps cols band_scale), or read such a file and record its
 * entries, overriding the classes it names (*entries, may be NULL, receives
 * their number).  A malformed file records nothing and returns RQA_EINVAL. */
int rqa_autotune_save(const char* path);
int rqa_autotune_load(const char* path, int32_t* entries);
void rqa_autotune_clear(void);
const char* rqa_autotune_last_error(void);
/* ------------------------------------------------------ failure self-test
 * The paper has no counterpart.  The tile kernel's warps hand carries to
 * each other through bounded waits (about 2 s of SM clock); a wait that runs
 * out raises an abort flag and the series fails with RQA_ETIMEOUT instead of
 * hanging the GPU.  rqa_selftest_bounded_wait() exercises exactly that wait
 * on a counter that nothing raises: *status receives the status the waiting
 * warp reported (RQA_ETIMEOUT when the mechanism works) and *cycles_waited
 * the SM cycles it waited.  Returns RQA_OK if the wait gave up and raised the
 * abort flag; the CUDA context stays usable afterwards. */
int rqa_selftest_bounded_wait(int32_t* status, int64_t* cycles_waited);
/* The same mechanism inside the real tile kernel: runs the handle's series
 * (host_series, n_points values; the handle's settings must be m = 3, L2,
 * FP32 distances) through a test instantiation of the tile kernel with eight
 * warps per CTA strip, no row bands and a wait limit of 10^6 SM cycles, in
 * which warp `warp` (0..6) of every CTA stops handing its row and diagonal
 * carries to warp `warp` + 1 from its `from_handover`-th hand-over (>= 1)
 * on.  The waiting warp gives up, raises the CTA's abort flag (every other
 * wait of the CTA then returns), and the series fails: the call returns
 * RQA_ETIMEOUT if the strips reach that hand-over (a series too short to
 * reach it returns RQA_OK).  No wait is unbounded and nothing faults; the
 * handle stays usable, and its next run is exact. */
int rqa_selftest_ring_timeout(rqa_handle* h, const double* host_series,
                              int64_t n_points, int32_t warp,
                              int32_t from_handover);
/* ---------------------------------------------------------- ALU probe
 * The paper has no counterpart.  rqa_probe_alu() measures, on the current
 * device, the throughput of one FP32 operation of the distance loop with
 * every SM fully occupied by independent dependency chains: kind 0 fma.f32,
 * 1 fma.f32x2, 2 add.f32, 3 sub.f32x2, 4 max.f32.  *ops_per_s counts one
 * operation per lane (two for the packed f32x2 forms), the unit of the
 * roofline's per-pair operation count; the benchmark divides by the larger of
 * this and SMs x 128 lanes x clock.  Takes a few milliseconds. */
int rqa_probe_alu(int32_t kind, double* ops_per_s);
/* ------------------------------------------------------------ preloading
 * The paper has no counterpart.  CUDA loads kernels lazily, at their first
 * launch, and a load can stall the whole context while other work runs.
 * rqa_preload_kernels() loads every kernel a run can launch (all tile kernel
 * instantiations and the preparation and merge kernels) into the current
 * device's context and resolves the device address of rqa_run_noalloc's
 * static scratch array, once per process; later calls return at once.
 * *loaded (may be NULL) receives the number of kernels it loaded.
 * rqa_server_create calls it.  RQA_ENODEV without an sm_103 device,
 * RQA_ECUDA if a load fails. */
int rqa_preload_kernels(int32_t* loaded);
/* ----------------------------------------------------------------- batched
 * Many independent series in one submission: the work of all series is one
 * queue of (series, strip) items processed by persistent CTAs, one launch
 * per (m, norm) class, all launches captured in one CUDA graph that later
 * calls with the same shapes replay.  settings[q] and series[q] (host
 * pointers to lens[q] FP64 values) describe series q; out[q] receives its
 * measures and status[q] its status.  The call returns RQA_OK if every
 * series succeeded, else the first failing status. */
typedef struct rqa_batch rqa_batch;

int rqa_batch_create(rqa_batch** out);
int rqa_batch_run(rqa_batch* b, const rqa_settings* settings,
                  const double* const* series, const int64_t* lens,
                  int32_t count, rqa_measures_t* out, int32_t* status);
/* The batched run in the shape of a single call (no batch object to
 * manage): series q (lens[q] FP64 values in host memory) is analysed with
 * settings[q] -- `settings` holds one entry per series, so a uniform batch
 * repeats one set of parameters -- and out[q] receives its measures (zeroed
 * if the series failed).  The device work is ordered on `stream` (a
 * cudaStream_t, NULL = the library's own stream): it starts after work
 * already queued there and the call returns once the results are on the
 * host.  The work queue, CUDA graph and device buffers are those of
 * rqa_batch_run, held in a batch object that belongs to the calling host
 * thread and is reused by its later calls (repeated shapes replay the
 * captured graph) until rqa_run_batch_release() frees it.  Returns RQA_OK
 * if every series succeeded, else the first failing status. */
int rqa_run_batch(const rqa_settings* settings, const double* const* series,
                  const int64_t* lens, int32_t count, rqa_measures_t* out,
                  void* stream);
/* Free the calling thread's rqa_run_batch buffers (a later call recreates
 * them). */
void rqa_run_batch_release(void);
/* Histogram of series q of the last batch run (same layout as
 * rqa_histogram). */
int rqa_batch_histogram(const rqa_batch* b, int32_t q, int32_t kind,
                        uint64_t* out, int64_t cap, int64_t* len);
int rqa_batch_stats(const rqa_batch* b, rqa_stats_t* out);
void rqa_batch_destroy(rqa_batch* b);

/* ----------------------------------------------------------------- served
 * The paper has no counterpart: it runs one computation at a time
 * (Sect. 7.3-7.4).  This is the same computation served to many callers
 * with continuous batching.  Requests are admitted while their device memory
 * (series, embedded vectors, descriptors, histograms) fits in
 * mem_budget_bytes and a slot is free; admitted requests are batched into
 * launch epochs as they arrive, so work of requests that arrive while others
 * run overlaps on the device.  Each request keeps its own histograms and
 * boundary state on the device until it completes. */
typedef struct rqa_server rqa_server;

/* Create a server with a device-memory budget (bytes) and at most
 * max_slots requests in flight; *out receives it.  Loads every kernel first
 * (rqa_preload_kernels).  RQA_ENODEV without an sm_103 device. */
int rqa_server_create(size_t mem_budget_bytes, int32_t max_slots,
                      rqa_server** out);
/* Copy the series and queue the request (an RQAComputation.run of Sect. 7.4
 * with its own Settings); *ticket identifies it.  RQA_EINVAL for invalid
 * settings, RQA_ESHORT / RQA_ETOOBIG for series that cannot run, RQA_ENOMEM
 * if the request alone exceeds the server's budget. */
int rqa_submit(rqa_server* s, const rqa_settings* settings,
               const double* host_series, int64_t n, uint64_t* ticket);
/* RQA_PENDING until done; then the request's status, with *out filled on
 * RQA_OK (the request's RQAResult, Sect. 7.4).  A finished ticket may be
 * polled until rqa_release(); RQA_ENOTFOUND for an unknown ticket. */
int rqa_poll(rqa_server* s, uint64_t ticket, rqa_measures_t* out);
/* Block until the ticket finishes or timeout_ms passes (RQA_PENDING). */
int rqa_wait(rqa_server* s, uint64_t ticket, int64_t timeout_ms,
             rqa_measures_t* out);
/* Forget a finished ticket, or cancel a queued one. */
int rqa_release(rqa_server* s, uint64_t ticket);
/* Server counters: admitted, completed, queued, in_flight, bytes_in_use,
 * epochs (launches).  Any pointer may be NULL. */
int rqa_server_counters(rqa_server* s, int64_t* admitted, int64_t* completed,
                        int64_t* queued, int64_t* in_flight,
                        int64_t* bytes_in_use, int64_t* epochs);
/* Stop the server: waits for the requests in flight, drops queued ones and
 * frees every buffer.  NULL is ignored. */
void rqa_server_destroy(rqa_server* s);

#ifdef __cplusplus
}
#endif
#endif /* RQA_B300_H */
