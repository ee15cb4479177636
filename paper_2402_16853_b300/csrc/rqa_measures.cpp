// rqa_measures.cpp -- RQA measures from the three line-length histograms
// (Table 3 of the PyRQA paper; definitions after Marwan et al. 2007, which
// the paper cites in Sect. 2).  The formulas and the evaluation order are
// the ones documented for rqa_measures_t in include/rqa.h; this file is
// compiled with -ffp-contract=off so every product and sum is rounded on its
// own and the result does not depend on the compiler's choice of FMA.
#include <cmath>
#include <cstdint>

#include "../../include/rqa.h"

namespace rqa {

namespace {

// One pass over a histogram h[1..last]: the sums the measures need for
// lengths >= lo (and the total over all lengths) and the longest such length.
struct Scan {
  const uint64_t* h = nullptr;
  int64_t last = 0;        // bins above last are zero
  int64_t lo = 1;          // first length counted (l_min, v_min or w_min, at least 1)
  uint64_t count = 0;      // lines with length >= lo
  uint64_t cells = 0;      // sum of their lengths
  uint64_t cells_all = 0;  // sum of the lengths of all lines
  int64_t longest = 0;     // longest length >= lo (0 if none)
};

Scan scan(const uint64_t* h, int64_t last, int64_t lo) {
  Scan s;
  s.h = h;
  s.last = last;
  s.lo = lo < 1 ? 1 : lo;
  for (int64_t l = 1; l <= last; ++l) {
    const uint64_t v = h[l];
    if (!v) continue;
    s.cells_all += static_cast<uint64_t>(l) * v;
    if (l < s.lo) continue;
    s.count += v;
    s.cells += static_cast<uint64_t>(l) * v;
    s.longest = l;
  }
  return s;
}

// Shannon entropy (natural log) of the lengths >= lo, terms in ascending l
// (a second pass over the same bins, so no list of them is kept).  Within
// one histogram equal counts give the same p = v / total and so the same
// term; the terms of small counts, which most bins hold, are computed once.
double entropy(const Scan& s) {
  double acc = 0.0;
  const double total = static_cast<double>(s.count);
  constexpr uint64_t kMemo = 64;
  double memo[kMemo];
  uint64_t have = 0;  // bit v: memo[v] holds the term of count v
  for (int64_t l = s.lo; l <= s.last; ++l) {
    const uint64_t v = s.h[l];
    if (!v) continue;
    double term;
    if (v < kMemo && ((have >> v) & 1u)) {
      term = memo[v];
    } else {
      const double p = static_cast<double>(v) / total;
      term = p * std::log(p);
      if (v < kMemo) {
        memo[v] = term;
        have |= 1ull << v;
      }
    }
    acc = acc + term;
  }
  return 0.0 - acc;
}

}  // namespace

void measures_from_histograms_rect(const uint64_t* hd, const uint64_t* hv, const uint64_t* hw,
                                   int64_t n, int64_t rows, int64_t cols, int32_t l_min,
                                   int32_t v_min, int32_t w_min, rqa_measures_t* out);
void measures_from_histograms_last(const uint64_t* hd, const uint64_t* hv, const uint64_t* hw,
                                   const int64_t last[3], int64_t rows, int64_t cols,
                                   int32_t l_min, int32_t v_min, int32_t w_min,
                                   rqa_measures_t* out);

void measures_from_histograms(const uint64_t* hd, const uint64_t* hv, const uint64_t* hw,
                              int64_t n, int32_t l_min, int32_t v_min, int32_t w_min,
                              rqa_measures_t* out) {
  measures_from_histograms_rect(hd, hv, hw, n, n, n, l_min, v_min, w_min, out);
}

void measures_from_histograms_rect(const uint64_t* hd, const uint64_t* hv, const uint64_t* hw,
                                   int64_t n, int64_t rows, int64_t cols, int32_t l_min,
                                   int32_t v_min, int32_t w_min, rqa_measures_t* out) {
  const int64_t last[3] = {n, n, n};
  measures_from_histograms_last(hd, hv, hw, last, rows, cols, l_min, v_min, w_min, out);
}

void measures_from_histograms_last(const uint64_t* hd, const uint64_t* hv, const uint64_t* hw,
                                   const int64_t last[3], int64_t rows, int64_t cols,
                                   int32_t l_min, int32_t v_min, int32_t w_min,
                                   rqa_measures_t* out) {
  // bins above last[t] are zero and add nothing to any sum
  const Scan d = scan(hd, last[0], l_min), v = scan(hv, last[1], v_min),
             w = scan(hw, last[2], w_min);
  // every recurrence point lies on exactly one vertical line
  const uint64_t rp = v.cells_all;
  out->n_vec = rows;
  out->recurrence_points = static_cast<int64_t>(rp);
  const double nn = static_cast<double>(rows) * static_cast<double>(cols);
  out->rr = static_cast<double>(rp) / nn;
  out->det = static_cast<double>(d.cells) / static_cast<double>(d.cells_all);
  out->l = static_cast<double>(d.cells) / static_cast<double>(d.count);
  out->l_max = d.longest;
  out->div = 1.0 / static_cast<double>(out->l_max);
  out->l_entr = entropy(d);
  out->lam = static_cast<double>(v.cells) / static_cast<double>(v.cells_all);
  out->tt = static_cast<double>(v.cells) / static_cast<double>(v.count);
  out->v_max = v.longest;
  out->v_entr = entropy(v);
  out->w = static_cast<double>(w.cells) / static_cast<double>(w.count);
  out->w_max = w.longest;
  out->w_entr = entropy(w);
}

}  // namespace rqa
