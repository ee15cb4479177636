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

struct Sums {
  uint64_t count = 0;  // number of lines with length >= lo
  uint64_t cells = 0;  // sum of their lengths
};

Sums sums_from(const uint64_t* h, int64_t n, int64_t lo) {
  Sums s;
  for (int64_t l = lo < 1 ? 1 : lo; l <= n; ++l) {
    s.count += h[l];
    s.cells += static_cast<uint64_t>(l) * h[l];
  }
  return s;
}

int64_t longest(const uint64_t* h, int64_t n, int64_t lo) {
  const int64_t floor_len = lo < 1 ? 1 : lo;
  int64_t l = n;
  while (l >= floor_len && h[l] == 0) --l;
  return l >= floor_len ? l : 0;
}

// Shannon entropy (natural log) of the lengths >= lo, terms in ascending l.
double entropy(const uint64_t* h, int64_t n, int64_t lo, uint64_t count) {
  double acc = 0.0;
  const double total = static_cast<double>(count);
  for (int64_t l = lo < 1 ? 1 : lo; l <= n; ++l) {
    if (!h[l]) continue;
    const double p = static_cast<double>(h[l]) / total;
    const double term = p * std::log(p);
    acc = acc + term;
  }
  return 0.0 - acc;
}

}  // namespace

void measures_from_histograms_rect(const uint64_t* hd, const uint64_t* hv, const uint64_t* hw,
                                   int64_t n, int64_t rows, int64_t cols, int32_t l_min,
                                   int32_t v_min, int32_t w_min, rqa_measures_t* out);

void measures_from_histograms(const uint64_t* hd, const uint64_t* hv, const uint64_t* hw,
                              int64_t n, int32_t l_min, int32_t v_min, int32_t w_min,
                              rqa_measures_t* out) {
  measures_from_histograms_rect(hd, hv, hw, n, n, n, l_min, v_min, w_min, out);
}

void measures_from_histograms_rect(const uint64_t* hd, const uint64_t* hv, const uint64_t* hw,
                                   int64_t n, int64_t rows, int64_t cols, int32_t l_min,
                                   int32_t v_min, int32_t w_min, rqa_measures_t* out) {
  const Sums d = sums_from(hd, n, l_min), d_all = sums_from(hd, n, 1);
  const Sums v = sums_from(hv, n, v_min), v_all = sums_from(hv, n, 1);
  const Sums w = sums_from(hw, n, w_min);
  // every recurrence point lies on exactly one vertical line
  const uint64_t rp = v_all.cells;
  out->n_vec = rows;
  out->recurrence_points = static_cast<int64_t>(rp);
  const double nn = static_cast<double>(rows) * static_cast<double>(cols);
  out->rr = static_cast<double>(rp) / nn;
  out->det = static_cast<double>(d.cells) / static_cast<double>(d_all.cells);
  out->l = static_cast<double>(d.cells) / static_cast<double>(d.count);
  out->l_max = longest(hd, n, l_min);
  out->div = 1.0 / static_cast<double>(out->l_max);
  out->l_entr = entropy(hd, n, l_min, d.count);
  out->lam = static_cast<double>(v.cells) / static_cast<double>(v_all.cells);
  out->tt = static_cast<double>(v.cells) / static_cast<double>(v.count);
  out->v_max = longest(hv, n, v_min);
  out->v_entr = entropy(hv, n, v_min, v.count);
  out->w = static_cast<double>(w.cells) / static_cast<double>(w.count);
  out->w_max = longest(hw, n, w_min);
  out->w_entr = entropy(hw, n, w_min, w.count);
}

}  // namespace rqa
