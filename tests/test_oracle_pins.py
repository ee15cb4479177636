"""Pins for the FP64 oracle: checks against what the paper and the
mathematics fix, not against the oracle itself.

* closed forms: constant series (every pair recurs), linear ramps (band
  matrices whose width follows from the norm), period-p integer sequences
  (lines only on diagonals k = 0 mod p);
* exact distances of hand-made vectors (3-4-5 triangle) and the tie d == eps;
* brute force on tiny inputs: a separately written pure-Python enumeration
  of maximal line segments by their start cell;
* invariants: sum l*P(l) over diagonal and vertical lines equals the number
  of recurrence points, white lines cover the rest of the n^2 cells, the
  matrix is symmetric;
* power-of-two scaling and dyadic translation leave every histogram
  bit-identical;
* measures of hand-made histograms (entropy of k equally likely lengths is
  ln k, and so on);
* Table 3's structural fact: with no Theiler window the line of identity is
  a diagonal line, so Lmax = n (732 for 744 points) and DIV = 1/n.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import NORM_L1, NORM_L2, NORM_MAX, Settings

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
NORMS = (NORM_MAX, NORM_L2, NORM_L1)


def _hist_from_lengths(n, lengths):
    h = np.zeros(n + 1, np.uint64)
    for L in lengths:
        if L > 0:
            h[L] += 1
    return h


def _both_modes(series, st):
    a = oracle.rqa(series, st, mode="matrix")
    b = oracle.rqa(series, st, mode="streaming", threads=2)
    for k in ("hd", "hv", "hw"):
        assert np.array_equal(a[k], b[k]), k
    assert a["rp"] == b["rp"]
    return a


# ---------------------------------------------------------------- distances
@pytest.mark.parametrize("norm,expected", [(NORM_L2, 5.0), (NORM_L1, 7.0),
                                           (NORM_MAX, 4.0)])
def test_distance_345(norm, expected):
    # tau = 2: x_0 = (s0, s2) = (0, 0), x_1 = (s1, s3) = (3, 4)
    s = np.array([0.0, 3.0, 0.0, 4.0])
    assert oracle.distance(s, 0, 1, 2, 2, norm) == expected
    assert oracle.distance(s, 1, 0, 2, 2, norm) == expected


@pytest.mark.parametrize("norm,d", [(NORM_L2, 5.0), (NORM_L1, 7.0), (NORM_MAX, 4.0)])
def test_tie_is_recurrent(norm, d):
    """The neighbourhood is closed: d == eps recurs, d just above does not."""
    s = np.array([0.0, 3.0, 0.0, 4.0])
    R, rp = oracle.matrix(s, Settings(m=2, tau=2, eps=d, norm=norm, theiler=1))
    assert R[0, 1] == 1 and R[1, 0] == 1 and rp == 2
    R, rp = oracle.matrix(s, Settings(m=2, tau=2, eps=np.nextafter(d, 0), norm=norm, theiler=1))
    assert rp == 0


def test_nvec():
    assert oracle.nvec(2000, 3, 2) == 1996
    assert oracle.nvec(1_048_576, 3, 1) == 1_048_574
    assert oracle.nvec(100_000, 5, 3) == 99_988
    assert oracle.nvec(5, 4, 2) == 0


# -------------------------------------------------------------- closed forms
@pytest.mark.parametrize("n,w", [(1, 0), (1, 1), (2, 0), (7, 0), (7, 1), (7, 3),
                                 (30, 2), (30, 29), (30, 30), (30, 45)])
@pytest.mark.parametrize("norm", NORMS)
def test_constant_series(n, w, norm):
    m, tau = 2, 3
    s = synth.constant(n + (m - 1) * tau, 0.7)
    st = Settings(m=m, tau=tau, eps=0.01, norm=norm, theiler=w, l_min=2, v_min=2, w_min=2)
    r = _both_modes(s, st)
    assert r["n"] == n
    hd = _hist_from_lengths(n, [n - abs(k) for k in range(-(n - 1), n) if abs(k) >= w])
    black, white = [], []
    for j in range(n):
        if w == 0:
            black.append(n)
            continue
        black += [j - w + 1, n - j - w]
        lo, hi = max(0, j - w + 1), min(n - 1, j + w - 1)
        white.append(hi - lo + 1)
    assert np.array_equal(r["hd"], hd)
    assert np.array_equal(r["hv"], _hist_from_lengths(n, black))
    assert np.array_equal(r["hw"], _hist_from_lengths(n, white))
    window = sum(n - abs(k) for k in range(-(n - 1), n) if abs(k) < w)
    assert r["rp"] == n * n - window
    if w == 0:
        ms = r["measures"]
        assert ms["rr"] == 1.0
        assert math.isnan(ms["w"])           # no white lines: 0 / 0
        if n >= 2:                           # the one line per column is >= v_min
            # the corner diagonals k = +-(n-1) are single cells, below l_min = 2
            assert ms["det"] == (n * n - 2) / (n * n) and ms["lam"] == 1.0
            assert ms["l_max"] == n and ms["v_max"] == n and ms["tt"] == float(n)
        else:                                # a single cell: shorter than the minima
            assert ms["l_max"] == 0 and ms["v_max"] == 0 and ms["lam"] == 0.0


@pytest.mark.parametrize("norm,reach", [(NORM_MAX, 1), (NORM_L2, 1), (NORM_L1, 0)])
@pytest.mark.parametrize("w", [0, 1, 2])
def test_linear_ramp_band(norm, reach, w):
    """s_t = t, m = 2, tau = 3: x_i = (i, i+3), so d(x_i, x_j) = c |i - j| with
    c = 1 (max), sqrt(2) (L2), 2 (L1).  With eps = 1.5 the matrix is the band
    |i - j| <= reach (minus the Theiler window)."""
    n = 25
    s = np.arange(n + 3, dtype=np.float64)
    st = Settings(m=2, tau=3, eps=1.5, norm=norm, theiler=w, l_min=1, v_min=1, w_min=1)
    r = _both_modes(s, st)
    ks = [k for k in range(-(n - 1), n) if w <= abs(k) <= reach]
    assert np.array_equal(r["hd"], _hist_from_lengths(n, [n - abs(k) for k in ks]))
    black, white = [], []
    for j in range(n):
        col = [1 if (w <= abs(i - j) <= reach) else 0 for i in range(n)]
        # runs of the explicit column, counted by boundaries
        edges = [0] + [i for i in range(1, n) if col[i] != col[i - 1]] + [n]
        for a, b in zip(edges[:-1], edges[1:]):
            (black if col[a] else white).append(b - a)
    assert np.array_equal(r["hv"], _hist_from_lengths(n, black))
    assert np.array_equal(r["hw"], _hist_from_lengths(n, white))


@pytest.mark.parametrize("p", [2, 3, 5])
@pytest.mark.parametrize("m,tau", [(1, 1), (3, 2)])
@pytest.mark.parametrize("w", [0, 1, 4])
@pytest.mark.parametrize("norm", NORMS)
def test_periodic_sequence(p, m, tau, w, norm):
    """s_t = t mod p, eps = 0.5: distinct embedded vectors differ by >= 1 in
    the first coordinate, so R_ij = [i = j mod p] and |i - j| >= w.  Every
    diagonal k = 0 mod p is one full line of length n - |k|; every vertical
    line has length 1; white lines are the gaps between recurrences."""
    n = 40
    s = synth.periodic(n + (m - 1) * tau, p, offset=1)
    st = Settings(m=m, tau=tau, eps=0.5, norm=norm, theiler=w, l_min=2, v_min=2, w_min=2)
    r = _both_modes(s, st)
    ks = [k for k in range(-(n - 1), n) if k % p == 0 and abs(k) >= w]
    assert np.array_equal(r["hd"], _hist_from_lengths(n, [n - abs(k) for k in ks]))
    ones = sum(1 for i in range(n) for j in range(n) if (i - j) % p == 0 and abs(i - j) >= w)
    assert r["rp"] == ones
    hv = np.zeros(n + 1, np.uint64)
    hv[1] = ones
    assert np.array_equal(r["hv"], hv)
    white = []
    for j in range(n):
        rows = [i for i in range(n) if (i - j) % p == 0 and abs(i - j) >= w]
        prev = -1
        for i in rows + [n]:
            white.append(i - prev - 1)
            prev = i
    assert np.array_equal(r["hw"], _hist_from_lengths(n, white))
    ms = r["measures"]
    assert ms["lam"] == 0.0 and ms["v_max"] == 0
    short = sum(1 for k in ks if n - abs(k) < 2)
    assert ms["det"] == (ones - short) / ones


# ---------------------------------------------------------------- brute force
def _brute(series, m, tau, eps, norm, w):
    """Independent restatement: explicit vectors, explicit distances, and
    lines found as maximal segments identified by their first cell."""
    N = len(series)
    n = N - (m - 1) * tau
    vec = [[series[i + k * tau] for k in range(m)] for i in range(n)]

    def dist(a, b):
        diffs = [a[k] - b[k] for k in range(m)]
        if norm == NORM_MAX:
            return max(abs(d) for d in diffs)
        if norm == NORM_L1:
            return sum(abs(d) for d in diffs)
        return math.sqrt(sum(d * d for d in diffs))

    R = [[1 if abs(i - j) >= w and dist(vec[i], vec[j]) <= eps else 0
          for j in range(n)] for i in range(n)]

    def inside(i, j):
        return 0 <= i < n and 0 <= j < n

    hd = np.zeros(n + 1, np.uint64)
    hv = np.zeros(n + 1, np.uint64)
    hw = np.zeros(n + 1, np.uint64)
    for i in range(n):
        for j in range(n):
            # diagonal line of 1s starting at (i, j)
            if R[i][j] and not (inside(i - 1, j - 1) and R[i - 1][j - 1]):
                L = 0
                while inside(i + L, j + L) and R[i + L][j + L]:
                    L += 1
                hd[L] += 1
            # vertical line of value v starting at (i, j)
            v = R[i][j]
            if not (i > 0 and R[i - 1][j] == v):
                L = 0
                while i + L < n and R[i + L][j] == v:
                    L += 1
                (hv if v else hw)[L] += 1
    rp = sum(map(sum, R))
    return hd, hv, hw, rp


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("norm", NORMS)
@pytest.mark.parametrize("w", [0, 1, 3])
def test_brute_force_tiny(seed, norm, w):
    rng = np.random.default_rng(seed)
    N = int(rng.integers(2, 26))
    m = int(rng.integers(1, 4))
    tau = int(rng.integers(1, 3))
    if N - (m - 1) * tau < 1:
        m, tau = 1, 1
    s = rng.standard_normal(N)
    eps = float(rng.uniform(0.3, 1.5))
    st = Settings(m=m, tau=tau, eps=eps, norm=norm, theiler=w)
    r = _both_modes(s, st)
    hd, hv, hw, rp = _brute(list(s), m, tau, eps, norm, w)
    assert r["rp"] == rp
    assert np.array_equal(r["hd"], hd)
    assert np.array_equal(r["hv"], hv)
    assert np.array_equal(r["hw"], hw)


def test_brute_force_dyadic_ties():
    """Dyadic values: many pairs sit exactly at d == eps."""
    for seed in range(4):
        s = synth.dyadic(24, seed, levels=4, scale_log2=-1)
        for norm in NORMS:
            st = Settings(m=2, tau=1, eps=0.5, norm=norm, theiler=1)
            r = _both_modes(s, st)
            hd, hv, hw, rp = _brute(list(s), 2, 1, 0.5, norm, 1)
            assert r["rp"] == rp and np.array_equal(r["hd"], hd)
            assert np.array_equal(r["hv"], hv) and np.array_equal(r["hw"], hw)


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("gen", ["logistic", "ar1", "lorenz"])
@pytest.mark.parametrize("norm", NORMS)
def test_invariants(gen, norm):
    N = 700
    s = {"logistic": lambda: synth.logistic(N, 7),
         "ar1": lambda: synth.ar1(N, 7, 0.9),
         "lorenz": lambda: synth.lorenz_x(N, 7, discard=2000)}[gen]()
    st = Settings(m=3, tau=2, eps=0.35 * float(np.std(s)), norm=norm, theiler=1,
                  l_min=1, v_min=1, w_min=1)
    R, rp = oracle.matrix(s, st)
    assert np.array_equal(R, R.T)
    r = _both_modes(s, st)
    n = r["n"]
    L = np.arange(n + 1, dtype=np.uint64)
    assert int((L * r["hd"]).sum()) == rp == r["rp"]
    assert int((L * r["hv"]).sum()) == rp
    assert int((L * r["hw"]).sum()) == n * n - rp
    # each column holds runs that alternate in colour: the counts differ by <= 1
    assert abs(int(r["hv"].sum()) - int(r["hw"].sum())) <= n
    ms = r["measures"]
    assert ms["det"] == 1.0 and ms["lam"] == 1.0      # l_min = v_min = 1
    assert ms["rr"] == rp / (n * n)


@pytest.mark.parametrize("k", [-7, -1, 3, 12])
@pytest.mark.parametrize("norm", NORMS)
def test_power_of_two_scaling(k, norm):
    s = synth.ar1(300, 11, 0.8)
    st = Settings(m=3, tau=1, eps=0.6, norm=norm, theiler=2)
    a = oracle.rqa(s, st, mode="matrix")
    b = oracle.rqa(s * 2.0 ** k, Settings(m=3, tau=1, eps=0.6 * 2.0 ** k, norm=norm,
                                          theiler=2), mode="matrix")
    for key in ("hd", "hv", "hw"):
        assert np.array_equal(a[key], b[key])


@pytest.mark.parametrize("norm", NORMS)
def test_dyadic_translation(norm):
    s = synth.dyadic(200, 5, levels=16, scale_log2=-2)
    st = Settings(m=2, tau=3, eps=1.0, norm=norm, theiler=1)
    a = oracle.rqa(s, st, mode="matrix")
    b = oracle.rqa(s + 37.25, st, mode="matrix")
    for key in ("hd", "hv", "hw"):
        assert np.array_equal(a[key], b[key])


def test_theiler_window_zero_vs_one():
    s = synth.logistic(300, 3)
    a = oracle.rqa(s, Settings(m=2, tau=1, eps=0.05, theiler=0), mode="matrix")
    b = oracle.rqa(s, Settings(m=2, tau=1, eps=0.05, theiler=1), mode="matrix")
    n = a["n"]
    assert a["rp"] - b["rp"] == n               # exactly the line of identity
    d = a["hd"].astype(np.int64) - b["hd"].astype(np.int64)
    assert d[n] == 1 and (d[:n] == 0).all()     # the LOI is one line of length n


# ------------------------------------------------------------------ measures
def test_measures_hand_histograms():
    n = 10
    hd = _hist_from_lengths(n, [1, 1, 2, 3])
    hv = _hist_from_lengths(n, [2, 2, 4, 4, 1])
    hw = _hist_from_lengths(n, [5, 6, 7])
    st = Settings(m=1, tau=1, eps=1.0, l_min=2, v_min=2, w_min=2)
    rp = 1 + 1 + 2 + 3
    ms = oracle.measures(hd, hv, hw, n, rp, st)
    assert ms["rr"] == rp / 100
    assert ms["det"] == 5 / 7                  # lines >= 2 carry 5 of 7 points
    assert ms["l"] == 2.5 and ms["l_max"] == 3 and ms["div"] == 1 / 3
    assert ms["l_entr"] == pytest.approx(math.log(2), rel=1e-15)
    assert ms["lam"] == 12 / 13 and ms["tt"] == 3.0 and ms["v_max"] == 4
    assert ms["v_entr"] == pytest.approx(math.log(2), rel=1e-15)
    assert ms["w"] == 6.0 and ms["w_max"] == 7
    assert ms["w_entr"] == pytest.approx(math.log(3), rel=1e-15)


def test_measures_empty():
    n = 5
    z = np.zeros(n + 1, np.uint64)
    ms = oracle.measures(z, z, z, n, 0, Settings(m=1, tau=1, eps=1.0))
    assert ms["rr"] == 0.0 and ms["l_max"] == 0 and ms["div"] == math.inf
    assert math.isnan(ms["det"]) and math.isnan(ms["l"])
    assert ms["l_entr"] == 0.0 and math.copysign(1.0, ms["l_entr"]) == 1.0


def test_table3_lmax_is_n_without_theiler_window():
    """Table 3: Lmax = 732 for 744-point series (no Theiler window), so the
    line of identity counts as a diagonal line; DIV = 1/732 prints as 0.001."""
    g = json.load(open(os.path.join(GOLDEN, "table3_structure.json")))
    N, span = g["series_points"], g["embedding_span"]
    for m, tau in [(4, 4), (5, 3), (13, 1)]:
        assert (m - 1) * tau == span
        s = synth.ar1(N, 42, 0.9)
        st = Settings(m=m, tau=tau, eps=0.4, norm=NORM_L2, theiler=0)
        r = oracle.rqa(s, st, mode="matrix")
        ms = r["measures"]
        assert r["n"] == g["l_max"] == ms["l_max"]
        assert round(ms["div"], g["div_print_decimals"]) == g["div_printed"]


def test_full_size_golden_is_consistent():
    """The stored full-size oracle result (AR(1), n = 1,048,574, w = 1) obeys
    the invariants of any recurrence matrix: every recurrence point lies on
    one diagonal and one vertical line, white lines fill the remaining
    cells, the two triangles mirror each other, and the measures follow from
    the histograms' stored totals."""
    path = os.path.join(GOLDEN, "ar1_n1m_oracle.json")
    g = json.load(open(path))
    n, rp = g["n_vec"], g["rp"]
    assert n == 1_048_574
    assert g["hd"]["weighted_sum"] == rp == g["hv"]["weighted_sum"]
    assert g["hw"]["weighted_sum"] == n * n - rp
    assert g["hd"]["sum"] % 2 == 0            # w = 1: mirrored triangles
    assert g["measures"]["recurrence_points"] == rp
    assert g["measures"]["rr"] == rp / (n * n)
    assert g["measures"]["l_max"] == g["hd"]["max_len"]


def test_sine_golden_is_consistent():
    """The stored oracle result for the paper's runtime series (Sect. 8.2:
    sin over 1,000,001 points, m = 2, tau = 2, eps = 1, no Theiler window)
    obeys the same invariants, plus those of w = 0: the line of identity is
    one diagonal line of length n, which is also the longest (Table 3's
    Lmax = n reading), and the other diagonal lines come in mirrored pairs."""
    g = json.load(open(os.path.join(GOLDEN, "sine_paper_oracle.json")))
    n, rp = g["n_vec"], g["rp"]
    assert n == 999_999 and g["N"] == 1_000_001
    assert g["params"] == dict(m=2, tau=2, norm=1, eps=1.0, theiler=0, l_min=2, v_min=2,
                               w_min=2)
    assert g["hd"]["weighted_sum"] == rp == g["hv"]["weighted_sum"]
    assert g["hw"]["weighted_sum"] == n * n - rp
    assert g["hd"]["max_len"] == n == g["measures"]["l_max"]
    assert (g["hd"]["sum"] - 1) % 2 == 0      # all lines but the LOI are mirrored
    assert all(v % 2 == 0 for v in g["hd"]["head"].values())
    assert g["measures"]["recurrence_points"] == rp
    assert g["measures"]["rr"] == rp / (n * n)
    assert g["measures"]["div"] == 1.0 / n


@pytest.mark.parametrize("norm", NORMS)
@pytest.mark.parametrize("m,tau", [(1, 1), (3, 2)])
def test_time_reversal_on_dyadic_data(norm, m, tau):
    """Reversing the series maps x_i to x_{n-1-i} with its coordinates in
    reverse order, i.e. rotates the matrix by 180 degrees; on dyadic data
    every distance is exact, so all three histograms are unchanged."""
    s = synth.dyadic(700, 9, levels=6, scale_log2=-2)
    st = Settings(m=m, tau=tau, eps=0.75, norm=norm, theiler=1)
    a = oracle.rqa(s, st)
    b = oracle.rqa(s[::-1].copy(), st)
    for k in ("hd", "hv", "hw"):
        assert np.array_equal(a[k], b[k]), k
