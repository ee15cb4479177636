"""Pins for the oracle's cross recurrence (Sect. 3.3: the vectors of two
series on the two axes of the matrix; Sect. 4.2: the non-symmetric matrix
has 2N - 1 diagonals).  Checked against what the definition fixes, not
against the cross code itself:

* the same series on both axes reduces to ordinary RQA (Sect. 3.3 notes this
  for crqa), whose oracle is pinned separately, for every norm and Theiler
  window, histograms and measures alike;
* a separately written pure-Python enumeration of the n1 x n2 matrix and its
  maximal lines by their start cell, on tiny rectangles of both shapes;
* closed forms: two period-p integer sequences recur exactly on the
  diagonals j - i = -offset (mod p), every such diagonal is one line of its
  full length and every column holds single-cell lines p apart;
* invariants: sum l P(l) over diagonal and vertical lines is the number of
  recurrence points, white lines cover the rest of the n1 * n2 cells, and
  swapping the two series transposes the matrix, which keeps the diagonal
  histogram;
* RR is the recurrence points over n1 * n2.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import NORM_L1, NORM_L2, NORM_MAX, Settings

NORMS = (NORM_MAX, NORM_L2, NORM_L1)


def _vec(s, i, m, tau):
    return [s[i + k * tau] for k in range(m)]


def _dist(a, b, norm):
    d = [abs(x - y) for x, y in zip(a, b)]
    if norm == NORM_MAX:
        return max(d)
    if norm == NORM_L1:
        return sum(d)
    return math.sqrt(sum(x * x for x in d))


def _brute(s1, s2, m, tau, eps, norm, w):
    """The n1 x n2 cross matrix from the definition and its lines, each
    found from its first cell (pure Python, independent of the oracle)."""
    n1 = len(s1) - (m - 1) * tau
    n2 = len(s2) - (m - 1) * tau
    R = [[1 if abs(i - j) >= w and
          _dist(_vec(s1, i, m, tau), _vec(s2, j, m, tau), norm) <= eps else 0
          for j in range(n2)] for i in range(n1)]
    L = max(n1, n2)
    hd, hv, hw = (np.zeros(L + 1, np.uint64) for _ in range(3))
    for i in range(n1):
        for j in range(n2):
            if R[i][j] and not (i > 0 and j > 0 and R[i - 1][j - 1]):
                ln = 0
                while i + ln < n1 and j + ln < n2 and R[i + ln][j + ln]:
                    ln += 1
                hd[ln] += 1
            v = R[i][j]
            if not (i > 0 and R[i - 1][j] == v):
                ln = 0
                while i + ln < n1 and R[i + ln][j] == v:
                    ln += 1
                (hv if v else hw)[ln] += 1
    return hd, hv, hw, sum(map(sum, R)), n1, n2


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("norm", NORMS)
@pytest.mark.parametrize("w", [0, 1, 3])
def test_cross_brute_force_tiny(seed, norm, w):
    rng = np.random.default_rng(100 + seed)
    m = int(rng.integers(1, 4))
    tau = int(rng.integers(1, 3))
    N1 = int(rng.integers((m - 1) * tau + 1, 24))
    N2 = int(rng.integers((m - 1) * tau + 1, 24))
    s1 = rng.standard_normal(N1)
    s2 = rng.standard_normal(N2) * 0.8 + 0.1
    eps = float(rng.uniform(0.3, 1.5))
    st = Settings(m=m, tau=tau, eps=eps, norm=norm, theiler=w)
    r = oracle.cross_rqa(s1, s2, st, threads=2)
    hd, hv, hw, rp, n1, n2 = _brute(list(s1), list(s2), m, tau, eps, norm, w)
    assert (r["n"], r["cols"]) == (n1, n2)
    assert r["rp"] == rp
    assert np.array_equal(r["hd"], hd)
    assert np.array_equal(r["hv"], hv)
    assert np.array_equal(r["hw"], hw)
    assert r["measures"]["rr"] == rp / (n1 * n2)


def test_cross_brute_force_dyadic_ties():
    """Dyadic values: many cross pairs sit exactly at d == eps."""
    for seed in range(4):
        s1 = synth.dyadic(21, seed, levels=4, scale_log2=-1)
        s2 = synth.dyadic(17, seed + 50, levels=4, scale_log2=-1)
        for norm in NORMS:
            st = Settings(m=2, tau=1, eps=0.5, norm=norm, theiler=1)
            r = oracle.cross_rqa(s1, s2, st)
            hd, hv, hw, rp, _, _ = _brute(list(s1), list(s2), 2, 1, 0.5, norm, 1)
            assert r["rp"] == rp and np.array_equal(r["hd"], hd)
            assert np.array_equal(r["hv"], hv) and np.array_equal(r["hw"], hw)


@pytest.mark.parametrize("norm", NORMS)
@pytest.mark.parametrize("w", [0, 1, 4])
@pytest.mark.parametrize("gen", ["logistic", "ar1"])
def test_same_series_is_rqa(norm, w, gen):
    s = synth.logistic(300, 7) if gen == "logistic" else synth.ar1(300, 8, 0.9)
    st = Settings(m=3, tau=2, eps=0.2 if gen == "logistic" else 0.6, norm=norm, theiler=w,
                  l_min=2, v_min=3, w_min=2)
    a = oracle.rqa(s, st)
    b = oracle.cross_rqa(s, s, st)
    n = a["n"]
    for k in ("hd", "hv", "hw"):
        assert np.array_equal(a[k], b[k]), k
    assert a["rp"] == b["rp"] and b["cols"] == n
    for f, v in a["measures"].items():
        vb = b["measures"][f]
        assert (math.isnan(v) and math.isnan(vb)) or v == vb, f


@pytest.mark.parametrize("p,off", [(3, 0), (4, 1), (5, 3), (2, 1)])
@pytest.mark.parametrize("m,tau", [(1, 1), (3, 2)])
@pytest.mark.parametrize("norm", NORMS)
def test_periodic_closed_form(p, off, m, tau, norm):
    N1, N2 = 61, 47
    s1 = synth.periodic(N1, p)
    s2 = synth.periodic(N2, p, offset=off)
    n1, n2 = N1 - (m - 1) * tau, N2 - (m - 1) * tau
    r = oracle.cross_rqa(s1, s2, Settings(m=m, tau=tau, eps=0.5, norm=norm, theiler=0))
    L = max(n1, n2)
    # x_i == y_j iff i = j + off (mod p); other vectors differ by >= 1
    hd = np.zeros(L + 1, np.uint64)
    for k in range(-(n1 - 1), n2):
        if (k + off) % p == 0:
            hd[min(n1, n2 - k) - max(0, -k)] += 1
    hv = np.zeros(L + 1, np.uint64)
    hw = np.zeros(L + 1, np.uint64)
    rp = 0
    for j in range(n2):
        r0 = (j + off) % p               # the first recurrent row of column j
        ones = 0 if r0 >= n1 else (n1 - 1 - r0) // p + 1
        rp += ones
        hv[1] += ones                    # p >= 2: no two recurrent rows touch
        if ones == 0:
            hw[n1] += 1
            continue
        if r0 > 0:
            hw[r0] += 1
        hw[p - 1] += ones - 1
        tail = n1 - 1 - (r0 + (ones - 1) * p)
        if tail > 0:
            hw[tail] += 1
    assert r["rp"] == rp
    assert np.array_equal(r["hd"], hd)
    assert np.array_equal(r["hv"], hv)
    assert np.array_equal(r["hw"], hw)
    assert r["measures"]["rr"] == rp / (n1 * n2)
    assert r["measures"]["l_max"] == int(np.nonzero(hd)[0].max())


@pytest.mark.parametrize("p,w", [(3, 2), (4, 5)])
def test_periodic_diagonals_with_theiler(p, w):
    """A Theiler window removes exactly the diagonals |k| < w."""
    N1, N2 = 50, 66
    s1, s2 = synth.periodic(N1, p), synth.periodic(N2, p, offset=1)
    r = oracle.cross_rqa(s1, s2, Settings(m=2, tau=1, eps=0.5, norm=NORM_L2, theiler=w))
    n1, n2 = N1 - 1, N2 - 1
    hd = np.zeros(max(n1, n2) + 1, np.uint64)
    rp = 0
    for k in range(-(n1 - 1), n2):
        if (k + 1) % p == 0 and abs(k) >= w:
            ln = min(n1, n2 - k) - max(0, -k)
            hd[ln] += 1
            rp += ln
    assert r["rp"] == rp and np.array_equal(r["hd"], hd)


@pytest.mark.parametrize("norm", NORMS)
@pytest.mark.parametrize("w", [0, 2])
def test_invariants_and_transpose(norm, w):
    s1 = synth.lorenz_x(400, 3)[:400]
    s2 = synth.lorenz_x(333, 4)
    st = Settings(m=3, tau=3, eps=0.5, norm=norm, theiler=w)
    a = oracle.cross_rqa(s1, s2, st)
    b = oracle.cross_rqa(s2, s1, st)
    n1, n2 = a["n"], a["cols"]
    ln = np.arange(len(a["hd"]), dtype=np.uint64)
    assert int((ln * a["hd"]).sum()) == a["rp"] == int((ln * a["hv"]).sum())
    assert int((ln * a["hw"]).sum()) == n1 * n2 - a["rp"]
    assert a["rp"] == b["rp"] and np.array_equal(a["hd"], b["hd"])
    assert 0 < a["rp"] < n1 * n2


def test_empty_and_single_vector():
    st = Settings(m=3, tau=2, eps=0.5, norm=NORM_L2, theiler=0)
    r = oracle.cross_rqa(np.zeros(5), np.ones(5), st)        # one vector each, far apart
    assert (r["n"], r["cols"], r["rp"]) == (1, 1, 0)
    assert r["hw"][1] == 1 and r["hd"].sum() == 0
    r = oracle.cross_rqa(np.zeros(5), np.zeros(9), st)
    assert r["rp"] == 5 and r["hd"][1] == 5 and r["hv"][1] == 5   # 1 x 5, all recurrent
