"""Pins for the oracle's line detection over a precomputed binary matrix
(Sect. 9: users asked for the quantitative analysis of precomputed
recurrence matrices).  Checked against what the definition fixes:

* a separately written pure-Python enumeration of maximal lines by their
  first cell on random tiny rectangles of several densities;
* closed forms: all-ones and all-zero rectangles, a checkerboard (every
  even diagonal one full line, every column alternating single cells), and
  period-p diagonal stripes;
* the matrix of a series fed back in gives that series' RQA result (the
  separately pinned RQA oracle), and the cross matrix of two series gives
  their cross recurrence result;
* the Theiler window masks |i - j| < w exactly as for a computed matrix.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import NORM_L1, NORM_L2, NORM_MAX, Settings

ST = Settings(m=1, tau=1, eps=1.0, norm=NORM_MAX, theiler=0)


def _brute(R, w):
    rows, cols = len(R), len(R[0])
    C = [[1 if R[i][j] and abs(i - j) >= w else 0 for j in range(cols)] for i in range(rows)]
    L = max(rows, cols)
    hd, hv, hw = (np.zeros(L + 1, np.uint64) for _ in range(3))
    for i in range(rows):
        for j in range(cols):
            if C[i][j] and not (i > 0 and j > 0 and C[i - 1][j - 1]):
                ln = 0
                while i + ln < rows and j + ln < cols and C[i + ln][j + ln]:
                    ln += 1
                hd[ln] += 1
            v = C[i][j]
            if not (i > 0 and C[i - 1][j] == v):
                ln = 0
                while i + ln < rows and C[i + ln][j] == v:
                    ln += 1
                (hv if v else hw)[ln] += 1
    return hd, hv, hw, sum(map(sum, C))


@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("w", [0, 1, 3])
def test_brute_force_tiny(seed, w):
    rng = np.random.default_rng(900 + seed)
    rows, cols = (int(x) for x in rng.integers(1, 19, 2))
    R = (rng.random((rows, cols)) < rng.uniform(0.1, 0.9)).astype(np.uint8)
    r = oracle.matrix_rqa(R, Settings(m=1, tau=1, eps=1.0, norm=0, theiler=w))
    hd, hv, hw, rp = _brute(R.tolist(), w)
    assert r["rp"] == rp and (r["n"], r["cols"]) == (rows, cols)
    assert np.array_equal(r["hd"], hd)
    assert np.array_equal(r["hv"], hv)
    assert np.array_equal(r["hw"], hw)
    assert r["measures"]["rr"] == rp / (rows * cols)


@pytest.mark.parametrize("rows,cols", [(1, 1), (1, 9), (9, 1), (7, 12), (12, 7), (10, 10)])
def test_all_ones_and_zeros(rows, cols):
    L = max(rows, cols)
    r = oracle.matrix_rqa(np.ones((rows, cols)), ST)
    hd = np.zeros(L + 1, np.uint64)
    for k in range(-(rows - 1), cols):
        hd[min(rows, cols - k) - max(0, -k)] += 1
    hv = np.zeros(L + 1, np.uint64)
    hv[rows] = cols
    assert np.array_equal(r["hd"], hd) and np.array_equal(r["hv"], hv)
    assert r["hw"].sum() == 0 and r["rp"] == rows * cols
    z = oracle.matrix_rqa(np.zeros((rows, cols)), ST)
    hw = np.zeros(L + 1, np.uint64)
    hw[rows] = cols
    assert z["hd"].sum() == 0 and z["hv"].sum() == 0 and np.array_equal(z["hw"], hw)
    assert z["rp"] == 0


@pytest.mark.parametrize("rows,cols", [(8, 8), (9, 14), (15, 6)])
def test_checkerboard(rows, cols):
    R = ((np.arange(rows)[:, None] + np.arange(cols)[None, :]) % 2 == 0).astype(np.uint8)
    r = oracle.matrix_rqa(R, ST)
    L = max(rows, cols)
    hd = np.zeros(L + 1, np.uint64)
    for k in range(-(rows - 1), cols):
        if k % 2 == 0:                     # cell (i, i + k) is 1 iff k is even
            hd[min(rows, cols - k) - max(0, -k)] += 1
    ones = int(R.sum())
    assert np.array_equal(r["hd"], hd)
    assert r["hv"][1] == ones and r["hv"].sum() == ones
    assert r["hw"][1] == rows * cols - ones and r["hw"].sum() == rows * cols - ones


@pytest.mark.parametrize("p", [2, 3, 7])
def test_diagonal_stripes(p):
    rows, cols = 23, 31
    R = ((np.arange(cols)[None, :] - np.arange(rows)[:, None]) % p == 0).astype(np.uint8)
    r = oracle.matrix_rqa(R, ST)
    L = max(rows, cols)
    hd = np.zeros(L + 1, np.uint64)
    for k in range(-(rows - 1), cols):
        if k % p == 0:
            hd[min(rows, cols - k) - max(0, -k)] += 1
    assert np.array_equal(r["hd"], hd)
    assert r["hv"][1] == r["rp"] == int(R.sum())


@pytest.mark.parametrize("norm", [NORM_MAX, NORM_L2, NORM_L1])
@pytest.mark.parametrize("w", [0, 1, 4])
def test_series_matrix_gives_rqa(norm, w):
    s = synth.logistic(260, 17)
    st = Settings(m=3, tau=2, eps=0.15, norm=norm, theiler=w, l_min=2, v_min=2, w_min=3)
    R, _ = oracle.matrix(s, st)
    a = oracle.rqa(s, st)
    b = oracle.matrix_rqa(R, st)          # the window again: idempotent
    c = oracle.matrix_rqa(R, Settings(m=3, tau=2, eps=0.15, norm=norm, theiler=0,
                                      l_min=2, v_min=2, w_min=3))
    for k in ("hd", "hv", "hw"):
        assert np.array_equal(a[k], b[k]) and np.array_equal(a[k], c[k]), k
    assert a["measures"]["det"] == b["measures"]["det"]
    assert a["measures"]["rr"] == b["measures"]["rr"]


def test_cross_matrix_gives_cross_rqa():
    x, y = synth.ar1(70, 1, 0.9), synth.ar1(55, 2, 0.9)
    st = Settings(m=2, tau=2, eps=0.6, norm=NORM_L2, theiler=2)
    n1, n2 = len(x) - 2, len(y) - 2
    R = np.array([[oracle.cross_distance(x, y, i, j, 2, 2, NORM_L2) <= 0.6 for j in range(n2)]
                  for i in range(n1)], dtype=np.uint8)
    a = oracle.cross_rqa(x, y, st)
    b = oracle.matrix_rqa(R, st)          # the window is applied by matrix_rqa
    for k in ("hd", "hv", "hw"):
        assert np.array_equal(a[k], b[k]), k
    assert a["rp"] == b["rp"] and a["measures"]["rr"] == b["measures"]["rr"]
