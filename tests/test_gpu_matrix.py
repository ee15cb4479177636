"""GPU parity for line detection over a precomputed binary matrix (Sect. 9):
rqa_run_matrix against the oracle's matrix_rqa, histograms and measures bit
for bit.  This is also the hook for adversarial line patterns that series
rarely produce: lines longer than the shared-memory bins, lines that cross
every strip, all-black strips, word-misaligned columns and checkerboards.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import _diff, assert_same_measures, gpu_settings, oracle_settings

import paper_2402_16853_b300 as gp

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _default_tiles(monkeypatch):
    monkeypatch.delenv("RQA_TILE_WARPS", raising=False)


def check_matrix(R, w=0, l_min=2, v_min=2, w_min=2):
    want = oracle.matrix_rqa(R, oracle_settings(1, 1, 1.0, 0, w, l_min, v_min, w_min))
    r = gp.RQA(gpu_settings(1, 1, 1.0, 0, w, l_min, v_min, w_min))
    meas = r.run_matrix(R)
    hd, hv, hw = r.histograms()
    assert np.array_equal(hd, want["hd"]), _diff("diag", hd, want["hd"])
    assert np.array_equal(hv, want["hv"]), _diff("vert", hv, want["hv"])
    assert np.array_equal(hw, want["hw"]), _diff("white", hw, want["hw"])
    assert_same_measures(meas, want["measures"])
    st = r.stats()
    assert st["mode"] == 2 and st["n_vec"] == R.shape[0] and st["n_cols"] == R.shape[1]
    return r, want


@pytest.mark.parametrize("rows,cols", [(1, 1), (1, 33), (33, 1), (31, 32), (32, 31), (64, 64),
                                       (129, 127), (500, 37), (37, 500), (1000, 1001),
                                       (2100, 1300)])
@pytest.mark.parametrize("p", [0.05, 0.5, 0.95])
def test_random_shapes(rows, cols, p):
    rng = np.random.default_rng(rows * 7 + cols)
    check_matrix((rng.random((rows, cols)) < p).astype(np.uint8))


@pytest.mark.parametrize("w", [0, 1, 5, 64, 3000])
def test_theiler_window(w):
    rng = np.random.default_rng(w)
    check_matrix((rng.random((1500, 1800)) < 0.7).astype(np.uint8), w=w)


@pytest.mark.parametrize("rows,cols", [(3000, 2500), (2500, 3000), (1100, 1100)])
def test_all_ones_long_lines(rows, cols):
    """Lines far longer than the 1,023 shared-memory bins and black across
    whole strips (the all-black descriptor path)."""
    check_matrix(np.ones((rows, cols), np.uint8))


def test_all_zeros():
    check_matrix(np.zeros((1234, 2345), np.uint8))


@pytest.mark.parametrize("rows,cols", [(700, 900), (901, 333)])
def test_checkerboard(rows, cols):
    R = ((np.arange(rows)[:, None] + np.arange(cols)[None, :]) % 2 == 0).astype(np.uint8)
    check_matrix(R)


@pytest.mark.parametrize("L", [1022, 1023, 1024, 1025, 2047])
def test_runs_at_bin_edges(L):
    """Diagonal and vertical runs of lengths around the bin count, placed to
    cross strip and word boundaries."""
    R = np.zeros((2600, 2600), np.uint8)
    for t in range(L):
        R[37 + t, 301 + t] = 1             # one diagonal line of length L
    R[100:100 + L, 2000] = 1               # one vertical line of length L
    R[5, 5:5 + min(L, 2590)] = 1           # a horizontal line: single-cell verticals
    check_matrix(R)


@pytest.mark.parametrize("warps", [1, 2, 3, 5, 8])
def test_warps_per_strip(monkeypatch, warps):
    monkeypatch.setenv("RQA_TILE_WARPS", str(warps))
    rng = np.random.default_rng(warps)
    R = (rng.random((1700, 2900)) < 0.6).astype(np.uint8)
    R[:, 1000:1300] = 1                    # black band across strip edges
    check_matrix(R)


@pytest.mark.parametrize("p", [2, 3, 33])
def test_diagonal_stripes(p):
    rows, cols = 1800, 1500
    R = ((np.arange(cols)[None, :] - np.arange(rows)[:, None]) % p == 0).astype(np.uint8)
    check_matrix(R)


def test_series_plot_round_trip():
    """A series' recurrence plot fed back as a matrix gives the series' RQA."""
    s = synth.lorenz_x(1600, 21)
    st = gpu_settings(4, 2, 0.6, 1, 3)
    a = gp.RQA(st)
    ma = a.run(s)
    plot = gp.recurrence_plot(st, s)
    b = gp.RQA(st)
    mb = b.run_matrix(plot)
    for u, v in zip(a.histograms(), b.histograms()):
        assert np.array_equal(u, v)
    assert_same_measures(mb, ma)


def test_cross_plot_round_trip():
    x, y = synth.ar1(1300, 3, 0.9), synth.ar1(1700, 4, 0.9)
    st = gpu_settings(3, 1, 0.5, 0, 2)
    a = gp.RQA(st)
    ma = a.run_cross(x, y)
    packed = gp.cross_recurrence_plot(st, x, y, packed=True)
    b = gp.RQA(st)
    mb = b.run_matrix(packed, cols=len(y) - 2)
    for u, v in zip(a.histograms(), b.histograms()):
        assert np.array_equal(u, v)
    assert_same_measures(mb, ma)


def test_device_matrix_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    R = (rng.random((1200, 1000)) < 0.4).astype(np.uint8)
    words = gp.pack_matrix(R)
    want = oracle.matrix_rqa(R, oracle_settings(1, 1, 1.0, 0, 1))
    r = gp.RQA(gpu_settings(1, 1, 1.0, 0, 1))
    t = torch.from_numpy(words.view(np.int32)).cuda()
    meas = r.run_matrix(t, cols=1000)
    assert np.array_equal(r.histogram(0), want["hd"])
    assert np.array_equal(r.histogram(2), want["hw"])
    assert_same_measures(meas, want["measures"])


def test_errors():
    r = gp.RQA(gpu_settings(1, 1, 1.0, 0, 0))
    r.run_matrix(np.ones((40, 40), np.uint8))
    with pytest.raises(gp.RQAError) as ei:
        r.sample([0], [1])                 # a given matrix has no decisions
    assert ei.value.status == 1
    with pytest.raises(gp.RQAError) as ei:
        r.run_matrix(np.zeros((0, 1), np.uint32), cols=5)
    assert ei.value.status == 2            # no rows
    meas = r.run_matrix(np.ones((3, 4), np.uint8))   # the handle still works
    assert meas["recurrence_points"] == 12


def test_large_random_bit_exact():
    rng = np.random.default_rng(11)
    R = (rng.random((12000, 9000)) < 0.3).astype(np.uint8)
    R[2000:7000, 3000:3400] = 1
    check_matrix(R, w=2)
