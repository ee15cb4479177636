"""GPU parity with CTA strips split into row bands (items (strip, band)):
column runs joined across bands, diagonals walked through items left and
top, row runs untouched.  RQA_BAND_ROWS forces band heights small enough
for the materialised oracle; the automatic rule is exercised at 20,000 and
(in test_gpu_fullsize.py) 100,000 points."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same_measures, check_parity, gpu_settings

import paper_2402_16853_b300 as gp

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _clean(monkeypatch):
    monkeypatch.delenv("RQA_TILE_WARPS", raising=False)
    monkeypatch.delenv("RQA_BAND_ROWS", raising=False)


@pytest.mark.parametrize("rows", [32, 64, 160, 1024])
@pytest.mark.parametrize("warps", [1, 2, 5, 8])
@pytest.mark.parametrize("n", [700, 2500])
def test_band_heights_and_widths(monkeypatch, rows, warps, n):
    monkeypatch.setenv("RQA_BAND_ROWS", str(rows))
    monkeypatch.setenv("RQA_TILE_WARPS", str(warps))
    s = synth.lorenz_x(n + 6, 700 + n, discard=1000)
    r, st, _ = check_parity(s, m=4, tau=2, eps=0.6, norm=0, theiler=2)
    assert st["band_rows"] == (rows if rows < n else 0)


@pytest.mark.parametrize("norm", [0, 1, 2])
@pytest.mark.parametrize("w", [0, 1, 3, 100])
def test_norms_and_windows(monkeypatch, norm, w):
    monkeypatch.setenv("RQA_BAND_ROWS", "96")
    monkeypatch.setenv("RQA_TILE_WARPS", "2")
    s = synth.ar1(1800, 50 + norm + w, 0.9)
    check_parity(s, m=3, tau=2, eps=0.5, norm=norm, theiler=w)


@pytest.mark.parametrize("w", [0, 1, 7])
def test_constant_series_runs_through_every_band(monkeypatch, w):
    """Every cell outside the window recurs: column runs span all bands,
    diagonals are black through every item."""
    monkeypatch.setenv("RQA_BAND_ROWS", "64")
    monkeypatch.setenv("RQA_TILE_WARPS", "3")
    check_parity(np.full(1500, 0.25), m=2, tau=1, eps=0.1, norm=1, theiler=w)


@pytest.mark.parametrize("p", [2, 5, 37])
def test_periodic(monkeypatch, p):
    monkeypatch.setenv("RQA_BAND_ROWS", "128")
    check_parity(synth.periodic(2000, p), m=3, tau=1, eps=0.5, norm=2, theiler=0)


def test_exact_ties_and_fp64(monkeypatch):
    monkeypatch.setenv("RQA_BAND_ROWS", "64")
    s = synth.dyadic(1400, 3, levels=4, scale_log2=-1)
    check_parity(s, m=2, tau=1, eps=0.5, norm=1, theiler=1)
    check_parity(synth.ar1(1300, 9, 0.9), m=3, tau=1, eps=0.5, norm=1, theiler=1,
                 precision=gp.PREC_FP64)


def test_batch_with_banded_series(monkeypatch):
    """Series of one batch run banded and unbanded side by side."""
    monkeypatch.setenv("RQA_BAND_ROWS", "96")
    rng = np.random.default_rng(4)
    settings, series = [], []
    for q in range(12):
        L = int(rng.integers(50, 1800))
        settings.append(gp.Settings(m=2, tau=1, eps=0.3, norm=q % 3, theiler=q % 3))
        series.append(synth.ar1(L, 100 + q, 0.9))
    b = gp.Batch()
    res, st, rc = b.run(settings, series)
    assert rc == 0
    for q, (stg, s) in enumerate(zip(settings, series)):
        want = oracle.rqa(s, oracle.Settings(m=2, tau=1, eps=0.3, norm=q % 3, theiler=q % 3))
        assert np.array_equal(b.histogram(q, 0), want["hd"]), q
        assert np.array_equal(b.histogram(q, 1), want["hv"]), q
        assert np.array_equal(b.histogram(q, 2), want["hw"]), q
        assert_same_measures(res[q], want["measures"])


def test_automatic_bands_n20000():
    s = synth.logistic(20_002, 61)
    want = oracle.rqa(s, oracle.Settings(m=3, tau=1, eps=0.05, norm=1, theiler=1),
                      mode="streaming")
    r = gp.RQA(gpu_settings(3, 1, 0.05, 1, 1))
    meas = r.run(s)
    st = r.stats()
    assert st["band_rows"] > 0            # 40 strips of 512 columns alone are too few
    for got, k in zip(r.histograms(), ("hd", "hv", "hw")):
        assert np.array_equal(got, want[k]), k
    assert_same_measures(meas, want["measures"])


# ---------------------------------------------------------------- cross / matrix
def _cross_check(x, y, **kw):
    want = oracle.cross_rqa(x, y, oracle.Settings(**kw))
    r = gp.RQA(gpu_settings(**kw))
    meas = r.run_cross(x, y)
    for got, k in zip(r.histograms(), ("hd", "hv", "hw")):
        assert np.array_equal(got, want[k]), k
    assert_same_measures(meas, want["measures"])
    return r.stats()


@pytest.mark.parametrize("rows", [32, 96, 512])
@pytest.mark.parametrize("warps", [1, 3, 8])
@pytest.mark.parametrize("n1,n2", [(900, 2400), (2400, 900), (1000, 1000)])
def test_cross_bands(monkeypatch, rows, warps, n1, n2):
    monkeypatch.setenv("RQA_BAND_ROWS", str(rows))
    monkeypatch.setenv("RQA_TILE_WARPS", str(warps))
    x = synth.lorenz_x(n1 + 6, 800 + n1, discard=1000)
    y = synth.lorenz_x(n2 + 6, 900 + n2, discard=1000)
    st = _cross_check(x, y, m=4, tau=2, eps=0.6, norm=0, theiler=2)
    assert st["band_rows"] == rows


@pytest.mark.parametrize("w", [0, 5])
def test_cross_bands_constant_and_same_series(monkeypatch, w):
    monkeypatch.setenv("RQA_BAND_ROWS", "64")
    monkeypatch.setenv("RQA_TILE_WARPS", "2")
    _cross_check(np.full(900, 0.3), np.full(1300, 0.3), m=2, tau=1, eps=0.1, norm=1, theiler=w)
    s = synth.ar1(1500, 5, 0.9)
    a = gp.RQA(gpu_settings(3, 1, 0.5, 1, w))
    ma = a.run(s)
    b = gp.RQA(gpu_settings(3, 1, 0.5, 1, w))
    mb = b.run_cross(s, s)
    for u, v in zip(a.histograms(), b.histograms()):
        assert np.array_equal(u, v)
    assert_same_measures(mb, ma)


@pytest.mark.parametrize("rows", [32, 160])
def test_matrix_bands(monkeypatch, rows):
    monkeypatch.setenv("RQA_BAND_ROWS", str(rows))
    rng = np.random.default_rng(rows)
    for R in (np.ones((1300, 1700), np.uint8),
              (rng.random((1700, 1100)) < 0.5).astype(np.uint8),
              ((np.arange(1300)[None, :] - np.arange(900)[:, None]) % 3 == 0).astype(np.uint8)):
        want = oracle.matrix_rqa(R, oracle.Settings(m=1, tau=1, eps=1.0, norm=0, theiler=1))
        r = gp.RQA(gpu_settings(1, 1, 1.0, 0, 1))
        meas = r.run_matrix(R)
        for got, k in zip(r.histograms(), ("hd", "hv", "hw")):
            assert np.array_equal(got, want[k]), k
        assert_same_measures(meas, want["measures"])
        assert r.stats()["band_rows"] == rows


def test_cross_automatic_bands():
    x = synth.ar1(20_000, 71, 0.9)
    y = synth.ar1(15_000, 72, 0.9)
    st = _cross_check(x, y, m=3, tau=1, eps=0.4, norm=1, theiler=0)
    assert st["band_rows"] > 0
