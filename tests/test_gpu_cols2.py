"""GPU parity of the tile kernels with two columns per lane (FP32 distances;
strips half as wide for the same warps), which the autotuner may choose for
a class: histograms and measures bit for bit against the oracle, forced
through RQA_TILE_COLS=2 over every norm, several m and Theiler windows,
every strip width, ragged sizes, row bands, cross recurrence and the batched
path; FP64 runs keep four columns per lane."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import _diff, assert_same_measures, check_parity, gpu_settings, oracle_settings

import paper_2402_16853_b300 as gp

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _two_cols(monkeypatch):
    monkeypatch.delenv("RQA_TILE_WARPS", raising=False)
    monkeypatch.delenv("RQA_BAND_ROWS", raising=False)
    monkeypatch.setenv("RQA_TILE_COLS", "2")


@pytest.mark.parametrize("norm", [0, 1, 2])
@pytest.mark.parametrize("m", [1, 3, 8])
@pytest.mark.parametrize("w", [0, 1, 5])
def test_norms_dims_windows(norm, m, w):
    s = synth.ar1(1300 + 37 * m, 400 + 10 * m + norm + w, 0.9)
    r, st, _ = check_parity(s, m=m, tau=2, eps=0.45 + 0.1 * m, norm=norm, theiler=w)
    assert st["cols_per_lane"] == 2


@pytest.mark.parametrize("warps", [1, 2, 3, 8])
@pytest.mark.parametrize("n", [1, 31, 64, 65, 200, 1025])
def test_widths_and_ragged_sizes(monkeypatch, warps, n):
    monkeypatch.setenv("RQA_TILE_WARPS", str(warps))
    s = synth.logistic(n + 4, 900 + n, r=3.9)
    r, st, _ = check_parity(s, m=3, tau=2, eps=0.1, norm=1, theiler=1)
    assert st["strip_width"] == 64 * warps


@pytest.mark.parametrize("rows", [32, 96, 512])
def test_row_bands(monkeypatch, rows):
    monkeypatch.setenv("RQA_BAND_ROWS", str(rows))
    monkeypatch.setenv("RQA_TILE_WARPS", "2")
    s = synth.lorenz_x(2400, 77, discard=1000)
    r, st, _ = check_parity(s, m=4, tau=2, eps=0.6, norm=0, theiler=2)
    assert st["band_rows"] == rows and st["cols_per_lane"] == 2


def test_automatic_bands_and_dyadic_ties():
    s = synth.ar1(20_000, 78, 0.95)
    r, st, _ = check_parity(s, m=3, tau=1, eps=0.5, norm=1, theiler=1)
    assert st["band_rows"] > 0 and st["cols_per_lane"] == 2
    d = synth.dyadic(3000, 79)
    r, st, _ = check_parity(d, m=2, tau=1, eps=0.5, norm=2, theiler=1)
    assert st["rechecks"] > 0


@pytest.mark.parametrize("n1,n2", [(700, 1300), (1300, 700), (33, 2000)])
def test_cross(n1, n2):
    x = synth.ar1(n1, 80, 0.9)
    y = synth.ar1(n2, 81, 0.9)
    want = oracle.cross_rqa(x, y, oracle_settings(3, 1, 0.5, 1, 2))
    r = gp.RQA(gpu_settings(3, 1, 0.5, 1, 2))
    meas = r.run_cross(x, y)
    hd, hv, hw = r.histograms()
    assert np.array_equal(hd, want["hd"]), _diff("diag", hd, want["hd"])
    assert np.array_equal(hv, want["hv"]), _diff("vert", hv, want["hv"])
    assert np.array_equal(hw, want["hw"]), _diff("white", hw, want["hw"])
    assert_same_measures(meas, want["measures"])
    assert r.stats()["cols_per_lane"] == 2


def test_batch_and_fp64_keeps_four():
    specs = [synth.SeriesSpec("ar1", L, m, 1, norm, 0.3, 0.9)
             for L, m, norm in ((900, 2, 0), (2500, 5, 1), (1700, 8, 2), (700, 3, 1))]
    series, eps = synth.make_series(specs, 82)
    settings = [gp.Settings(m=sp.m, tau=sp.tau, eps=e, norm=sp.norm, theiler=1)
                for sp, e in zip(specs, eps)]
    b = gp.Batch()
    res, st, rc = b.run(settings, series)
    assert rc == 0
    for q, (stg, s) in enumerate(zip(settings, series)):
        want = oracle.rqa(s, oracle_settings(stg.m, stg.tau, stg.eps, stg.norm, 1))
        assert np.array_equal(b.histogram(q, 0), want["hd"]), q
        assert np.array_equal(b.histogram(q, 1), want["hv"]), q
        assert np.array_equal(b.histogram(q, 2), want["hw"]), q
        assert_same_measures(res[q], want["measures"])
    s = synth.ar1(1500, 83, 0.9)
    r, st64, _ = check_parity(s, m=3, tau=1, eps=0.5, norm=1, theiler=1, precision=gp.PREC_FP64)
    assert st64["cols_per_lane"] == 4
