"""The autotuner (Sect. 9 plans picking the best-performing implementation
at runtime): it times every CTA-strip width on a series, records the
fastest for the series' class, later runs of the class use it, and the
results stay identical to the oracle whatever width runs."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same_measures, check_parity, gpu_settings, oracle_settings

import paper_2402_16853_b300 as gp

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _clean_table(monkeypatch):
    monkeypatch.delenv("RQA_TILE_WARPS", raising=False)
    monkeypatch.delenv("RQA_TILE_COLS", raising=False)
    gp.autotune_clear()
    yield
    gp.autotune_clear()


def test_tuned_width_is_used_and_exact():
    st = gpu_settings(3, 2, 0.4, 1, 1)
    t = gp.autotune(st, n_points=9000)
    assert t["warps"] in (1, 2, 4, 8)
    assert all(np.isfinite(v) and v > 0 for v in t["ms"].values())
    s = synth.ar1(9100, 3, 0.9)        # the same class: L2, m = 3, ceil(log2 n) = 14
    r, stt, _ = check_parity(s, m=3, tau=2, eps=0.4, norm=1, theiler=1)
    assert stt["warps_per_cta"] == t["warps"]
    gp.autotune_clear()
    r2 = gp.RQA(st)
    r2.run(s)
    assert r2.stats()["warps_per_cta"] == 2          # the size rule again (4096 <= n < 16384)
    assert r2.stats()["cols_per_lane"] == 4


def test_shape_search_and_table_round_trip(tmp_path):
    """The full search (width, columns per lane, band height) on a series
    that runs in row bands; its winner is used by later runs of the class,
    survives a save / clear / load round trip, and the results stay exact."""
    st = gpu_settings(4, 1, 0.5, 0, 1)
    t = gp.autotune_shape(st, n_points=30_000)
    assert t["warps"] in (1, 2, 4, 8) and t["cols"] in (2, 4) and t["band_scale"] in (-1, 0, 1)
    assert np.isfinite(t["ms"]) and t["ms"] > 0
    path = str(tmp_path / "table.txt")
    gp.save_tuning_table(path)
    gp.autotune_clear()
    assert gp.load_tuning_table(path) == 1
    s = synth.lorenz_x(29_000, 8, discard=2000)   # same class: ceil(log2 n) = 15
    r, stt, _ = check_parity(s, m=4, tau=1, eps=0.5, norm=0, theiler=1)
    assert (stt["warps_per_cta"], stt["cols_per_lane"]) == (t["warps"], t["cols"])


def test_tune_on_callers_series_and_cross():
    x = synth.lorenz_x(3000, 5)
    st = gpu_settings(4, 1, 0.5, 0, 2)
    t = gp.autotune(st, series=x, cross=True)
    y = synth.lorenz_x(2900, 6)
    want = oracle.cross_rqa(x, y, oracle_settings(4, 1, 0.5, 0, 2))
    r = gp.RQA(st)
    meas = r.run_cross(x, y)
    assert r.stats()["warps_per_cta"] == t["warps"]
    assert np.array_equal(r.histogram(0), want["hd"])
    assert_same_measures(meas, want["measures"])
    r.run(x)                                         # an RQA run is another class
    assert r.stats()["warps_per_cta"] == 1


def test_other_classes_untouched():
    gp.autotune(gpu_settings(2, 1, 0.3, 2, 1), n_points=5000)
    r = gp.RQA(gpu_settings(2, 1, 0.3, 0, 1))        # another norm
    r.run(synth.ar1(5000, 1, 0.9))
    assert r.stats()["warps_per_cta"] == 2


def test_errors():
    with pytest.raises(gp.RQAError) as ei:
        gp.autotune(gpu_settings(3, 4, 0.4, 1, 1), n_points=5)
    assert ei.value.status == 2
    with pytest.raises(gp.RQAError) as ei:
        gp.autotune(gpu_settings(0, 1, 0.4, 1, 1), n_points=500)
    assert ei.value.status == 1
