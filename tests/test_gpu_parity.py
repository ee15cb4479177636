"""GPU parity: the CUDA path through the C ABI against the FP64 oracle,
histograms and measures compared bit for bit.

Sizes are ones the oracle finishes in seconds but that still span several
32 x 32 sub-blocks, several warps of a CTA strip, several CTA strips and a
ragged tail; the edge cases cover n = 1, 2, tile +- 1, Theiler windows of 0,
1, many and >= n, constant and periodic series, exact ties, every norm and
m = 1..10.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same_measures, check_parity, gpu_settings, run_gpu

import paper_2402_16853_b300 as gp

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _default_tiles(monkeypatch):
    monkeypatch.delenv("RQA_TILE_WARPS", raising=False)


def test_logistic_n2000():
    """Logistic map, N = 2,000, m = 3, tau = 2, L2, eps = 0.1, w = 1."""
    s, p = synth.workload("logistic_n2000")
    r, st, want = check_parity(s, **p)
    assert st["n_vec"] == 1996 and st["exact"] == 1


@pytest.mark.parametrize("norm", [0, 1, 2])
@pytest.mark.parametrize("w", [0, 1, 3])
def test_small_random(norm, w):
    s = synth.ar1(700, 100 + norm * 7 + w, 0.9)
    check_parity(s, m=3, tau=2, eps=0.4, norm=norm, theiler=w)


@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 63, 64, 65, 127, 128, 129, 130, 255, 256,
                               257, 1023, 1024, 1025, 1500])
def test_ragged_sizes(n):
    m, tau = 2, 1
    s = synth.logistic(n + (m - 1) * tau, 200 + n)
    check_parity(s, m=m, tau=tau, eps=0.08, norm=1, theiler=1)


@pytest.mark.parametrize("warps", [1, 2, 3, 4, 5, 8])
@pytest.mark.parametrize("n", [900, 2400])
def test_warps_per_strip(monkeypatch, warps, n):
    """Every CTA-strip width: carries between warps of a strip and boundary
    descriptors between strips."""
    monkeypatch.setenv("RQA_TILE_WARPS", str(warps))
    s = synth.lorenz_x(n + 6, 300 + n, discard=1000)
    check_parity(s, m=4, tau=2, eps=0.6, norm=0, theiler=2, l_min=2, v_min=2, w_min=2)


@pytest.mark.parametrize("m", list(range(1, 11)))
def test_every_m(m):
    tau = 1 + (m % 3)
    s = synth.ar1(600 + (m - 1) * tau, 400 + m, 0.95)
    check_parity(s, m=m, tau=tau, eps=0.3 * np.sqrt(m), norm=m % 3, theiler=1)


@pytest.mark.parametrize("w", [0, 1, 5, 200, 599, 600, 601, 5000])
def test_theiler_windows(w):
    s = synth.logistic(603, 500 + w)
    check_parity(s, m=2, tau=3, eps=0.1, norm=1, theiler=w)


@pytest.mark.parametrize("norm", [0, 1, 2])
@pytest.mark.parametrize("w", [0, 1, 7])
def test_constant_series(norm, w):
    """Every pair recurs: lines span every tile and strip."""
    n = 1100
    s = synth.constant(n + 2, 0.3)
    check_parity(s, m=2, tau=2, eps=0.01, norm=norm, theiler=w)


@pytest.mark.parametrize("norm", [0, 1, 2])
@pytest.mark.parametrize("w", [0, 1])
def test_long_lines_end_together(norm, w):
    """A constant series with one outlier: the outlier's white row and column
    end thousands of long column, row and diagonal runs in the same
    sub-blocks, every lane of a warp at once, so lengths beyond the shared
    bins pile up between two drains of the per-warp queue."""
    s = synth.constant(4100, 0.3)
    s[1500] = 100.0
    _, _, want = check_parity(s, m=2, tau=1, eps=0.01, norm=norm, theiler=w)
    assert want["hd"][1024:].sum() > 1000 and want["hv"][1024:].sum() > 1000


@pytest.mark.parametrize("p", [2, 3, 37])
def test_periodic(p):
    s = synth.periodic(1300, p, offset=2)
    check_parity(s, m=3, tau=1, eps=0.5, norm=1, theiler=1)


@pytest.mark.parametrize("norm", [0, 1, 2])
def test_exact_ties(norm):
    """Dyadic values: many pairs sit exactly at d == eps, decided by the
    FP64 recheck."""
    s = synth.dyadic(900, 9, levels=4, scale_log2=-1)
    r, st, _ = check_parity(s, m=2, tau=1, eps=0.5 if norm else 0.5, norm=norm, theiler=1)
    assert st["rechecks"] > 0


@pytest.mark.parametrize("norm", [0, 1, 2])
def test_fp64_path(norm):
    s = synth.ar1(1200, 600 + norm, 0.9)
    r, st, _ = check_parity(s, m=3, tau=1, eps=0.5, norm=norm, theiler=1, precision=2)
    assert st["precision_used"] == 2 and st["rechecks"] == 0


def test_band_everything_rechecked():
    s = synth.ar1(800, 700, 0.9)
    r, st, _ = check_parity(s, m=3, tau=1, eps=0.5, norm=1, theiler=1,
                            band_override=float("inf"))
    assert st["rechecks"] == st["pairs"]
    r2, st2, _ = check_parity(s, m=3, tau=1, eps=0.5, norm=1, theiler=1)
    assert st2["rechecks"] < st["rechecks"]


def test_band_zero_reported_inexact():
    s = synth.ar1(800, 701, 0.9)
    r, meas, hd, hv, hw, st = run_gpu(s, m=3, tau=1, eps=0.5, norm=1, theiler=1,
                                      band_override=0.0)
    assert st["exact"] == 0


def test_large_scale_offset_data():
    """Values far from zero with a small radius: the FP32 copy is centred
    and scaled, the band covers the rest."""
    s = 1e6 + synth.ar1(900, 702, 0.9) * 1e-3
    check_parity(s, m=3, tau=1, eps=4e-4, norm=1, theiler=1)


def test_device_series_torch():
    import torch
    s, p = synth.workload("logistic_n2000")
    want = oracle.rqa(s, oracle.Settings(**p))
    t = torch.tensor(s, dtype=torch.float64, device="cuda")
    r = gp.RQA(gpu_settings(**p))
    meas = r.run(t)
    assert_same_measures(meas, want["measures"])
    assert np.array_equal(r.histogram(0), want["hd"])


def test_nan_input_reported():
    s = synth.ar1(500, 703, 0.9)
    s[123] = np.nan
    r = gp.RQA(gpu_settings(m=2, tau=1, eps=0.3, norm=1, theiler=1))
    with pytest.raises(gp.RQAError) as ei:
        r.run(s)
    assert ei.value.status == 3
    # the handle stays usable
    s[123] = 0.0
    r.run(s)


def test_short_series_rejected():
    r = gp.RQA(gpu_settings(m=3, tau=5, eps=0.3, norm=1, theiler=1))
    with pytest.raises(gp.RQAError) as ei:
        r.run(np.zeros(10))
    assert ei.value.status == 2


def test_sampled_decisions_match_oracle():
    s, p = synth.workload("logistic_n2000")
    r = gp.RQA(gpu_settings(**p))
    r.run(s)
    rng = np.random.default_rng(5)
    n = 1996
    i = rng.integers(0, n, 5000)
    j = rng.integers(0, n, 5000)
    got = r.sample(i, j)
    R, _ = oracle.matrix(s, oracle.Settings(**p))
    assert np.array_equal(got, R[i, j])


@pytest.mark.parametrize("norm", [0, 1, 2])
@pytest.mark.parametrize("scale", [1e200, 1e-200, 1e-305, 1e305])
def test_extreme_magnitudes(norm, scale):
    """Values whose FP64 squares or sums overflow or underflow: the library
    re-decides every pair in FP64 so the decisions stay the definition's."""
    s = synth.ar1(500, 31, 0.9) * scale
    eps = 0.5 * scale
    r, st, want = check_parity(s, m=3, tau=1, eps=eps, norm=norm, theiler=1)
    assert st["exact"] == 1


@pytest.mark.parametrize("w", [0, 1])
def test_all_white_tiny_radius(w):
    """A radius below every distance: only the line of identity (w = 0) can
    recur; every column is white otherwise."""
    s = synth.ar1(1500, 17, 0.9)
    r, st, want = check_parity(s, m=2, tau=1, eps=1e-12, norm=1, theiler=w)
    n = len(s) - 1
    assert want["rp"] == (n if w == 0 else 0)


@pytest.mark.parametrize("norm", [0, 1, 2])
@pytest.mark.parametrize("m", [1, 2])
def test_pairs_within_ulps_of_radius(norm, m):
    """Neighbouring values spaced eps plus a few units in the last place, so
    that many pairs sit within a handful of ulps of the radius on both
    sides; the FP32 test must hand all of them to the FP64 recheck."""
    rng = np.random.default_rng(m * 3 + norm)
    eps = 0.3125
    ulp = np.spacing(eps)
    steps = eps + ulp * rng.integers(-3, 4, 3000)
    s = np.cumsum(steps) * rng.choice([1.0, -1.0], 3000).cumprod()  # zig-zag walk
    s = np.concatenate([[0.0], s])
    e = eps * (m if norm == 2 else (m ** 0.5 if norm == 1 else 1.0))
    r, st, want = check_parity(s, m=m, tau=1, eps=e, norm=norm, theiler=1)
    assert st["rechecks"] > 0
