"""Seeded random sweep: RQA, cross recurrence and matrix input on random
sizes, embeddings, norms, radii, Theiler windows, strip widths and row-band
heights, each against the oracle bit for bit.  Sizes stay small enough for
the materialised oracle; the draws cover ragged tails on both axes.  Odd
cases run two columns per lane, even ones four.  RQA_FUZZ_CASES sets the
number of RQA cases (40; half as many cross and matrix cases) for a longer
sweep."""
import os

import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same_measures, gpu_settings

import paper_2402_16853_b300 as gp

pytestmark = pytest.mark.gpu

CASES = int(os.environ.get("RQA_FUZZ_CASES", "40"))


def _series(rng, N):
    kind = int(rng.integers(0, 4))
    seed = int(rng.integers(0, 1 << 30))
    if kind == 0:
        return synth.logistic(N, seed, r=float(rng.uniform(3.6, 4.0)))
    if kind == 1:
        return synth.lorenz_x(N, seed, discard=500)
    if kind == 2:
        return synth.ar1(N, seed, float(rng.uniform(0.3, 0.99)))
    return synth.dyadic(N, seed, levels=int(rng.integers(2, 9)), scale_log2=-2)


def _env(monkeypatch, rng, case):
    monkeypatch.setenv("RQA_TILE_COLS", "2" if case % 2 else "4")
    monkeypatch.setenv("RQA_TILE_WARPS", str(int(rng.integers(1, 9))))
    rows = int(rng.choice([0, 32, 64, 96, 256, 1024]))
    monkeypatch.setenv("RQA_BAND_ROWS", str(rows))


def _settings(rng, kind_std):
    m = int(rng.integers(1, 7))
    tau = int(rng.integers(1, 4))
    norm = int(rng.integers(0, 3))
    eps = float(rng.uniform(0.05, 0.6)) * kind_std * (m ** 0.5 if norm else 1.0)
    w = int(rng.choice([0, 1, 2, 5, 40]))
    mins = [int(x) for x in rng.integers(1, 4, 3)]
    return dict(m=m, tau=tau, eps=eps, norm=norm, theiler=w, l_min=mins[0], v_min=mins[1],
                w_min=mins[2])


def _compare(r, meas, want):
    for got, k in zip(r.histograms(), ("hd", "hv", "hw")):
        assert np.array_equal(got, want[k]), k
    assert_same_measures(meas, want["measures"])


@pytest.mark.parametrize("case", range(CASES))
def test_random_rqa(monkeypatch, case):
    rng = np.random.default_rng(5000 + case)
    _env(monkeypatch, rng, case)
    s = _series(rng, int(rng.integers(20, 2600)))
    kw = _settings(rng, float(np.std(s)) or 1.0)
    if len(s) - (kw["m"] - 1) * kw["tau"] < 1:
        kw.update(m=1, tau=1)
    want = oracle.rqa(s, oracle.Settings(**kw))
    r = gp.RQA(gpu_settings(**kw))
    _compare(r, r.run(s), want)


@pytest.mark.parametrize("case", range(CASES // 2))
def test_random_cross(monkeypatch, case):
    rng = np.random.default_rng(6000 + case)
    _env(monkeypatch, rng, case)
    x = _series(rng, int(rng.integers(20, 2200)))
    y = _series(rng, int(rng.integers(20, 2200)))
    kw = _settings(rng, float(np.std(np.concatenate([x, y]))) or 1.0)
    span = (kw["m"] - 1) * kw["tau"]
    if min(len(x), len(y)) - span < 1:
        kw.update(m=1, tau=1)
    want = oracle.cross_rqa(x, y, oracle.Settings(**kw))
    r = gp.RQA(gpu_settings(**kw))
    _compare(r, r.run_cross(x, y), want)


@pytest.mark.parametrize("case", range(CASES // 2))
def test_random_matrix(monkeypatch, case):
    rng = np.random.default_rng(7000 + case)
    _env(monkeypatch, rng, case)
    rows, cols = (int(v) for v in rng.integers(1, 2100, 2))
    R = (rng.random((rows, cols)) < float(rng.uniform(0.02, 0.98))).astype(np.uint8)
    w = int(rng.choice([0, 1, 3]))
    want = oracle.matrix_rqa(R, oracle.Settings(m=1, tau=1, eps=1.0, norm=0, theiler=w))
    r = gp.RQA(gpu_settings(1, 1, 1.0, 0, w))
    _compare(r, r.run_matrix(R), want)


MID_CASES = int(os.environ.get("RQA_FUZZ_MID_CASES", "4"))


@pytest.mark.parametrize("case", range(MID_CASES))
def test_random_rqa_mid_size(monkeypatch, case):
    """Longer series (5,000-30,000 points) against the streaming oracle:
    many blocks right of the diagonal, long white runs, row bands chosen by
    the library or forced."""
    rng = np.random.default_rng(8000 + case)
    monkeypatch.setenv("RQA_TILE_COLS", "2" if case % 2 else "4")
    monkeypatch.setenv("RQA_TILE_WARPS", str(int(rng.choice([1, 2, 4, 8]))))
    if rng.random() < 0.5:
        monkeypatch.setenv("RQA_BAND_ROWS", str(int(rng.choice([0, 256, 1024, 4096]))))
    s = _series(rng, int(rng.integers(5000, 30000)))
    kw = _settings(rng, float(np.std(s)) or 1.0)
    want = oracle.rqa(s, oracle.Settings(**kw), mode="streaming")
    r = gp.RQA(gpu_settings(**kw))
    _compare(r, r.run(s), want)
