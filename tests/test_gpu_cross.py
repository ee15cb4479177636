"""GPU parity for cross recurrence (Sect. 3.3; Sect. 4.2's non-symmetric
matrix): rqa_run_cross against the oracle's cross_rqa, histograms and
measures bit for bit.

Shapes span several 32-row blocks, several warps of a CTA strip, several
strips and ragged tails on both axes, tall and wide rectangles; the edge
cases are a single row or column, Theiler windows of 0, 1, many and beyond
the matrix, exact ties, every norm, m = 1..10, the FP64 path, device
series, the same series twice (which must give RQA) and bad input.
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


def check_cross(x, y, **kw):
    okw = {k: v for k, v in kw.items() if k not in ("precision", "band_override")}
    want = oracle.cross_rqa(x, y, oracle_settings(**okw))
    r = gp.RQA(gpu_settings(**kw))
    meas = r.run_cross(x, y)
    hd, hv, hw = r.histograms()
    assert np.array_equal(hd, want["hd"]), _diff("diag", hd, want["hd"])
    assert np.array_equal(hv, want["hv"]), _diff("vert", hv, want["hv"])
    assert np.array_equal(hw, want["hw"]), _diff("white", hw, want["hw"])
    assert_same_measures(meas, want["measures"])
    st = r.stats()
    assert st["mode"] == 1 and st["n_vec"] == want["n"] and st["n_cols"] == want["cols"]
    return r, st, want


@pytest.mark.parametrize("norm", [0, 1, 2])
@pytest.mark.parametrize("w", [0, 1, 4])
def test_ar1_pair(norm, w):
    x = synth.ar1(700, 11 + norm, 0.9)
    y = synth.ar1(900, 21 + w, 0.8)
    check_cross(x, y, m=3, tau=2, eps=0.5, norm=norm, theiler=w)


@pytest.mark.parametrize("n1,n2", [(1, 1), (1, 300), (300, 1), (31, 33), (32, 32), (33, 31),
                                   (127, 129), (129, 127), (700, 64), (64, 700), (1025, 1023),
                                   (2000, 130), (130, 2000)])
def test_shapes(n1, n2):
    x = synth.logistic(n1 + 1, 300 + n1)
    y = synth.logistic(n2 + 1, 400 + n2, r=3.95)
    check_cross(x, y, m=2, tau=1, eps=0.08, norm=1, theiler=1)


@pytest.mark.parametrize("warps", [1, 2, 3, 4, 5, 8])
@pytest.mark.parametrize("n1,n2", [(900, 2400), (2400, 900)])
def test_warps_per_strip(monkeypatch, warps, n1, n2):
    """Every CTA-strip width: diagonal carries between the warps of a strip
    and boundary descriptors between strips, with a ragged last strip."""
    monkeypatch.setenv("RQA_TILE_WARPS", str(warps))
    x = synth.lorenz_x(n1 + 6, 500 + n1, discard=1000)
    y = synth.lorenz_x(n2 + 6, 600 + n2, discard=1000)
    check_cross(x, y, m=4, tau=2, eps=0.6, norm=0, theiler=2)


@pytest.mark.parametrize("m", range(1, 11))
def test_every_m(m):
    x = synth.ar1(600 + m, 40 + m, 0.95)
    y = synth.ar1(450 + 3 * m, 50 + m, 0.95)
    check_cross(x, y, m=m, tau=1, eps=0.3 * m, norm=m % 3, theiler=1)


@pytest.mark.parametrize("w", [0, 1, 2, 31, 32, 33, 500, 1999, 2000, 10**6])
def test_theiler_windows(w):
    x = synth.logistic(1500, 7)
    y = synth.logistic(2000, 8)
    check_cross(x, y, m=2, tau=1, eps=0.1, norm=2, theiler=w)


@pytest.mark.parametrize("norm", [0, 1, 2])
def test_exact_ties(norm):
    """Dyadic values: many cross pairs at d == eps, re-decided in FP64."""
    x = synth.dyadic(1300, 1, levels=4, scale_log2=-1)
    y = synth.dyadic(1100, 2, levels=4, scale_log2=-1)
    r, st, _ = check_cross(x, y, m=2, tau=1, eps=0.5, norm=norm, theiler=0)
    assert st["rechecks"] > 0


@pytest.mark.parametrize("norm", [0, 1, 2])
def test_long_lines_end_together(norm):
    """Constant series with one outlier each: the white row and column end
    thousands of runs longer than the shared bins in the same sub-blocks."""
    x = synth.constant(4100, 0.3)
    y = synth.constant(3900, 0.3)
    x[1500] = 100.0
    y[2600] = -100.0
    _, _, want = check_cross(x, y, m=2, tau=1, eps=0.01, norm=norm, theiler=0)
    assert want["hd"][1024:].sum() > 1000 and want["hv"][1024:].sum() > 1000


@pytest.mark.parametrize("p,off", [(3, 0), (5, 2)])
def test_periodic(p, off):
    x = synth.periodic(1200, p)
    y = synth.periodic(1700, p, offset=off)
    check_cross(x, y, m=3, tau=2, eps=0.5, norm=1, theiler=0)


@pytest.mark.parametrize("norm", [0, 1, 2])
def test_fp64_path(norm):
    x = synth.lorenz_x(1300, 3)
    y = synth.lorenz_x(1000, 4)
    check_cross(x, y, m=3, tau=3, eps=0.7, norm=norm, theiler=1, precision=gp.PREC_FP64)


def test_scale_offset_between_series():
    """The two series share one FP32 centring: one sits far from zero."""
    x = synth.ar1(1400, 5, 0.9) * 3.0 + 1000.0
    y = synth.ar1(1100, 6, 0.9) * 3.0 + 1001.0
    check_cross(x, y, m=3, tau=1, eps=1.2, norm=1, theiler=0)


@pytest.mark.parametrize("norm", [0, 1, 2])
@pytest.mark.parametrize("w", [0, 1, 3])
def test_same_series_is_rqa(norm, w):
    """Sect. 3.3: the same series on both axes is ordinary RQA."""
    s = synth.ar1(2500, 77, 0.9)
    st = gpu_settings(m=3, tau=2, eps=0.5, norm=norm, theiler=w)
    a = gp.RQA(st)
    ma = a.run(s)
    ha = a.histograms()
    b = gp.RQA(st)
    mb = b.run_cross(s, s)
    hb = b.histograms()
    for u, v in zip(ha, hb):
        assert np.array_equal(u, v)
    assert_same_measures(mb, ma)


def test_device_series_torch():
    torch = pytest.importorskip("torch")
    x = synth.ar1(1800, 8, 0.9)
    y = synth.ar1(1300, 9, 0.9)
    want = oracle.cross_rqa(x, y, oracle_settings(3, 1, 0.4, 1, 1))
    r = gp.RQA(gpu_settings(3, 1, 0.4, 1, 1))
    meas = r.run_cross(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    assert np.array_equal(r.histogram(0), want["hd"])
    assert_same_measures(meas, want["measures"])


def test_sampled_decisions_match_oracle():
    x = synth.lorenz_x(3000, 12)
    y = synth.lorenz_x(2200, 13)
    m, tau, eps, norm, w = 3, 2, 0.5, 1, 2
    r = gp.RQA(gpu_settings(m, tau, eps, norm, w))
    r.run_cross(x, y)
    n1, n2 = len(x) - (m - 1) * tau, len(y) - (m - 1) * tau
    rng = np.random.default_rng(5)
    i = rng.integers(0, n1, 20000)
    j = rng.integers(0, n2, 20000)
    got = r.sample(i, j)
    want = np.array([abs(a - b) >= w and oracle.cross_distance(x, y, a, b, m, tau, norm) <= eps
                     for a, b in zip(i, j)], dtype=np.uint8)
    assert np.array_equal(got, want)


def test_cross_plot_window():
    x = synth.logistic(300, 31)
    y = synth.logistic(250, 32)
    m, tau, eps, norm, w = 2, 3, 0.1, 0, 1
    st = gpu_settings(m, tau, eps, norm, w)
    n1, n2 = len(x) - (m - 1) * tau, len(y) - (m - 1) * tau
    plot = gp.cross_recurrence_plot(st, x, y, i0=5, j0=17, rows=n1 - 5 + 3, cols=n2 - 17 + 40)
    want = np.zeros_like(plot)
    for r in range(n1 - 5):
        for c in range(n2 - 17):
            a, b = 5 + r, 17 + c
            want[r, c] = abs(a - b) >= w and oracle.cross_distance(x, y, a, b, m, tau, norm) <= eps
    assert np.array_equal(plot, want)


def test_bad_inputs_reported():
    r = gp.RQA(gpu_settings(3, 2, 0.5, 1, 1))
    y = synth.ar1(500, 1, 0.9)
    bad = y.copy()
    bad[100] = np.nan
    with pytest.raises(gp.RQAError) as ei:
        r.run_cross(synth.ar1(400, 2, 0.9), bad)
    assert ei.value.status == 3                   # RQA_ENAN
    with pytest.raises(gp.RQAError) as ei:
        r.run_cross(synth.ar1(400, 2, 0.9), np.zeros(4))
    assert ei.value.status == 2                   # RQA_ESHORT: no vector in the second series
    meas = r.run_cross(synth.ar1(400, 2, 0.9), y)  # the handle still works
    assert meas["n_vec"] == 396


def test_medium_lorenz_streaming_oracle():
    """n1 = 19,988 rows by n2 = 14,988 columns: 59 two-warp strips, bit-exact."""
    x = synth.lorenz_x(20_000, 1)
    y = synth.lorenz_x(15_000, 2)
    check_cross(x, y, m=5, tau=3, eps=0.3, norm=0, theiler=5)


def test_max_rows_rectangle():
    """n1 = RQA_MAX_N_RECT = 2^22 row vectors against n2 = 2^20 column vectors
    (4.4e12 cells): every cell lies in exactly one vertical black or white
    run of its column, the diagonal and vertical scans see the same
    recurrence points, and sampled decisions (uniform and near the radius)
    equal the oracle's."""
    m, tau, eps, norm, w = 3, 1, 0.5, 1, 1
    x = synth.ar1((1 << 22) + (m - 1) * tau, 1011, 0.95)
    y = synth.ar1((1 << 20) + (m - 1) * tau, 1013, 0.95)
    r = gp.RQA(gpu_settings(m, tau, eps, norm, w))
    meas = r.run_cross(x, y)
    hd, hv, hw = r.histograms()
    st = r.stats()
    n1, n2 = 1 << 22, 1 << 20
    assert st["mode"] == 1 and st["n_vec"] == n1 and st["n_cols"] == n2
    L = np.arange(len(hd), dtype=np.uint64)
    rp = int((L * hv).sum())
    assert int((L * hd).sum()) == rp == meas["recurrence_points"] > 0
    assert int((L * hw).sum()) == n1 * n2 - rp
    assert st["exact"] == 1
    rng = np.random.default_rng(11)
    i = rng.integers(0, n1, 6000)
    j = rng.integers(0, n2, 6000)
    pi = rng.integers(0, n1, 400_000)
    pj = rng.integers(0, n2, 400_000)
    d = np.sqrt(sum((x[pi + q * tau] - y[pj + q * tau]) ** 2 for q in range(m)))
    near = np.argsort(np.abs(d - eps))[:3000]
    i = np.concatenate([i, pi[near]])
    j = np.concatenate([j, pj[near]])
    got = r.sample(i, j)
    want = np.array([abs(a - b) >= w and oracle.cross_distance(x, y, a, b, m, tau, norm) <= eps
                     for a, b in zip(i, j)], dtype=np.uint8)
    assert np.array_equal(got, want)
