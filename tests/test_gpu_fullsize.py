"""Full-size checks in the launch configuration bench.py times.

* Lorenz-x, N = 100,000 (n = 99,988, max norm, w = 5): all histograms and
  measures bit-exact against the streaming FP64 oracle.
* AR(1), N = 1,048,576 (n = 1,048,574, L2, w = 1): the oracle's complete
  result, computed once on 16 host cores by tests/golden/make_ar1_n1m_oracle.py
  and stored as SHA-256 digests of the three histograms plus the measures,
  must match bit for bit; besides, properties that hold at any size and
  sampled decisions:
  - the diagonal scan and the column / row scans see the same recurrence
    points (sum l P_D(l) == sum l P_V(l)), and white lines cover the rest of
    the n^2 cells;
  - the FP32 + FP64-recheck path and the FP64-everywhere path give identical
    histograms;
  - 200,000 decisions R_ij, drawn uniformly, near the line of identity and
    near the radius, equal the oracle's FP64 decisions one by one.
* The largest series the library accepts, n = 2^22: the same properties and
  sampled decisions; one vector more is refused with RQA_ETOOBIG.
* The paper's timing series (Sect. 8.2, sin over 1,000,001 points, m = 2,
  tau = 2, eps = 1, no Theiler window): the oracle's complete result, stored
  by tests/golden/make_sine_paper_oracle.py as SHA-256 digests plus the
  measures, must match bit for bit; the line of identity is one line of
  length n, and the diagonal histogram is otherwise even (both triangles).
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same_measures

import paper_2402_16853_b300 as gp

pytestmark = pytest.mark.gpu


def test_lorenz_n100k_bit_exact():
    s, p = synth.workload("lorenz_n100k")
    want = oracle.rqa(s, oracle.Settings(**p), mode="streaming")
    r = gp.RQA(gp.Settings(**p))
    meas = r.run(s)
    hd, hv, hw = r.histograms()
    assert np.array_equal(hd, want["hd"])
    assert np.array_equal(hv, want["hv"])
    assert np.array_equal(hw, want["hw"])
    assert_same_measures(meas, want["measures"])


@pytest.fixture(scope="module")
def ar1_full():
    s, p = synth.workload("ar1_n1m")
    r = gp.RQA(gp.Settings(**p))
    meas = r.run(s)
    return s, p, r, meas, r.histograms(), r.stats()


GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ar1_n1m_oracle.json")


def test_ar1_n1m_equals_full_oracle(ar1_full):
    s, p, r, meas, (hd, hv, hw), st = ar1_full
    gold = json.load(open(GOLDEN))
    assert gold["n_vec"] == st["n_vec"] and gold["params"] == p
    for name, h in (("hd", hd), ("hv", hv), ("hw", hw)):
        g = gold[name]
        assert int(h.sum()) == g["sum"], name
        assert {str(l): int(h[l]) for l in range(1, 65) if h[l]} == g["head"], name
        assert hashlib.sha256(np.ascontiguousarray(h, dtype="<u8").tobytes()).hexdigest() \
            == g["sha256"], name
    assert meas["recurrence_points"] == gold["rp"]
    assert_same_measures(meas, gold["measures"])


def test_ar1_n1m_invariants(ar1_full):
    s, p, r, meas, (hd, hv, hw), st = ar1_full
    n = len(s) - (p["m"] - 1) * p["tau"]
    L = np.arange(n + 1, dtype=np.uint64)
    rp_d = int((L * hd).sum())
    rp_v = int((L * hv).sum())
    assert rp_d == rp_v == meas["recurrence_points"]
    assert int((L * hw).sum()) == n * n - rp_v
    assert hd[0] == hv[0] == hw[0] == 0
    assert int(hd.sum()) % 2 == 0           # w = 1: every line has a mirror image
    assert st["exact"] == 1 and st["rechecks"] > 0


def test_ar1_n1m_fp64_path_identical(ar1_full):
    s, p, r, meas, (hd, hv, hw), st = ar1_full
    r64 = gp.RQA(gp.Settings(**p, precision=gp.PREC_FP64))
    m64 = r64.run(s)
    h64 = r64.histograms()
    assert np.array_equal(h64[0], hd) and np.array_equal(h64[1], hv)
    assert np.array_equal(h64[2], hw)
    assert_same_measures(m64, meas)


def test_ar1_n1m_sampled_decisions(ar1_full):
    s, p, r, meas, hists, st = ar1_full
    n = len(s) - (p["m"] - 1) * p["tau"]
    rng = np.random.default_rng(99)
    i = rng.integers(0, n, 100_000)
    j = rng.integers(0, n, 100_000)
    k = rng.integers(0, 40, 50_000)            # near the line of identity
    i2 = rng.integers(0, n - 40, 50_000)
    i = np.concatenate([i, i2])
    j = np.concatenate([j, i2 + k])
    # pairs close to the radius: search a random pool for the smallest |d - eps|
    pi = rng.integers(0, n, 2_000_000)
    pj = rng.integers(0, n, 2_000_000)
    x = np.stack([s[pi + q * p["tau"]] - s[pj + q * p["tau"]] for q in range(p["m"])])
    d = np.sqrt((x * x).sum(axis=0))
    near = np.argsort(np.abs(d - p["eps"]))[:50_000]
    i = np.concatenate([i, pi[near]])
    j = np.concatenate([j, pj[near]])
    got = r.sample(i, j)
    st_o = oracle.Settings(**p)
    want = np.array([oracle.distance(s, a, b, p["m"], p["tau"], p["norm"]) <= p["eps"]
                     and abs(a - b) >= p["theiler"] for a, b in zip(i, j)], dtype=np.uint8)
    assert np.array_equal(got, want)
    del st_o


SINE_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sine_paper_oracle.json")


def test_paper_sine_series():
    """The paper's runtime workload (Sect. 8.2) against the FP64 oracle's
    complete result (tests/golden/make_sine_paper_oracle.py): all three
    histograms bit for bit (SHA-256), every measure, and the w = 0 facts."""
    s, p = synth.workload("sine_paper")
    r = gp.RQA(gp.Settings(**p))
    meas = r.run(s)
    hd, hv, hw = r.histograms()
    n = len(s) - 2
    assert meas["n_vec"] == n == 999_999
    gold = json.load(open(SINE_GOLDEN))
    assert gold["params"] == p and gold["n_vec"] == n
    for name, h in (("hd", hd), ("hv", hv), ("hw", hw)):
        g = gold[name]
        assert int(h.sum()) == g["sum"], name
        assert {str(l): int(h[l]) for l in range(1, 65) if h[l]} == g["head"], name
        assert hashlib.sha256(np.ascontiguousarray(h, dtype="<u8").tobytes()).hexdigest() \
            == g["sha256"], name
    assert meas["recurrence_points"] == gold["rp"]
    assert_same_measures(meas, gold["measures"])
    assert hd[n] == 1 and meas["l_max"] == n      # the line of identity (Table 3 reading)
    off = hd.copy()
    off[n] -= 1
    assert np.all(off % 2 == 0)                   # the two triangles mirror each other


def _large_series_checks(n_vec, seed, expect_groups):
    """A series of n_vec AR(1) vectors: it runs in strip groups (its
    boundary descriptors would exceed the budget), holds at most the budget
    at once, and the size-independent properties hold; sampled decisions
    (uniform, near the line of identity, near the radius) equal the
    oracle's."""
    m, tau = 3, 1
    s = synth.ar1(n_vec + (m - 1) * tau, seed, 0.95)
    p = dict(m=m, tau=tau, eps=0.5, norm=1, theiler=1)
    r = gp.RQA(gp.Settings(**p))
    meas = r.run(s)
    hd, hv, hw = r.histograms()
    st = r.stats()
    n = n_vec
    assert st["strip_groups"] >= expect_groups
    assert st["desc_bytes"] < st["desc_bytes_all_strips"]
    assert st["strip_groups"] * st["strips_per_group"] * st["strip_width"] >= n - 1
    assert st["n_vec"] == n and meas["n_vec"] == n
    L = np.arange(n + 1, dtype=np.uint64)
    rp = int((L * hv).sum())
    assert int((L * hd).sum()) == rp == meas["recurrence_points"] > 0
    assert int((L * hw).sum()) == n * n - rp
    assert hd[0] == hv[0] == hw[0] == 0 and int(hd.sum()) % 2 == 0
    assert st["exact"] == 1
    rng = np.random.default_rng(7)
    i = rng.integers(0, n, 6_000)
    j = rng.integers(0, n, 6_000)
    k = rng.integers(0, 40, 3_000)
    i2 = rng.integers(0, n - 40, 3_000)
    pi = rng.integers(0, n, 400_000)
    pj = rng.integers(0, n, 400_000)
    x = np.stack([s[pi + q * tau] - s[pj + q * tau] for q in range(m)])
    near = np.argsort(np.abs(np.sqrt((x * x).sum(axis=0)) - p["eps"]))[:3_000]
    i = np.concatenate([i, i2, pi[near]])
    j = np.concatenate([j, i2 + k, pj[near]])
    got = r.sample(i, j)
    want = np.array([oracle.distance(s, a, b, m, tau, p["norm"]) <= p["eps"]
                     and abs(a - b) >= p["theiler"] for a, b in zip(i, j)], dtype=np.uint8)
    assert np.array_equal(got, want)
    r.close()


def test_series_of_2_22_vectors():
    """n = 2^22 vectors: about 8.8e12 pairs; all its strips' boundary
    descriptors would take 69 GB, so it runs in strip groups under the
    default budget (a fifth of the device's memory)."""
    _large_series_checks(1 << 22, 1009, 2)


def test_series_of_2_23_vectors():
    """n = 2^23 vectors (3.5e13 pairs, 275 GB of descriptors for all
    strips at once, above the device's memory): strip groups bound it."""
    _large_series_checks(1 << 23, 1015, 5)


def test_largest_accepted_size():
    """RQA_MAX_N = 2^24 vectors is the largest series accepted; one vector
    more is refused before anything runs."""
    p = dict(m=3, tau=1, eps=0.5, norm=1, theiler=1)
    s = np.zeros((1 << 24) + 3)
    with pytest.raises(gp.RQAError) as e:
        gp.RQA(gp.Settings(**p)).run(s)
    assert e.value.status == 9  # RQA_ETOOBIG


def test_ar1_n1m_in_strip_groups_equals_full_oracle(monkeypatch):
    """The 1,048,576-point workload with the descriptor budget forced down to
    1.1 GB: its 1,024 strips run in groups, rows and diagonals carried from
    group to group, and the histograms still equal the oracle's complete
    result bit for bit."""
    monkeypatch.setenv("RQA_DESC_BUDGET", str(1_100_000_000))
    s, p = synth.workload("ar1_n1m")
    r = gp.RQA(gp.Settings(**p))
    meas = r.run(s)
    st = r.stats()
    assert st["strip_groups"] >= 4 and st["desc_bytes"] <= 1_100_000_000 + 2 * 4 * st["n_vec"] + 4096
    gold = json.load(open(GOLDEN))
    for name, h in zip(("hd", "hv", "hw"), r.histograms()):
        assert hashlib.sha256(np.ascontiguousarray(h, dtype="<u8").tobytes()).hexdigest() \
            == gold[name]["sha256"], name
    assert_same_measures(meas, gold["measures"])
