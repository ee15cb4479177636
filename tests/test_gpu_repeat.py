"""Repeated single-series calls: from the second consecutive call with an
unchanged plan a handle issues its launches through a cached CUDA graph.
Every repetition must still equal the oracle, also when the settings'
values (radius, Theiler window, minimum lengths) or the series' values
change between calls of the same shapes, and when the plan changes."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import assert_same_measures, gpu_settings, oracle_settings

import paper_2402_16853_b300 as gp

pytestmark = pytest.mark.gpu


def _check(r, meas, series, **kw):
    want = oracle.rqa(series, oracle_settings(**kw))
    hd, hv, hw = r.histograms()
    assert np.array_equal(hd, want["hd"])
    assert np.array_equal(hv, want["hv"])
    assert np.array_equal(hw, want["hw"])
    assert_same_measures(meas, want["measures"])


def test_host_series_repeated_with_changing_values():
    a = synth.ar1(2600, 21, 0.9)
    b = synth.zscore(synth.logistic(2600, 22))
    steps = [(a, 0.4, 1, 2), (a, 0.4, 1, 2), (a, 0.4, 1, 2),   # capture, replay
             (a, 0.3, 1, 2),                                   # another radius, same plan
             (b, 0.3, 1, 2), (b, 0.3, 1, 2),                   # other values, same length
             (b, 0.3, 7, 3),                                   # Theiler window and l_min
             (a[:2000], 0.3, 7, 3), (a[:2000], 0.3, 7, 3)]     # another length: a new plan
    r = gp.RQA(gpu_settings(3, 2, 0.4, 1, 1))
    for s, eps, w, lmin in steps:
        kw = dict(m=3, tau=2, eps=eps, norm=1, theiler=w, l_min=lmin, v_min=lmin, w_min=lmin)
        r.set_settings(gpu_settings(**kw))
        meas = r.run(s)
        _check(r, meas, s, **kw)


def test_replays_report_their_launches():
    s = synth.ar1(5000, 51, 0.9)
    r = gp.RQA(gpu_settings(3, 1, 0.5, 1, 1))
    counts = []
    for _ in range(4):
        r.run(s)
        st = r.stats()
        counts.append((st["launches"], st["ctas"]))
    assert counts[0][0] > 0 and all(c == counts[0] for c in counts), counts


def test_device_series_rewritten_in_place():
    """The same device buffer, new values written between calls: a replay
    must read the buffer again."""
    n = 3000
    t = torch.empty(n, dtype=torch.float64, device="cuda")
    kw = dict(m=4, tau=1, eps=0.5, norm=0, theiler=2)
    r = gp.RQA(gpu_settings(**kw))
    for seed in (31, 31, 32, 33, 33):
        s = synth.ar1(n, seed, 0.8)
        t.copy_(torch.from_numpy(s))
        meas = r.run(t)
        _check(r, meas, s, **kw)


def test_cross_repeated():
    x = synth.ar1(1500, 41, 0.9)
    y = synth.ar1(1700, 42, 0.9)
    kw = dict(m=2, tau=1, eps=0.4, norm=2, theiler=0)
    r = gp.RQA(gpu_settings(**kw))
    for _ in range(3):
        meas = r.run_cross(x, y)
        want = oracle.cross_rqa(x, y, oracle_settings(**kw))
        assert np.array_equal(r.histogram(0), want["hd"])
        assert_same_measures(meas, want["measures"])


def test_default_stream_work_is_waited_for():
    """A device series still being written by work queued on torch's default
    (the legacy) stream: a call given no stream runs after that work, as the
    entry points document."""
    n = 4000
    s = synth.ar1(n, 61, 0.9)
    src = torch.tensor(s, dtype=torch.float64, device="cuda")
    t = torch.zeros(n, dtype=torch.float64, device="cuda")
    assert torch.cuda.current_stream().cuda_stream == 0
    kw = dict(m=3, tau=1, eps=0.5, norm=1, theiler=1)
    r = gp.RQA(gpu_settings(**kw))
    for _ in range(2):           # a plain run, then a graph replay
        t.zero_()
        big = torch.randn(4096, 4096, device="cuda")
        for _ in range(12):      # tens of milliseconds of queued work first
            big = torch.tanh(big @ big)
        t.copy_(src)
        meas = r.run(t)
        _check(r, meas, s, **kw)
