"""Batched and served RQA through the C ABI: every series of a batch, and
every request of a served mix, must equal the FP64 oracle (and hence its own
single-series run) exactly; admission must queue under a small memory
budget and never exceed it; queued requests can be cancelled."""
import os
import threading
import time

import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same_measures

import paper_2402_16853_b300 as gp

pytestmark = pytest.mark.gpu


def _mixed(count, seed, lo=40, hi=3000):
    rng = np.random.default_rng(seed)
    specs = []
    for q in range(count):
        L = int(rng.integers(lo, hi))
        sp = synth.draw_spec(rng, L)
        specs.append(sp)
    series, eps = synth.make_series(specs, seed)
    settings = [gp.Settings(m=sp.m, tau=sp.tau, eps=e, norm=sp.norm, theiler=sp.theiler,
                            l_min=sp.l_min, v_min=sp.v_min, w_min=sp.w_min)
                for sp, e in zip(specs, eps)]
    return settings, series


def _oracle(st, s):
    return oracle.rqa(s, oracle.Settings(m=st.m, tau=st.tau, eps=st.eps, norm=st.norm,
                                         theiler=st.theiler, l_min=st.l_min, v_min=st.v_min,
                                         w_min=st.w_min))


def test_batch_equals_oracle_and_graph_replay():
    settings, series = _mixed(40, 11)
    # edge cases inside the batch: a single vector, a constant series, FP64 precision
    settings.append(gp.Settings(m=3, tau=2, eps=0.2, norm=1, theiler=0))
    series.append(np.array([0.1, 0.2, 0.3, 0.4, 0.5]))
    settings.append(gp.Settings(m=2, tau=1, eps=0.1, norm=0, theiler=1))
    series.append(np.full(700, 0.25))
    settings.append(gp.Settings(m=4, tau=3, eps=0.4, norm=2, theiler=2, precision=gp.PREC_FP64))
    series.append(synth.ar1(900, 5, 0.8))
    b = gp.Batch()
    res, st, rc = b.run(settings, series)
    assert rc == 0 and all(x == 0 for x in st)
    for q, (stg, s) in enumerate(zip(settings, series)):
        want = _oracle(stg, s)
        assert np.array_equal(b.histogram(q, 0), want["hd"]), q
        assert np.array_equal(b.histogram(q, 1), want["hv"]), q
        assert np.array_equal(b.histogram(q, 2), want["hw"]), q
        assert_same_measures(res[q], want["measures"])
    res2, st2, rc2 = b.run(settings, series)   # replays the captured graph
    assert rc2 == 0
    for m1, m2 in zip(res, res2):
        assert_same_measures(m2, m1)


def test_batch_failing_series_is_isolated():
    settings, series = _mixed(8, 12)
    bad = synth.ar1(500, 3, 0.9)
    bad[17] = np.inf
    settings.insert(3, gp.Settings(m=2, tau=1, eps=0.3, norm=1, theiler=1))
    series.insert(3, bad)
    settings.insert(5, gp.Settings(m=3, tau=4, eps=0.3, norm=1, theiler=1))
    series.insert(5, np.zeros(5))   # too short for the embedding
    b = gp.Batch()
    res, st, rc = b.run(settings, series)
    assert st[3] == 3 and st[5] == 2 and rc != 0
    for q, (stg, s) in enumerate(zip(settings, series)):
        if q in (3, 5):
            assert res[q] is None
            continue
        assert_same_measures(res[q], _oracle(stg, s)["measures"])


def test_served_results_equal_alone_and_in_the_mix():
    settings, series = _mixed(60, 13, lo=100, hi=6000)
    alone = []
    for stg, s in zip(settings, series):
        r = gp.RQA(stg)
        alone.append(r.run(s))
    srv = gp.Server(1 << 30, max_slots=16)
    try:
        _served_mix(srv, settings, series, alone)
    finally:
        srv.close()


def _served_mix(srv, settings, series, alone):
    tickets = []

    def submitter(lo, hi):
        for q in range(lo, hi):
            tickets.append((q, srv.submit(settings[q], series[q])))
            time.sleep(0.001)

    th = [threading.Thread(target=submitter, args=(k * 20, (k + 1) * 20)) for k in range(3)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for q, t in tickets:
        rc, m = srv.wait(t, 60_000)
        assert rc == 0, (q, rc)
        assert_same_measures(m, alone[q])
    c = srv.counters()
    assert c["completed"] == len(series) and c["bytes_in_use"] == 0 and c["epochs"] >= 1


def test_admission_small_budget_never_overcommits():
    settings, series = _mixed(30, 14, lo=2000, hi=4000)
    srv = gp.Server(24 << 20, max_slots=4)   # 24 MiB: a few requests at a time
    try:
        _admission(srv, settings, series)
    finally:
        srv.close()


def _admission(srv, settings, series):
    peak = [0, 0]
    stop = threading.Event()

    def watch():
        while not stop.is_set():
            c = srv.counters()
            peak[0] = max(peak[0], c["bytes_in_use"])
            peak[1] = max(peak[1], c["in_flight"])
            time.sleep(0.0005)

    w = threading.Thread(target=watch)
    w.start()
    try:
        ts = [srv.submit(stg, s) for stg, s in zip(settings, series)]
        for t, stg, s in zip(ts, settings, series):
            rc, m = srv.wait(t, 60_000)
            assert rc == 0
            assert_same_measures(m, _oracle(stg, s)["measures"])
    finally:
        stop.set()
        w.join()
    assert 0 < peak[0] <= 24 << 20 and 1 <= peak[1] <= 4


def test_memory_held_between_epochs_stays_within_budget():
    """Each worker keeps its device arena from epoch to epoch; one larger than
    its share of the budget is released, so what the server holds once the
    stream is done stays within the budget."""
    import torch
    torch.zeros(1, device="cuda")
    settings, series = _mixed(40, 17, lo=20000, hi=60000)
    budget = 256 << 20
    srv = gp.Server(budget, max_slots=8)
    try:
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        ts = [srv.submit(stg, s) for stg, s in zip(settings, series)]
        got = []
        for t in ts:
            rc, m = srv.wait(t, 60_000)
            assert rc == 0
            got.append(m)
        time.sleep(0.2)
        held = free0 - torch.cuda.mem_get_info()[0]
        assert held <= budget, (held, budget)
        for q in (0, 13, 27, 39):   # the same results as single runs
            r = gp.RQA(settings[q])
            assert_same_measures(got[q], r.run(series[q]))
            r.close()
    finally:
        srv.close()


def test_oversized_request_and_cancel():
    srv = gp.Server(8 << 20, max_slots=1)
    try:
        _oversized_and_cancel(srv)
    finally:
        srv.close()


def _oversized_and_cancel(srv):
    big = synth.ar1(60000, 1, 0.9)
    with pytest.raises(gp.RQAError) as ei:
        srv.submit(gp.Settings(m=3, tau=1, eps=0.5, norm=1, theiler=1), big)
    assert ei.value.status == 4   # RQA_ENOMEM: more than the budget allows
    small = [synth.ar1(3000, k, 0.9) for k in range(6)]
    st = gp.Settings(m=3, tau=1, eps=0.5, norm=1, theiler=1)
    ts = [srv.submit(st, s) for s in small]
    # the last ones are still queued behind a single slot: cancel one
    rel = srv.release(ts[-1])
    assert rel in (0, 7)
    for t in ts[:-1]:
        rc, m = srv.wait(t, 60_000)
        assert rc == 0
    if rel == 0:
        assert srv.poll(ts[-1])[0] == 10   # forgotten


def test_served_banded_requests_equal_alone():
    """Requests of 70,000 points run in row bands in the server's epochs (and
    alone); results must equal the oracle and the single runs."""
    big = [synth.ar1(70_000, 41 + k, 0.9) for k in range(2)]
    small, eps_small = synth.make_series([synth.draw_spec(np.random.default_rng(7), 3000)
                                          for _ in range(6)], 8)
    settings = [gp.Settings(m=3, tau=1, eps=0.4, norm=1, theiler=1) for _ in big]
    settings += [gp.Settings(m=2, tau=1, eps=e, norm=0, theiler=1) for e in eps_small]
    series = big + small
    alone = []
    for stg, s in zip(settings, series):
        r = gp.RQA(stg)
        alone.append(r.run(s))
        if len(s) >= 70_000:
            assert r.stats()["band_rows"] > 0
    want = oracle.rqa(big[0], oracle.Settings(m=3, tau=1, eps=0.4, norm=1, theiler=1),
                      mode="streaming")
    assert_same_measures(alone[0], want["measures"])
    srv = gp.Server(8 << 30, max_slots=8)
    try:
        ts = [srv.submit(stg, s) for stg, s in zip(settings, series)]
        for t, a in zip(ts, alone):
            rc, m = srv.wait(t, 120_000)
            assert rc == 0
            assert_same_measures(m, a)
    finally:
        srv.close()


def test_preload_kernels_once_per_process():
    """Every tile kernel instantiation (m = 1..10, three norms, FP32 and FP64,
    RQA and cross, with and without row bands, at four columns per lane, the
    FP32 ones also at two, and the two matrix-input ones), the thirteen
    preparation and merge kernels and the set-up kernel of the
    allocation-free entry point (whose static scratch address is resolved at
    the same time) are loaded; a second call finds them loaded and reports
    the same count."""
    n = gp.preload_kernels()
    assert n == 10 * 3 * 2 * 2 * 2 + 10 * 3 * 2 * 2 + 2 + 13 + 1
    assert gp.preload_kernels() == n
    # a run afterwards is unaffected
    s = synth.ar1(600, 5, 0.9)
    st = gp.Settings(m=2, tau=1, eps=0.5, norm=1, theiler=1)
    want = oracle.rqa(s, oracle.Settings(m=2, tau=1, eps=0.5, norm=1, theiler=1))
    r = gp.RQA(st)
    r.run(s)
    hd, hv, hw = r.histograms()
    assert np.array_equal(hd, want["hd"]) and np.array_equal(hw, want["hw"])


def test_batch_cfg4_long_series_equal_oracle():
    """Series of the batched workload's upper lengths (5,000 to 20,000
    points): all three generators, m from 2 to 8, all norms, mixed in one
    batch so that several kernel classes run on the side streams with row
    bands, plus a short series alone in its class (no row bands).  Every
    histogram equals the FP64 oracle's."""
    rng = np.random.default_rng(4242)
    plan = [("logistic", 8, 19_800, 0), ("lorenz", 5, 12_000, 1), ("ar1", 2, 20_000, 2),
            ("logistic", 3, 5_100, 1), ("lorenz", 8, 16_000, 0), ("ar1", 7, 9_000, 2),
            ("ar1", 4, 17_500, 1), ("lorenz", 2, 7_300, 2), ("logistic", 6, 14_000, 0),
            ("ar1", 3, 400, 0)]
    specs = [synth.SeriesSpec(kind, L, m, int(rng.integers(1, 5)), norm,
                              float(rng.uniform(0.05, 0.5)),
                              float(rng.uniform(3.6, 4.0)) if kind == "logistic"
                              else float(rng.uniform(0.5, 0.99)) if kind == "ar1" else 0.0)
             for kind, m, L, norm in plan]
    series, eps = synth.make_series(specs, 4243)
    settings = [gp.Settings(m=sp.m, tau=sp.tau, eps=e, norm=sp.norm, theiler=sp.theiler)
                for sp, e in zip(specs, eps)]
    b = gp.Batch()
    res, st, rc = b.run(settings, series)
    assert rc == 0 and all(x == 0 for x in st)
    for q, (stg, s) in enumerate(zip(settings, series)):
        want = _oracle(stg, s)
        for kind, key in ((0, "hd"), (1, "hv"), (2, "hw")):
            assert np.array_equal(b.histogram(q, kind), want[key]), (q, key)
        assert_same_measures(res[q], want["measures"])
    b.close()


def test_run_batch_on_a_caller_stream():
    """rqa_run_batch (the batched call with the boundary's shape): its
    device work is ordered after work already queued on the caller's stream,
    its measures equal those of the batch object and of the oracle, and a
    second call with the same shapes (graph replay) repeats them."""
    import torch
    settings, series = _mixed(24, 77, lo=300, hi=6000)
    b = gp.Batch()
    want, st, rc = b.run(settings, series)
    assert rc == 0
    b.close()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        busy = torch.empty(1 << 28, dtype=torch.float32, device="cuda")
        busy.fill_(1.0)   # queued ahead of the batch on the same stream
    for _ in range(2):
        got, rc = gp.run_batch(settings, series, stream)
        assert rc == 0
        for g, w in zip(got, want):
            assert_same_measures(g, w)
    for q in (0, 5, 11):
        assert_same_measures(got[q], _oracle(settings[q], series[q])["measures"])
    gp.run_batch_release()
    del busy


def test_set_settings_reuses_one_handle():
    """rqa_set_settings: one handle runs series with different parameters
    (the sequential baseline of the batched benchmark); each result equals a
    fresh handle's and the oracle's, and invalid settings are refused while
    the previous ones stay in force."""
    settings, series = _mixed(6, 91, lo=500, hi=4000)
    r = gp.RQA(settings[0])
    for stg, s in zip(settings, series):
        r.set_settings(stg)
        got = r.run(s)
        assert_same_measures(got, _oracle(stg, s)["measures"])
    with pytest.raises(gp.RQAError) as ei:
        r.set_settings(gp.Settings(m=0, tau=1, eps=0.5))
    assert ei.value.status == 1
    again = r.run(series[-1])           # still the last valid settings
    assert_same_measures(again, _oracle(settings[-1], series[-1])["measures"])
    r.close()


def test_served_stream_equals_single_runs():
    """A Poisson stream with the served workload's lengths (1,000-200,000
    points) and parameters, submitted on its arrival schedule: every result
    equals the same series' single run (which the parity tests pin to the
    oracle).  RQA_SERVE_TEST_SECONDS sets the stream's length (4 s; 60 s is
    the measured workload's)."""
    seconds = float(os.environ.get("RQA_SERVE_TEST_SECONDS", "4"))
    arrivals, specs, series, eps = synth.serve_stream(rate=200.0, duration=seconds, seed=1105)
    settings = [gp.Settings(m=sp.m, tau=sp.tau, eps=e, norm=sp.norm, theiler=sp.theiler,
                            l_min=sp.l_min, v_min=sp.v_min, w_min=sp.w_min)
                for sp, e in zip(specs, eps)]
    srv = gp.Server(40 << 30, max_slots=64)
    try:
        t0 = time.perf_counter()
        tickets = []
        for at, stg, s in zip(arrivals, settings, series):
            wait = at - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            tickets.append(srv.submit(stg, s))
        got = []
        for t in tickets:
            rc, m = srv.wait(t, 120_000)
            assert rc == 0
            got.append(m)
    finally:
        srv.close()
    r = gp.RQA(settings[0])
    for q, (stg, s) in enumerate(zip(settings, series)):
        r.set_settings(stg)
        assert_same_measures(got[q], r.run(s))
    r.close()
