"""rqa_run_noalloc: the entry point for callers that cannot let the library
allocate device memory (programs that own the whole GPU through their own
pool, services that must keep a fixed device footprint, paths where
cudaMalloc's device-wide synchronisation is unacceptable).  It keeps all
intermediate buffers in one static device array; these tests check, through
the C ABI, that its histograms equal those of the allocating entry point
(exactly: they are integers) on two calls in a row and those of the FP64
oracle, that a failed call (non-finite input) leaves the shared array fit
for the next one, that Theiler windows far beyond n behave as a window of n,
that band overrides it cannot report are refused, and that oversized series
are refused before anything runs.  This file is collected last."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
import paper_2402_16853_b300 as gp
from paper_2402_16853_b300.rqa import _CSettings, _cs

pytestmark = pytest.mark.gpu

MAX_N = 32768


def _lib():
    lib = gp.load()
    f = lib.rqa_run_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(_CSettings), ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_void_p]
    lib.rqa_noalloc_last_error.restype = ctypes.c_char_p
    lib.rqa_noalloc_last_error.argtypes = []
    return lib


def _run_noalloc(settings, series):
    import torch
    lib = _lib()
    t = torch.tensor(series, dtype=torch.float64, device="cuda")
    n = len(series) - (settings.m - 1) * settings.tau
    out = torch.full((3 * (n + 1),), 7, dtype=torch.int64, device="cuda")  # stale contents
    stream = torch.cuda.current_stream()
    cs = _cs(settings)
    rc = lib.rqa_run_noalloc(ctypes.byref(cs), ctypes.c_void_p(t.data_ptr()), len(series),
                             ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    msg = lib.rqa_noalloc_last_error().decode()
    h = out.cpu().numpy().view(np.uint64).reshape(3, n + 1)
    return rc, msg, h


def _run_regular(settings, series):
    r = gp.RQA(settings)
    r.run(series)
    return np.stack(r.histograms())


def test_noalloc_matches_allocating_entry_point_twice():
    cases = [
        (gp.Settings(m=3, tau=2, eps=0.1, norm=1, theiler=1), synth.logistic(2000, 1001)),
        (gp.Settings(m=4, tau=1, eps=0.6, norm=0, theiler=3), synth.ar1(9000, 77, 0.9)),
    ]
    for settings, series in cases:   # two calls in a row on the shared scratch
        rc, msg, got = _run_noalloc(settings, series)
        assert rc == 0, msg
        want = _run_regular(settings, series)
        assert np.array_equal(got, want)


def test_noalloc_largest_size_and_fp64():
    s = synth.ar1(MAX_N + 2, 5, 0.95)
    st = gp.Settings(m=3, tau=1, eps=0.5, norm=1, theiler=1)
    rc, msg, got = _run_noalloc(st, s)
    assert rc == 0, msg
    assert np.array_equal(got, _run_regular(st, s))
    st64 = gp.Settings(m=2, tau=3, eps=0.3, norm=2, theiler=1, precision=gp.PREC_FP64)
    s2 = synth.lorenz_x(3000, 6, discard=500)
    rc, msg, got = _run_noalloc(st64, s2)
    assert rc == 0, msg
    assert np.array_equal(got, _run_regular(st64, s2))


def test_noalloc_refuses_oversized_series():
    st = gp.Settings(m=1, tau=1, eps=0.5, norm=1, theiler=1)
    rc, msg, _ = _run_noalloc(st, np.zeros(MAX_N + 1))
    assert rc == 9 and "RQA_NOALLOC_MAX_N" in msg


def _oracle_hists(settings, series):
    p = dict(m=settings.m, tau=settings.tau, eps=settings.eps, norm=settings.norm,
             theiler=settings.theiler)
    want = oracle.rqa(series, oracle.Settings(**p))
    return np.stack([want["hd"], want["hv"], want["hw"]])


def test_noalloc_equals_oracle():
    """The histograms straight against the FP64 oracle (no other GPU path in
    between): the logistic workload of 2,000 points and a Lorenz series with
    row counts that leave ragged tiles."""
    cases = [
        (gp.Settings(m=3, tau=2, eps=0.1, norm=1, theiler=1), synth.logistic(2000, 1001)),
        (gp.Settings(m=5, tau=3, eps=0.3, norm=0, theiler=5), synth.lorenz_x(4111, 12, discard=800)),
        (gp.Settings(m=2, tau=1, eps=0.4, norm=2, theiler=0), synth.ar1(3333, 13, 0.9)),
    ]
    for settings, series in cases:
        rc, msg, got = _run_noalloc(settings, series)
        assert rc == 0, msg
        assert np.array_equal(got, _oracle_hists(settings, series))


def test_noalloc_nan_then_clean_call():
    """A non-finite value fails the call with RQA_ENAN; the next call on the
    shared array starts from a cleared status word and is exact."""
    st = gp.Settings(m=3, tau=1, eps=0.5, norm=1, theiler=1)
    bad = synth.ar1(5000, 21, 0.9)
    bad[1234] = np.nan
    rc, msg, _ = _run_noalloc(st, bad)
    assert rc == 3, msg
    good = synth.ar1(5000, 22, 0.9)
    rc, msg, got = _run_noalloc(st, good)
    assert rc == 0, msg
    assert np.array_equal(got, _run_regular(st, good))


def test_noalloc_theiler_beyond_n():
    """theiler = 2^31 - 1 passes validation; every cell is inside the window,
    so the matrix is all white, exactly as the allocating entry point says."""
    series = synth.ar1(3000, 23, 0.9)
    st = gp.Settings(m=2, tau=1, eps=0.5, norm=1, theiler=2 ** 31 - 1)
    rc, msg, got = _run_noalloc(st, series)
    assert rc == 0, msg
    want = _run_regular(st, series)
    assert np.array_equal(got, want)
    n = len(series) - 1
    assert got[0].sum() == 0 and got[1].sum() == 0 and got[2][n] == n


def test_noalloc_band_override_rules():
    """+inf (every pair re-decided in FP64) is exact and accepted; a finite
    band, which could be below the proven bound, is refused."""
    series = synth.ar1(2500, 24, 0.9)
    st = gp.Settings(m=3, tau=1, eps=0.5, norm=1, theiler=1, band_override=float("inf"))
    rc, msg, got = _run_noalloc(st, series)
    assert rc == 0, msg
    assert np.array_equal(got, _run_regular(gp.Settings(m=3, tau=1, eps=0.5, norm=1, theiler=1),
                                            series))
    st2 = gp.Settings(m=3, tau=1, eps=0.5, norm=1, theiler=1, band_override=1e-3)
    rc, msg, _ = _run_noalloc(st2, series)
    assert rc == 1 and "band_override" in msg
