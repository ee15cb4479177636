"""rqa_run_noalloc: the entry point for callers that cannot let the library
allocate device memory (programs that own the whole GPU through their own
pool, services that must keep a fixed device footprint, paths where
cudaMalloc's device-wide synchronisation is unacceptable).  It keeps all
intermediate buffers in one static device array; these tests check, through
the C ABI, that its histograms equal those of the allocating entry point
(exactly: they are integers) on two calls in a row, and that oversized
series are refused before anything runs.  This file is collected last."""
import ctypes

import numpy as np
import pytest

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
