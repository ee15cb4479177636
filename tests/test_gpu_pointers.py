"""Device pointers a caller hands to the device entry points are checked
before any kernel reads them: a misaligned pointer or pageable host memory
is refused with RQA_EINVAL (a kernel reading it would fault the device), the
handle stays usable, and mapped pinned host memory, which the device can
read, is accepted and gives the oracle's result."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import assert_same_measures, gpu_settings, oracle_settings

import paper_2402_16853_b300 as gp
from paper_2402_16853_b300.rqa import _CSettings, _cs

pytestmark = pytest.mark.gpu

KW = dict(m=3, tau=1, eps=0.5, norm=1, theiler=1)


def _run_ptr(r, ptr, n):
    lib = gp.load()
    rc = lib.rqa_run_device(r._h, ctypes.c_void_p(ptr), n, ctypes.c_void_p(0))
    return rc, lib.rqa_last_error(r._h).decode()


def test_misaligned_and_host_pointers_refused():
    s = synth.ar1(3000, 71, 0.9)
    t = torch.zeros(len(s) + 1, dtype=torch.float64, device="cuda")
    r = gp.RQA(gpu_settings(**KW))
    rc, msg = _run_ptr(r, t.data_ptr() + 4, len(s))
    assert rc == 1 and "aligned" in msg, (rc, msg)
    host = np.ascontiguousarray(s)
    rc, msg = _run_ptr(r, host.ctypes.data, len(s))
    assert rc == 1 and "host memory" in msg, (rc, msg)
    # the handle still runs a proper series afterwards
    t[: len(s)].copy_(torch.from_numpy(s))
    meas = r.run(t[: len(s)])
    want = oracle.rqa(s, oracle_settings(**KW))
    assert np.array_equal(r.histogram(0), want["hd"])
    assert_same_measures(meas, want["measures"])


def test_pinned_host_series_is_read_in_place():
    s = synth.ar1(2500, 72, 0.9)
    pinned = torch.from_numpy(s.copy()).pin_memory()
    r = gp.RQA(gpu_settings(**KW))
    rc, msg = _run_ptr(r, pinned.data_ptr(), len(s))
    assert rc == 0, msg
    want = oracle.rqa(s, oracle_settings(**KW))
    hd, hv, hw = r.histograms()
    assert np.array_equal(hd, want["hd"]) and np.array_equal(hv, want["hv"])
    assert np.array_equal(hw, want["hw"])


def test_noalloc_refuses_bad_pointers():
    lib = gp.load()
    f = lib.rqa_run_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(_CSettings), ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_void_p]
    lib.rqa_noalloc_last_error.restype = ctypes.c_char_p
    lib.rqa_noalloc_last_error.argtypes = []
    s = synth.ar1(2000, 73, 0.9)
    t = torch.tensor(s, dtype=torch.float64, device="cuda")
    n = len(s) - 2
    out = torch.zeros(3 * (n + 1) + 1, dtype=torch.int64, device="cuda")
    cs = _cs(gpu_settings(**KW))
    rc = f(ctypes.byref(cs), ctypes.c_void_p(t.data_ptr()), len(s),
           ctypes.c_void_p(out.data_ptr() + 4), ctypes.c_void_p(0))
    assert rc == 1 and "aligned" in lib.rqa_noalloc_last_error().decode()
    host = np.ascontiguousarray(s)
    rc = f(ctypes.byref(cs), ctypes.c_void_p(host.ctypes.data), len(s),
           ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(0))
    assert rc == 1 and "host memory" in lib.rqa_noalloc_last_error().decode()
    rc = f(ctypes.byref(cs), ctypes.c_void_p(t.data_ptr()), len(s),
           ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(0))
    assert rc == 0, lib.rqa_noalloc_last_error().decode()
