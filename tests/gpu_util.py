"""Helpers shared by the GPU parity tests: run the CUDA path through the C
ABI and compare with the oracle bit for bit."""
import math

import numpy as np

import oracle
import paper_2402_16853_b300 as gp


def oracle_settings(m, tau, eps, norm, theiler, l_min=2, v_min=2, w_min=2):
    return oracle.Settings(m=m, tau=tau, eps=eps, norm=norm, theiler=theiler, l_min=l_min,
                           v_min=v_min, w_min=w_min)


def gpu_settings(m, tau, eps, norm, theiler, l_min=2, v_min=2, w_min=2, precision=0,
                 band_override=-1.0):
    return gp.Settings(m=m, tau=tau, eps=eps, norm=norm, theiler=theiler, l_min=l_min,
                       v_min=v_min, w_min=w_min, precision=precision,
                       band_override=band_override)


def same_float(a, b):
    if isinstance(a, float) and math.isnan(a):
        return isinstance(b, float) and math.isnan(b)
    return np.float64(a).view(np.uint64) == np.float64(b).view(np.uint64)


def assert_same_measures(got, want):
    for k, v in want.items():
        assert k in got, k
        if isinstance(v, float):
            assert same_float(got[k], v), (k, got[k], v)
        else:
            assert got[k] == v, (k, got[k], v)


def run_gpu(series, **kw):
    r = gp.RQA(gpu_settings(**kw))
    meas = r.run(series)
    hd, hv, hw = r.histograms()
    st = r.stats()
    return r, meas, hd, hv, hw, st


def check_parity(series, mode="auto", **kw):
    """Run both sides and compare histograms and measures exactly."""
    okw = {k: v for k, v in kw.items() if k not in ("precision", "band_override")}
    want = oracle.rqa(series, oracle_settings(**okw), mode=mode)
    r, meas, hd, hv, hw, st = run_gpu(series, **kw)
    assert np.array_equal(hd, want["hd"]), _diff("diag", hd, want["hd"])
    assert np.array_equal(hv, want["hv"]), _diff("vert", hv, want["hv"])
    assert np.array_equal(hw, want["hw"]), _diff("white", hw, want["hw"])
    assert_same_measures(meas, want["measures"])
    return r, st, want


def _diff(name, got, want):
    idx = np.nonzero(got != want)[0][:10]
    return f"{name} histogram differs at lengths {idx.tolist()}: " \
           f"gpu {got[idx].tolist()} oracle {want[idx].tolist()}"
