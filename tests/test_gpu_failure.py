"""Failure detection without a GPU fault: the tile kernel's bounded wait,
run on a counter that nothing raises, gives up after its limit (about two
seconds of SM clock), raises the abort flag and reports RQA_ETIMEOUT; the
context stays usable for the next computation.  The same happens inside the
real tile kernel when a warp withholds its carries (a test instantiation
with a short limit)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same_measures, gpu_settings, oracle_settings

import paper_2402_16853_b300 as gp

pytestmark = pytest.mark.gpu

SPIN_CYCLES = 4_000_000_000  # the kernel's wait limit


def test_bounded_wait_gives_up_and_context_survives():
    status, cycles = gp.selftest_bounded_wait()
    assert status == 6                       # RQA_ETIMEOUT
    assert SPIN_CYCLES < cycles < 4 * SPIN_CYCLES
    s = synth.logistic(900, 5)
    r = gp.RQA(gpu_settings(3, 2, 0.1, 1, 1))
    meas = r.run(s)
    want = oracle.rqa(s, oracle_settings(3, 2, 0.1, 1, 1))
    assert np.array_equal(r.histogram(0), want["hd"])
    assert_same_measures(meas, want["measures"])


def test_ring_wait_in_the_tile_kernel_times_out():
    """The real tile kernel's hand-over wait (warp w+1 waiting for warp w's
    row and diagonal carries) in its test instantiation, with warp 1 of
    every CTA withholding its hand-overs from the third on: the waiting warp
    gives up after 10^6 cycles, every CTA aborts, and the run returns
    RQA_ETIMEOUT with no fault and no hang.  The same handle then runs the
    same series exactly, and the test instantiation is exact when the
    withheld hand-over is never reached."""
    s = synth.ar1(20_000, 41, 0.95)
    p = dict(m=3, tau=1, eps=0.5, norm=1, theiler=1)
    r = gp.RQA(gpu_settings(**p))
    assert r.selftest_ring_timeout(s, warp=1, from_handover=3) == 6
    assert r.selftest_ring_timeout(s, warp=5, from_handover=1) == 6
    want = oracle.rqa(s, oracle_settings(**p))
    meas = r.run(s)
    hd, hv, hw = r.histograms()
    assert np.array_equal(hd, want["hd"]) and np.array_equal(hv, want["hv"])
    assert np.array_equal(hw, want["hw"])
    assert_same_measures(meas, want["measures"])
    small = synth.ar1(3000, 42, 0.9)
    assert r.selftest_ring_timeout(small, warp=2, from_handover=10**6) == 0
    assert_same_measures(r.measures(), oracle.rqa(small, oracle_settings(**p))["measures"])
    r4 = gp.RQA(gpu_settings(4, 1, 0.5, 1, 1))   # only m = 3, L2 has the test instantiation
    assert r4.selftest_ring_timeout(s) == 1
