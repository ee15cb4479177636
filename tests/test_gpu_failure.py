"""Failure detection without a GPU fault: the tile kernel's bounded wait,
run on a counter that nothing raises, gives up after its limit (about two
seconds of SM clock), raises the abort flag and reports RQA_ETIMEOUT; the
context stays usable for the next computation."""
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
