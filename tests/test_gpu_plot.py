"""Recurrence plot (the paper's RecurrencePlotComputation, Table 2): windows
of the matrix computed on the GPU equal the oracle's materialised matrix
cell by cell, for every norm, with and without a Theiler window, with
windows that are ragged (not multiples of 32) or reach past the border."""
import os

import numpy as np
import pytest

import oracle
import synth

import paper_2402_16853_b300 as gp

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("norm", [0, 1, 2])
@pytest.mark.parametrize("w", [0, 1, 4])
def test_plot_equals_oracle_matrix(norm, w):
    s = synth.logistic(803, 40 + norm + w)
    st = gp.Settings(m=3, tau=2, eps=0.12, norm=norm, theiler=w)
    R, _ = oracle.matrix(s, oracle.Settings(m=3, tau=2, eps=0.12, norm=norm, theiler=w))
    got = gp.recurrence_plot(st, s)
    assert got.shape == R.shape and np.array_equal(got, R)
    part = gp.recurrence_plot(st, s, i0=37, j0=101, rows=250, cols=301)
    assert np.array_equal(part, R[37:287, 101:402])
    edge = gp.recurrence_plot(st, s, i0=700, j0=750, rows=150, cols=77)
    want = np.zeros((150, 77), np.uint8)
    want[:99, :49] = R[700:799, 750:799]
    assert np.array_equal(edge, want)


def test_plot_fp64_and_ties_and_pgm(tmp_path):
    s = synth.dyadic(400, 3, levels=4, scale_log2=-1)
    st = gp.Settings(m=2, tau=1, eps=0.5, norm=1, theiler=1, precision=gp.PREC_FP64)
    R, _ = oracle.matrix(s, oracle.Settings(m=2, tau=1, eps=0.5, norm=1, theiler=1))
    got = gp.recurrence_plot(st, s)
    assert np.array_equal(got, R)
    got32 = gp.recurrence_plot(gp.Settings(m=2, tau=1, eps=0.5, norm=1, theiler=1), s)
    assert np.array_equal(got32, R)
    path = os.path.join(tmp_path, "rp.pgm")
    gp.write_pgm(path, got)
    data = open(path, "rb").read()
    assert data.startswith(b"P5\n399 399\n255\n") and len(data) == 15 + 399 * 399


@pytest.mark.parametrize("m", range(1, 11))
def test_plot_every_m(m):
    s = synth.ar1(420 + m, 60 + m, 0.95)
    norm = m % 3
    eps = 0.3 * m if norm == 2 else 0.3 * (m ** 0.5 if norm == 1 else 1.0)
    st = gp.Settings(m=m, tau=1, eps=eps, norm=norm, theiler=m % 4)
    R, _ = oracle.matrix(s, oracle.Settings(m=m, tau=1, eps=eps, norm=norm, theiler=m % 4))
    assert np.array_equal(gp.recurrence_plot(st, s), R)
    assert np.array_equal(gp.recurrence_plot(st, s, i0=33, j0=5, rows=101, cols=70),
                          R[33:134, 5:75])
