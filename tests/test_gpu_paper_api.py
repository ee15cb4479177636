"""The paper's workflow (Sect. 7): Settings with a similarity measure and a
fixed-radius neighbourhood, RQAComputation.create(...).run() returning an
RQAResult with one member per measure, RecurrencePlotComputation returning
the matrix -- all equal to the oracle."""
import math

import numpy as np
import pytest

import oracle
import synth
from paper_2402_16853_b300.paper_api import (EuclideanMetric, FixedRadius, MaximumMetric,
                                             RecurrencePlotComputation, RQAComputation,
                                             Settings, TaxicabMetric)

pytestmark = pytest.mark.gpu

NAMES = {"rr": "recurrence_rate", "det": "determinism", "l": "average_diagonal_line",
         "l_max": "longest_diagonal_line", "div": "divergence", "l_entr": "entropy_diagonal_lines",
         "lam": "laminarity", "tt": "trapping_time", "v_max": "longest_vertical_line",
         "v_entr": "entropy_vertical_lines", "w": "average_white_vertical_line",
         "w_max": "longest_white_vertical_line", "w_entr": "entropy_white_vertical_lines",
         "n_vec": "number_of_vectors", "recurrence_points": "recurrence_points"}


def _same(a, b):
    return (isinstance(a, float) and math.isnan(a) and math.isnan(b)) or a == b


@pytest.mark.parametrize("metric,norm", [(MaximumMetric, 0), (EuclideanMetric, 1),
                                         (TaxicabMetric, 2)])
def test_rqa_workflow(metric, norm):
    s = synth.logistic(1200, 3)
    settings = Settings(s, embedding_dimension=2, time_delay=3, similarity_measure=metric,
                        neighbourhood=FixedRadius(0.1), theiler_window=1)
    result = RQAComputation.create(settings).run()
    want = oracle.rqa(s, oracle.Settings(m=2, tau=3, eps=0.1, norm=norm, theiler=1))
    for k, attr in NAMES.items():
        assert _same(getattr(result, attr), want["measures"][k]), attr
    assert np.array_equal(result.diagonal_frequency_distribution, want["hd"])
    assert "Determinism (DET)" in str(result)


def test_cross_and_matrix_workflow():
    x, y = synth.ar1(900, 1, 0.9), synth.ar1(700, 2, 0.9)
    settings = Settings((x, y), embedding_dimension=3, time_delay=1,
                        neighbourhood=FixedRadius(0.5))
    result = RQAComputation.create(settings).run()
    want = oracle.cross_rqa(x, y, oracle.Settings(m=3, tau=1, eps=0.5, norm=1, theiler=0))
    assert _same(result.determinism, want["measures"]["det"])
    plot = RecurrencePlotComputation.create(settings).run().recurrence_matrix
    again = RQAComputation.create(Settings(plot)).run()
    assert np.array_equal(again.diagonal_frequency_distribution, want["hd"])
    assert np.array_equal(again.white_vertical_frequency_distribution, want["hw"])


def test_plot_workflow(tmp_path):
    s = synth.lorenz_x(300, 4)
    settings = Settings(s, embedding_dimension=3, time_delay=2, similarity_measure=MaximumMetric,
                        neighbourhood=FixedRadius(0.4))
    res = RecurrencePlotComputation.create(settings).run()
    want, _ = oracle.matrix(s, oracle.Settings(m=3, tau=2, eps=0.4, norm=0, theiler=0))
    assert np.array_equal(res.recurrence_matrix, want)
    res.save(str(tmp_path / "plot.pgm"))
    assert (tmp_path / "plot.pgm").read_bytes().startswith(b"P5\n296 296\n255\n")
