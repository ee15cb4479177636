"""The paper's analysis workflow (Sect. 7, Table 2) over the GPU library.

A PyRQA user writes against a handful of object classes: a `Settings` bundle
holding the time series, the embedding parameters, a similarity measure and a
fixed-radius neighbourhood (Sect. 7.2); `RQAComputation` and
`RecurrencePlotComputation`, created from the settings by a static `create`
and executed by `run` (Sect. 7.3); and the `RQAResult` / `RecurrencePlotResult`
they return, with one member per measure (Sect. 7.4, Table 3).  This module
offers the same workflow with the same class names, mapped onto the C ABI;
everything runs on the GPU (there is no OpenCL environment to choose: the
current CUDA device is used).  Beyond the paper's version, a pair of series
as `time_series` selects cross recurrence (Sect. 3.3), a 2-D 0/1 array
selects a precomputed matrix (Sect. 9), and `theiler_window` excludes cells
with |i - j| < w.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import rqa as _r

__all__ = ["MaximumMetric", "EuclideanMetric", "TaxicabMetric", "FixedRadius", "Settings",
           "RQAComputation", "RQAResult", "RecurrencePlotComputation", "RecurrencePlotResult"]


class MaximumMetric:
    """L-infinity norm."""
    norm = _r.NORM_MAX


class EuclideanMetric:
    """L2 norm."""
    norm = _r.NORM_L2


class TaxicabMetric:
    """L1 norm."""
    norm = _r.NORM_L1


@dataclass(frozen=True)
class FixedRadius:
    """Neighbourhood condition d(x_i, x_j) <= radius."""
    radius: float = 1.0


@dataclass
class Settings:
    """Analysis parameters.  `time_series`: one series (RQA), a pair of
    series (cross recurrence) or a 2-D 0/1 array (a precomputed matrix)."""
    time_series: object
    embedding_dimension: int = 1
    time_delay: int = 1
    similarity_measure: type = EuclideanMetric
    neighbourhood: FixedRadius = field(default_factory=FixedRadius)
    theiler_window: int = 0
    min_diagonal_line_length: int = 2
    min_vertical_line_length: int = 2
    min_white_vertical_line_length: int = 2

    def _kind(self) -> str:
        ts = self.time_series
        if isinstance(ts, (tuple, list)) and len(ts) == 2 and np.ndim(ts[0]) == 1:
            return "cross"
        return "matrix" if np.ndim(ts) == 2 else "rqa"

    def _native(self) -> _r.Settings:
        return _r.Settings(m=int(self.embedding_dimension), tau=int(self.time_delay),
                           eps=float(self.neighbourhood.radius),
                           norm=int(self.similarity_measure.norm),
                           theiler=int(self.theiler_window),
                           l_min=int(self.min_diagonal_line_length),
                           v_min=int(self.min_vertical_line_length),
                           w_min=int(self.min_white_vertical_line_length))


@dataclass
class RQAResult:
    """The quantitative measures of Table 3 (plus the white vertical line
    measures) and the three line-length distributions (entry l = number of
    lines of length l)."""
    settings: Settings
    number_of_vectors: int
    recurrence_points: int
    recurrence_rate: float
    determinism: float
    average_diagonal_line: float
    longest_diagonal_line: int
    divergence: float
    entropy_diagonal_lines: float
    laminarity: float
    trapping_time: float
    longest_vertical_line: int
    entropy_vertical_lines: float
    average_white_vertical_line: float
    longest_white_vertical_line: int
    entropy_white_vertical_lines: float
    diagonal_frequency_distribution: np.ndarray
    vertical_frequency_distribution: np.ndarray
    white_vertical_frequency_distribution: np.ndarray

    def __str__(self) -> str:
        rows = [("Recurrence rate (RR)", self.recurrence_rate),
                ("Determinism (DET)", self.determinism),
                ("Average diagonal line length (L)", self.average_diagonal_line),
                ("Longest diagonal line length (L_max)", self.longest_diagonal_line),
                ("Divergence (DIV)", self.divergence),
                ("Entropy diagonal lines (L_entr)", self.entropy_diagonal_lines),
                ("Laminarity (LAM)", self.laminarity),
                ("Trapping time (TT)", self.trapping_time),
                ("Longest vertical line length (V_max)", self.longest_vertical_line),
                ("Entropy vertical lines (V_entr)", self.entropy_vertical_lines),
                ("Average white vertical line length (W)", self.average_white_vertical_line),
                ("Longest white vertical line length (W_max)",
                 self.longest_white_vertical_line),
                ("Entropy white vertical lines (W_entr)", self.entropy_white_vertical_lines)]
        return "\n".join(f"{name}: {value}" for name, value in rows)


class RQAComputation:
    """An RQA computation on the current GPU."""

    def __init__(self, settings: Settings):
        self.settings = settings
        self._h = _r.RQA(settings._native())

    @staticmethod
    def create(settings: Settings, **_ignored) -> "RQAComputation":
        return RQAComputation(settings)

    def run(self) -> RQAResult:
        st = self.settings
        kind = st._kind()
        if kind == "cross":
            x, y = st.time_series
            m = self._h.run_cross(np.asarray(x, np.float64), np.asarray(y, np.float64))
        elif kind == "matrix":
            m = self._h.run_matrix(np.asarray(st.time_series))
        else:
            m = self._h.run(np.asarray(st.time_series, np.float64))
        hd, hv, hw = self._h.histograms()
        return RQAResult(settings=st, number_of_vectors=m["n_vec"],
                         recurrence_points=m["recurrence_points"], recurrence_rate=m["rr"],
                         determinism=m["det"], average_diagonal_line=m["l"],
                         longest_diagonal_line=m["l_max"], divergence=m["div"],
                         entropy_diagonal_lines=m["l_entr"], laminarity=m["lam"],
                         trapping_time=m["tt"], longest_vertical_line=m["v_max"],
                         entropy_vertical_lines=m["v_entr"], average_white_vertical_line=m["w"],
                         longest_white_vertical_line=m["w_max"],
                         entropy_white_vertical_lines=m["w_entr"],
                         diagonal_frequency_distribution=hd,
                         vertical_frequency_distribution=hv,
                         white_vertical_frequency_distribution=hw)


@dataclass
class RecurrencePlotResult:
    """The recurrence matrix as a 0/1 uint8 array (row i, column j)."""
    settings: Settings
    recurrence_matrix: np.ndarray

    def save(self, path: str) -> None:
        """Write the plot as a binary PGM image (recurrences black)."""
        _r.write_pgm(path, self.recurrence_matrix)


class RecurrencePlotComputation:
    """A recurrence-plot computation on the current GPU; `window` =
    (i0, j0, rows, cols) restricts it to part of the matrix."""

    def __init__(self, settings: Settings, window: Optional[tuple] = None):
        self.settings = settings
        self.window = window

    @staticmethod
    def create(settings: Settings, window: Optional[tuple] = None,
               **_ignored) -> "RecurrencePlotComputation":
        return RecurrencePlotComputation(settings, window)

    def run(self) -> RecurrencePlotResult:
        st = self.settings
        i0, j0, rows, cols = self.window if self.window else (0, 0, None, None)
        kind = st._kind()
        if kind == "cross":
            x, y = st.time_series
            plot = _r.cross_recurrence_plot(st._native(), x, y, i0, j0, rows, cols)
        elif kind == "rqa":
            plot = _r.recurrence_plot(st._native(), st.time_series, i0, j0, rows, cols)
        else:
            raise ValueError("a precomputed matrix is already a recurrence plot")
        return RecurrencePlotResult(settings=st, recurrence_matrix=plot)
