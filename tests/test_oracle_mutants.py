"""The pins must catch plausible mistakes in the oracle.

Each case copies the oracle's C source, plants one mistake (a strict tie, a
Theiler off-by-one, a wrong norm, a wrong vector count, dropped border or
single-cell lines, a wrong log base, a wrong denominator, a missed longest
line; for cross recurrence a missing first or last diagonal, a one-sided
Theiler window, a wrong RR denominator), builds the copy (every occurrence
of the anchor replaced), and runs the pin suite against it in a subprocess:
the suite must fail.  Everything runs on the CPU.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "rqa_oracle.c")

MUTANTS = {
    "strict_tie": ("st->norm) <= st->eps;", "st->norm) < st->eps;"),
    "theiler_off_by_one": ("if (gap < (int64_t)st->theiler) return 0;",
                           "if (gap <= (int64_t)st->theiler) return 0;"),
    "l2_as_l1": ("acc = acc + diff * diff;", "acc = acc + fabs(diff);"),
    "l1_without_abs": ("acc = acc + fabs(diff);", "acc = acc + diff;"),
    "nvec_wrong": ("int64_t n = N - (int64_t)(m - 1) * (int64_t)tau;",
                   "int64_t n = N - (int64_t)m * (int64_t)tau;"),
    "drop_single_cells": ("if (len <= 0) return;", "if (len <= 1) return;"),
    "drop_border_runs": ("  if (prev >= 0) close_run(hv, hw, prev, run);\n  return ones;",
                         "  return ones;"),
    "log2_entropy": ("acc = acc + p * log(p);", "acc = acc + p * log2(p);"),
    "det_wrong_denominator": ("out->det = (double)d1 / (double)dall1;",
                              "out->det = (double)d1 / (double)d0;"),
    "lmax_misses_n": ("for (int64_t l = n; l >= lo; --l)",
                      "for (int64_t l = n - 1; l >= lo; --l)"),
    "tau_ignored": ("double b = s[j + (int64_t)k * tau];", "double b = s[j + (int64_t)k];"),
}

# Mistakes in the cross-recurrence code, caught by the cross pins.
CROSS_MUTANTS = {
    "cross_drops_last_diagonal": ("for (int64_t k = -(n1 - 1); k <= n2 - 1; ++k)",
                                  "for (int64_t k = -(n1 - 1); k < n2 - 1; ++k)"),
    "cross_drops_first_diagonal": ("for (int64_t k = -(n1 - 1); k <= n2 - 1; ++k)",
                                   "for (int64_t k = -(n1 - 2); k <= n2 - 1; ++k)"),
    "cross_one_sided_theiler": ("int64_t gap = i > j ? i - j : j - i;",
                                "int64_t gap = j - i;"),
    "cross_tau_ignored_on_columns": ("- s2[j + (int64_t)k * tau];", "- s2[j + (int64_t)k];"),
    "cross_rr_square_of_rows": ("out->rr = (double)rp / ((double)rows * (double)cols);",
                                "out->rr = (double)rp / ((double)rows * (double)rows);"),
    "cross_column_runs_not_closed": ("      if (prev >= 0) close_run(lv, lw, prev, run);\n    }\n#pragma omp critical",
                                     "    }\n#pragma omp critical"),
}

# Mistakes in the precomputed-matrix code, caught by the matrix pins.
MATRIX_MUTANTS = {
    "matrix_theiler_ignored": ("if (gap < (int64_t)w) return 0;", "if (gap < 0) return 0;"),
    "matrix_drops_last_diagonal": ("for (int64_t k = -(rows - 1); k <= cols - 1; ++k)",
                                   "for (int64_t k = -(rows - 1); k < cols - 1; ++k)"),
    "matrix_diagonal_border_runs_dropped": (
        "    if (prev >= 0) close_run(hd, NULL, prev, run);\n  }\n  uint64_t ones = 0;",
        "  }\n  uint64_t ones = 0;"),
    "matrix_any_nonzero_not_one": ("return R[i * cols + j] != 0;", "return R[i * cols + j] & 2;"),
}


def _run_pins(name, old, new, pins, tmp_path):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    mut = tmp_path / "rqa_oracle.c"
    mut.write_text(src.replace(old, new))
    env = dict(os.environ, RQA_ORACLE_SRC=str(mut))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", pins)],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch mutant {name}:\n{r.stdout[-2000:]}"
    assert "failed" in r.stdout


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    _run_pins(name, old, new, "test_oracle_pins.py", tmp_path)


@pytest.mark.parametrize("name", sorted(CROSS_MUTANTS))
def test_cross_pins_catch_mutant(name, tmp_path):
    old, new = CROSS_MUTANTS[name]
    _run_pins(name, old, new, "test_oracle_cross_pins.py", tmp_path)


@pytest.mark.parametrize("name", sorted(MATRIX_MUTANTS))
def test_matrix_pins_catch_mutant(name, tmp_path):
    old, new = MATRIX_MUTANTS[name]
    _run_pins(name, old, new, "test_oracle_matrix_pins.py", tmp_path)
