"""B300-native recurrence quantification analysis (RQA).

The C ABI (include/rqa.h) of librqa_b300.so computes the time-delay
embedding, the implicit fixed-radius recurrence matrix and the fused
diagonal / vertical / white-vertical line histograms on an sm_103a GPU, with
the measures of the PyRQA paper (Table 3) derived on the host.  This package
is its thin Python binding (``rqa``) and build script (``build``).
"""
from .rqa import (HIST_DIAGONAL, HIST_VERTICAL, HIST_WHITE, NORM_L1, NORM_L2, NORM_MAX,
                  PREC_AUTO, PREC_FP32_RECHECK, PREC_FP64, RQA, Batch, RQAError, Server,
                  Settings, autotune, autotune_clear, autotune_shape, cross_recurrence_plot,
                  load, load_tuning_table, save_tuning_table, tuning_table_loaded,
                  pack_matrix, preload_kernels, probe_alu, recurrence_plot, run_batch,
                  run_batch_release, selftest_bounded_wait, strerror, write_pgm)

__all__ = ["RQA", "Batch", "Server", "Settings", "RQAError", "load", "strerror",
           "recurrence_plot", "cross_recurrence_plot", "pack_matrix", "write_pgm",
           "autotune", "autotune_clear", "autotune_shape", "save_tuning_table",
           "load_tuning_table", "tuning_table_loaded", "run_batch", "run_batch_release",
           "selftest_bounded_wait", "probe_alu", "preload_kernels",
           "NORM_MAX", "NORM_L2", "NORM_L1", "PREC_AUTO", "PREC_FP32_RECHECK", "PREC_FP64",
           "HIST_DIAGONAL", "HIST_VERTICAL", "HIST_WHITE"]
