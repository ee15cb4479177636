"""ctypes binding of librqa_b300.so (include/rqa.h).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels.  There is no CPU fallback: if the native library is
missing this module raises at load time, and on a machine without a B300 the
library's own calls return RQA_ENODEV.

PyTorch is used only to hand device memory and streams to the library
(``RQA.run`` with a CUDA tensor passes its data pointer and the current
stream to ``rqa_run_device``).
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librqa_b300.so")
# Tile shapes tuned on a B300 per (kind, m, norm, precision, ceil(log2 n))
# class by make_tuning_table.py; loaded into the library with it, unless
# RQA_NO_TUNING_TABLE is set.
TUNING_TABLE = os.path.join(_HERE, "tuning_b300.txt")
_tuned_entries = 0

RQA_OK, RQA_EINVAL, RQA_ESHORT, RQA_ENAN, RQA_ENOMEM, RQA_ECUDA = 0, 1, 2, 3, 4, 5
RQA_ETIMEOUT, RQA_PENDING, RQA_ENODEV, RQA_ETOOBIG, RQA_ENOTFOUND = 6, 7, 8, 9, 10
NORM_MAX, NORM_L2, NORM_L1 = 0, 1, 2
PREC_AUTO, PREC_FP32_RECHECK, PREC_FP64 = 0, 1, 2
HIST_DIAGONAL, HIST_VERTICAL, HIST_WHITE = 0, 1, 2


class RQAError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {strerror(status)} ({status})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


@dataclass(frozen=True)
class Settings:
    """The paper's Settings (Sect. 7.2): embedding, norm, radius, Theiler
    window and minimum line lengths, plus the GPU precision mode."""
    m: int
    tau: int
    eps: float
    norm: int = NORM_L2
    theiler: int = 1
    l_min: int = 2
    v_min: int = 2
    w_min: int = 2
    precision: int = PREC_AUTO
    band_override: float = -1.0


class _CSettings(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("tau", ctypes.c_int32), ("eps", ctypes.c_double),
                ("norm", ctypes.c_int32), ("theiler", ctypes.c_int32),
                ("l_min", ctypes.c_int32), ("v_min", ctypes.c_int32),
                ("w_min", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("band_override", ctypes.c_double)]


_MEAS_D = ("rr", "det", "l", "div", "l_entr", "lam", "tt", "v_entr", "w", "w_entr")
_MEAS_I = ("l_max", "v_max", "w_max", "n_vec", "recurrence_points")


class _CMeasures(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in _MEAS_D] + [(k, ctypes.c_int64) for k in _MEAS_I]


class _CStats(ctypes.Structure):
    _fields_ = [("n_vec", ctypes.c_int64), ("pairs", ctypes.c_int64),
                ("rechecks", ctypes.c_int64), ("band", ctypes.c_double),
                ("band_bound", ctypes.c_double), ("precision_used", ctypes.c_int32),
                ("exact", ctypes.c_int32), ("strip_width", ctypes.c_int32),
                ("warps_per_cta", ctypes.c_int32), ("cols_per_lane", ctypes.c_int32),
                ("ctas", ctypes.c_int32), ("kernel_ms", ctypes.c_float),
                ("total_ms", ctypes.c_float), ("h2d_bytes", ctypes.c_int64),
                ("d2h_bytes", ctypes.c_int64), ("launches", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("n_cols", ctypes.c_int64),
                ("band_rows", ctypes.c_int64), ("desc_bytes", ctypes.c_int64),
                ("desc_bytes_all_strips", ctypes.c_int64), ("strip_groups", ctypes.c_int32),
                ("strips_per_group", ctypes.c_int32)]


MEASURE_FIELDS = list(_MEAS_D + _MEAS_I)


def _struct_dtype(cls) -> np.dtype:
    """The numpy dtype with the field names, types and offsets of a ctypes
    structure (so an array of it can be passed where the C ABI wants one)."""
    kinds = {ctypes.c_int32: np.int32, ctypes.c_int64: np.int64, ctypes.c_double: np.float64}
    return np.dtype({"names": [f for f, _ in cls._fields_],
                     "formats": [kinds[t] for _, t in cls._fields_],
                     "offsets": [getattr(cls, f).offset for f, _ in cls._fields_],
                     "itemsize": ctypes.sizeof(cls)})


_SETTINGS_DT = _struct_dtype(_CSettings)
_MEASURES_DT = _struct_dtype(_CMeasures)
_lib = None


def load(path: str = LIB_PATH):
    """Load the native library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with "
                          "`python -m paper_2402_16853_b300.build`")
    lib = ctypes.CDLL(path)
    P, c = ctypes.POINTER, ctypes
    vp = c.c_void_p
    sig = {
        "rqa_create": (c.c_int, [P(_CSettings), P(vp)]),
        "rqa_run": (c.c_int, [vp, P(c.c_double), c.c_int64]),
        "rqa_set_settings": (c.c_int, [vp, P(_CSettings)]),
        "rqa_run_device": (c.c_int, [vp, vp, c.c_int64, vp]),
        "rqa_run_cross": (c.c_int, [vp, P(c.c_double), c.c_int64, P(c.c_double), c.c_int64]),
        "rqa_run_cross_device": (c.c_int, [vp, vp, c.c_int64, vp, c.c_int64, vp]),
        "rqa_run_matrix": (c.c_int, [vp, P(c.c_uint32), c.c_int64, c.c_int64]),
        "rqa_run_matrix_device": (c.c_int, [vp, vp, c.c_int64, c.c_int64, vp]),
        "rqa_measures": (c.c_int, [vp, P(_CMeasures)]),
        "rqa_histogram": (c.c_int, [vp, c.c_int32, P(c.c_uint64), c.c_int64, P(c.c_int64)]),
        "rqa_stats": (c.c_int, [vp, P(_CStats)]),
        "rqa_sample_decisions": (c.c_int, [vp, P(c.c_int64), P(c.c_int64), c.c_int64,
                                           P(c.c_uint8)]),
        "rqa_destroy": (None, [vp]),
        "rqa_strerror": (c.c_char_p, [c.c_int]),
        "rqa_last_error": (c.c_char_p, [vp]),
        "rqa_batch_create": (c.c_int, [P(vp)]),
        "rqa_batch_run": (c.c_int, [vp, P(_CSettings), P(P(c.c_double)), P(c.c_int64),
                                    c.c_int32, P(_CMeasures), P(c.c_int32)]),
        "rqa_batch_histogram": (c.c_int, [vp, c.c_int32, c.c_int32, P(c.c_uint64), c.c_int64,
                                          P(c.c_int64)]),
        "rqa_batch_stats": (c.c_int, [vp, P(_CStats)]),
        "rqa_run_batch": (c.c_int, [P(_CSettings), P(P(c.c_double)), P(c.c_int64), c.c_int32,
                                    P(_CMeasures), vp]),
        "rqa_run_batch_release": (None, []),
        "rqa_batch_destroy": (None, [vp]),
        "rqa_server_create": (c.c_int, [c.c_size_t, c.c_int32, P(vp)]),
        "rqa_submit": (c.c_int, [vp, P(_CSettings), P(c.c_double), c.c_int64, P(c.c_uint64)]),
        "rqa_poll": (c.c_int, [vp, c.c_uint64, P(_CMeasures)]),
        "rqa_wait": (c.c_int, [vp, c.c_uint64, c.c_int64, P(_CMeasures)]),
        "rqa_release": (c.c_int, [vp, c.c_uint64]),
        "rqa_server_counters": (c.c_int, [vp] + [P(c.c_int64)] * 6),
        "rqa_server_destroy": (None, [vp]),
        "rqa_recurrence_plot": (c.c_int, [P(_CSettings), P(c.c_double), c.c_int64, c.c_int64,
                                          c.c_int64, c.c_int64, c.c_int64, P(c.c_uint32)]),
        "rqa_cross_recurrence_plot": (c.c_int, [P(_CSettings), P(c.c_double), c.c_int64,
                                                P(c.c_double), c.c_int64, c.c_int64,
                                                c.c_int64, c.c_int64, c.c_int64,
                                                P(c.c_uint32)]),
        "rqa_plot_last_error": (c.c_char_p, []),
        "rqa_autotune": (c.c_int, [P(_CSettings), P(c.c_double), c.c_int64, c.c_int32,
                                   P(c.c_int32), P(c.c_float)]),
        "rqa_autotune_clear": (None, []),
        "rqa_autotune_shape": (c.c_int, [P(_CSettings), P(c.c_double), c.c_int64, c.c_int32,
                                         P(c.c_int32), P(c.c_int32), P(c.c_int32),
                                         P(c.c_float)]),
        "rqa_autotune_save": (c.c_int, [c.c_char_p]),
        "rqa_autotune_load": (c.c_int, [c.c_char_p, P(c.c_int32)]),
        "rqa_selftest_bounded_wait": (c.c_int, [P(c.c_int32), P(c.c_int64)]),
        "rqa_selftest_ring_timeout": (c.c_int, [vp, P(c.c_double), c.c_int64, c.c_int32,
                                                c.c_int32]),
        "rqa_probe_alu": (c.c_int, [c.c_int32, P(c.c_double)]),
        "rqa_preload_kernels": (c.c_int, [P(c.c_int32)]),
        "rqa_autotune_last_error": (c.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    global _tuned_entries
    if os.path.exists(TUNING_TABLE) and not os.environ.get("RQA_NO_TUNING_TABLE"):
        cnt = ctypes.c_int32()
        if lib.rqa_autotune_load(TUNING_TABLE.encode(), ctypes.byref(cnt)) == 0:
            _tuned_entries = cnt.value
    return lib


def strerror(status: int) -> str:
    return load().rqa_strerror(int(status)).decode()


def _cs(st: Settings) -> _CSettings:
    return _CSettings(int(st.m), int(st.tau), float(st.eps), int(st.norm), int(st.theiler),
                      int(st.l_min), int(st.v_min), int(st.w_min), int(st.precision),
                      float(st.band_override))


def _meas(m: _CMeasures) -> dict:
    return {k: getattr(m, k) for k in MEASURE_FIELDS}


def _f64(series) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(series, dtype=np.float64))


class RQA:
    """One RQA computation (the paper's RQAComputation, Sect. 7.3)."""

    def __init__(self, settings: Settings):
        lib = load()
        self.settings = settings
        self._cs = _cs(settings)
        h = ctypes.c_void_p()
        rc = lib.rqa_create(ctypes.byref(self._cs), ctypes.byref(h))
        if rc:
            raise RQAError(rc, "rqa_create")
        self._h = h
        self.n = None

    def close(self):
        if getattr(self, "_h", None):
            load().rqa_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc, where):
        if rc:
            raise RQAError(rc, where, load().rqa_last_error(self._h).decode())

    def selftest_ring_timeout(self, series, warp: int = 1, from_handover: int = 3) -> int:
        """rqa_selftest_ring_timeout: run `series` through the tile kernel's
        test instantiation with warp `warp` withholding its hand-overs from
        the given one on; returns the status (RQA_ETIMEOUT = 6 expected)."""
        s = _f64(series)
        return int(load().rqa_selftest_ring_timeout(
            self._h, s.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(s), warp,
            from_handover))

    def set_settings(self, settings: Settings) -> None:
        """New analysis parameters for this computation (rqa_set_settings):
        the device buffers and streams stay, so a run of many series with
        different parameters pays no per-series set-up."""
        cs = _cs(settings)
        self._check(load().rqa_set_settings(self._h, ctypes.byref(cs)), "rqa_set_settings")
        self.settings = settings
        self._cs = cs

    def run(self, series, stream=None) -> dict:
        """Run on a series: a host array (copied) or a CUDA torch tensor
        (used in place, ordered on `stream` or torch's current stream).
        Returns the measures."""
        lib = load()
        if hasattr(series, "is_cuda") and series.is_cuda:
            import torch
            t = series.contiguous()
            if t.dtype != torch.float64:
                raise TypeError("device series must be float64")
            if stream is None:
                stream = torch.cuda.current_stream(t.device)
            sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
            rc = lib.rqa_run_device(self._h, ctypes.c_void_p(t.data_ptr()), t.numel(),
                                    ctypes.c_void_p(sp))
            n_in = t.numel()
            self._keep = t  # the library samples from it later
        else:
            s = _f64(series)
            rc = lib.rqa_run(self._h, s.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(s))
            n_in = len(s)
        self._check(rc, "rqa_run")
        self.n = n_in - (self.settings.m - 1) * self.settings.tau
        return self.measures()

    def run_cross(self, x, y, stream=None) -> dict:
        """Cross recurrence of two series (rows: vectors of x, columns:
        vectors of y), both host arrays or both CUDA float64 tensors.
        Returns the measures; histograms / stats / sample then describe the
        n1 x n2 cross matrix."""
        lib = load()
        if hasattr(x, "is_cuda") and x.is_cuda:
            import torch
            tx, ty = x.contiguous(), y.contiguous()
            if tx.dtype != torch.float64 or ty.dtype != torch.float64 or not ty.is_cuda:
                raise TypeError("device series must both be CUDA float64 tensors")
            if stream is None:
                stream = torch.cuda.current_stream(tx.device)
            sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
            rc = lib.rqa_run_cross_device(self._h, ctypes.c_void_p(tx.data_ptr()), tx.numel(),
                                          ctypes.c_void_p(ty.data_ptr()), ty.numel(),
                                          ctypes.c_void_p(sp))
            self._keep = (tx, ty)
        else:
            a, b = _f64(x), _f64(y)
            P = ctypes.POINTER(ctypes.c_double)
            rc = lib.rqa_run_cross(self._h, a.ctypes.data_as(P), len(a), b.ctypes.data_as(P),
                                   len(b))
            self._keep = (a, b)
        self._check(rc, "rqa_run_cross")
        self.n = self.stats()["n_vec"]
        return self.measures()

    def run_matrix(self, matrix, cols: Optional[int] = None, stream=None) -> dict:
        """Lines and measures of a precomputed binary matrix: a 2-D array of
        0/1 (packed here), or packed uint32 words of shape (rows,
        ceil(cols/32)) with `cols` given -- a host array or a CUDA tensor
        (int32 / uint32 words, used in place).  Returns the measures."""
        lib = load()
        if hasattr(matrix, "is_cuda") and matrix.is_cuda:
            import torch
            if cols is None or matrix.dim() != 2 or matrix.element_size() != 4:
                raise TypeError("a device matrix must be packed 32-bit words with cols given")
            t = matrix.contiguous()
            if t.shape[1] != (cols + 31) // 32:
                raise ValueError("words per row must be ceil(cols / 32)")
            if stream is None:
                stream = torch.cuda.current_stream(t.device)
            sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
            rc = lib.rqa_run_matrix_device(self._h, ctypes.c_void_p(t.data_ptr()), t.shape[0],
                                           cols, ctypes.c_void_p(sp))
            self._keep = t
        else:
            words = pack_matrix(matrix) if cols is None else np.ascontiguousarray(matrix,
                                                                                    np.uint32)
            if cols is None:
                cols = np.asarray(matrix).shape[1]
            if words.ndim != 2 or words.shape[1] != (cols + 31) // 32:
                raise ValueError("words per row must be ceil(cols / 32)")
            rc = lib.rqa_run_matrix(self._h, words.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                    words.shape[0], cols)
            self._keep = words
        self._check(rc, "rqa_run_matrix")
        self.n = self.stats()["n_vec"]
        return self.measures()

    def measures(self) -> dict:
        m = _CMeasures()
        self._check(load().rqa_measures(self._h, ctypes.byref(m)), "rqa_measures")
        return _meas(m)

    def histogram(self, kind: int) -> np.ndarray:
        ln = ctypes.c_int64()
        load().rqa_histogram(self._h, kind, None, 0, ctypes.byref(ln))
        out = np.zeros(ln.value, dtype=np.uint64)
        self._check(load().rqa_histogram(self._h, kind,
                                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                         len(out), ctypes.byref(ln)), "rqa_histogram")
        return out

    def histograms(self):
        return tuple(self.histogram(k) for k in (HIST_DIAGONAL, HIST_VERTICAL, HIST_WHITE))

    def stats(self) -> dict:
        s = _CStats()
        self._check(load().rqa_stats(self._h, ctypes.byref(s)), "rqa_stats")
        return {k: getattr(s, k) for k, _ in _CStats._fields_}

    def sample(self, i, j) -> np.ndarray:
        i = np.ascontiguousarray(i, dtype=np.int64)
        j = np.ascontiguousarray(j, dtype=np.int64)
        out = np.zeros(len(i), dtype=np.uint8)
        P = ctypes.POINTER
        self._check(load().rqa_sample_decisions(
            self._h, i.ctypes.data_as(P(ctypes.c_int64)), j.ctypes.data_as(P(ctypes.c_int64)),
            len(i), out.ctypes.data_as(P(ctypes.c_uint8))), "rqa_sample_decisions")
        return out


class Batch:
    """Many series in one submission (one persistent launch per (m, norm)
    class, captured in a CUDA graph and replayed for unchanged shapes)."""

    def __init__(self):
        lib = load()
        h = ctypes.c_void_p()
        rc = lib.rqa_batch_create(ctypes.byref(h))
        if rc:
            raise RQAError(rc, "rqa_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().rqa_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, settings: Sequence[Settings], series: Sequence[np.ndarray]):
        """Returns (list of measure dicts or None, list of statuses, rc)."""
        k = len(series)
        if len(settings) != k:
            raise ValueError("one Settings per series")
        arrs = [_f64(s) for s in series]
        # numpy arrays in the C layouts: one vectorised fill per field
        # instead of a ctypes object per series
        cs = np.zeros(k, _SETTINGS_DT)
        for f in _SETTINGS_DT.names:
            cs[f] = [getattr(s, f) for s in settings]
        ptrs = np.fromiter((a.__array_interface__["data"][0] for a in arrs), np.uintp, k)
        lens = np.fromiter((a.shape[0] for a in arrs), np.int64, k)
        out = np.zeros(k, _MEASURES_DT)
        st = np.zeros(k, np.int32)
        P = ctypes.POINTER
        rc = load().rqa_batch_run(self._h, cs.ctypes.data_as(P(_CSettings)),
                                  ptrs.ctypes.data_as(P(P(ctypes.c_double))),
                                  lens.ctypes.data_as(P(ctypes.c_int64)), k,
                                  out.ctypes.data_as(P(_CMeasures)),
                                  st.ctypes.data_as(P(ctypes.c_int32)))
        self._arrs = arrs
        sts = st.tolist()
        res = [dict(zip(MEASURE_FIELDS, row)) if q == 0 else None
               for row, q in zip(out.tolist(), sts)]
        return res, sts, int(rc)

    def histogram(self, q: int, kind: int) -> np.ndarray:
        ln = ctypes.c_int64()
        load().rqa_batch_histogram(self._h, q, kind, None, 0, ctypes.byref(ln))
        out = np.zeros(ln.value, dtype=np.uint64)
        rc = load().rqa_batch_histogram(self._h, q, kind,
                                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                        len(out), ctypes.byref(ln))
        if rc:
            raise RQAError(rc, "rqa_batch_histogram")
        return out

    def stats(self) -> dict:
        s = _CStats()
        load().rqa_batch_stats(self._h, ctypes.byref(s))
        return {k: getattr(s, k) for k, _ in _CStats._fields_}


def run_batch(settings: Sequence[Settings], series: Sequence[np.ndarray], stream=None):
    """rqa_run_batch: one call over many host series, device work ordered on
    `stream` (a torch.cuda.Stream, a raw cudaStream_t as int, or None).
    Returns (list of measure dicts, None for a failed series; rc)."""
    k = len(series)
    if len(settings) != k:
        raise ValueError("one Settings per series")
    arrs = [_f64(s) for s in series]
    cs = np.zeros(k, _SETTINGS_DT)
    for f in _SETTINGS_DT.names:
        cs[f] = [getattr(s, f) for s in settings]
    ptrs = np.fromiter((a.__array_interface__["data"][0] for a in arrs), np.uintp, k)
    lens = np.fromiter((a.shape[0] for a in arrs), np.int64, k)
    out = np.zeros(k, _MEASURES_DT)
    P = ctypes.POINTER
    raw = getattr(stream, "cuda_stream", stream)
    rc = load().rqa_run_batch(cs.ctypes.data_as(P(_CSettings)),
                              ptrs.ctypes.data_as(P(P(ctypes.c_double))),
                              lens.ctypes.data_as(P(ctypes.c_int64)), k,
                              out.ctypes.data_as(P(_CMeasures)),
                              ctypes.c_void_p(raw) if raw else None)
    res = [dict(zip(MEASURE_FIELDS, row)) for row in out.tolist()]
    return res, int(rc)


def run_batch_release() -> None:
    load().rqa_run_batch_release()


class Server:
    """Continuous-batching server (rqa_server_*)."""

    def __init__(self, mem_budget_bytes: int, max_slots: int = 4096):
        lib = load()
        h = ctypes.c_void_p()
        rc = lib.rqa_server_create(int(mem_budget_bytes), int(max_slots), ctypes.byref(h))
        if rc:
            raise RQAError(rc, "rqa_server_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().rqa_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, settings: Settings, series) -> int:
        s = _f64(series)
        cs = _cs(settings)
        t = ctypes.c_uint64()
        rc = load().rqa_submit(self._h, ctypes.byref(cs),
                               s.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(s),
                               ctypes.byref(t))
        if rc:
            raise RQAError(rc, "rqa_submit")
        return t.value

    def poll(self, ticket: int):
        m = _CMeasures()
        rc = load().rqa_poll(self._h, ticket, ctypes.byref(m))
        return rc, (_meas(m) if rc == RQA_OK else None)

    def wait(self, ticket: int, timeout_ms: int = 60_000):
        m = _CMeasures()
        rc = load().rqa_wait(self._h, ticket, int(timeout_ms), ctypes.byref(m))
        return rc, (_meas(m) if rc == RQA_OK else None)

    def release(self, ticket: int) -> int:
        return load().rqa_release(self._h, ticket)

    def counters(self) -> dict:
        vals = [ctypes.c_int64() for _ in range(6)]
        load().rqa_server_counters(self._h, *[ctypes.byref(v) for v in vals])
        keys = ("admitted", "completed", "queued", "in_flight", "bytes_in_use", "epochs")
        return {k: v.value for k, v in zip(keys, vals)}


def recurrence_plot(settings: Settings, series, i0: int = 0, j0: int = 0,
                    rows: Optional[int] = None, cols: Optional[int] = None,
                    packed: bool = False):
    """A window of the recurrence matrix (the paper's RecurrencePlotComputation)
    computed on the GPU.  Returns a (rows, cols) uint8 array of 0/1, or with
    packed=True the raw (rows, ceil(cols/32)) uint32 words (bit b of word w is
    column 32 w + b)."""
    s = _f64(series)
    n = len(s) - (settings.m - 1) * settings.tau
    rows = n - i0 if rows is None else rows
    cols = n - j0 if cols is None else cols
    wpr = (cols + 31) // 32
    out = np.zeros((max(rows, 0), wpr), dtype=np.uint32)
    cs = _cs(settings)
    rc = load().rqa_recurrence_plot(ctypes.byref(cs), s.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    len(s), i0, j0, rows, cols,
                                    out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    if rc:
        raise RQAError(rc, "rqa_recurrence_plot", load().rqa_plot_last_error().decode())
    if packed:
        return out
    bits = np.unpackbits(out.view(np.uint8), axis=1, bitorder="little")
    return bits[:, :cols]


def cross_recurrence_plot(settings: Settings, x, y, i0: int = 0, j0: int = 0,
                          rows: Optional[int] = None, cols: Optional[int] = None,
                          packed: bool = False):
    """A window of the cross-recurrence matrix of x (rows) and y (columns),
    in the layout of recurrence_plot()."""
    a, b = _f64(x), _f64(y)
    span = (settings.m - 1) * settings.tau
    rows = len(a) - span - i0 if rows is None else rows
    cols = len(b) - span - j0 if cols is None else cols
    wpr = (cols + 31) // 32
    out = np.zeros((max(rows, 0), wpr), dtype=np.uint32)
    cs = _cs(settings)
    P = ctypes.POINTER(ctypes.c_double)
    rc = load().rqa_cross_recurrence_plot(ctypes.byref(cs), a.ctypes.data_as(P), len(a),
                                          b.ctypes.data_as(P), len(b), i0, j0, rows, cols,
                                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    if rc:
        raise RQAError(rc, "rqa_cross_recurrence_plot", load().rqa_plot_last_error().decode())
    if packed:
        return out
    bits = np.unpackbits(out.view(np.uint8), axis=1, bitorder="little")
    return bits[:, :cols]


def autotune(settings: Settings, n_points: Optional[int] = None, series=None,
             cross: bool = False) -> dict:
    """Time every CTA-strip width on `series` (or on a built-in AR(1) series
    of n_points values) and record the fastest for the settings' class; later
    runs of the class use it.  Returns {"warps": best, "ms": {width: ms}}."""
    P = ctypes.POINTER(ctypes.c_double)
    if series is not None:
        s = _f64(series)
        ptr, n_points = s.ctypes.data_as(P), len(s)
    else:
        ptr = None
    cs = _cs(settings)
    best = ctypes.c_int32()
    ms = (ctypes.c_float * 4)()
    rc = load().rqa_autotune(ctypes.byref(cs), ptr, int(n_points), 1 if cross else 0,
                             ctypes.byref(best), ms)
    if rc:
        raise RQAError(rc, "rqa_autotune", load().rqa_autotune_last_error().decode())
    return {"warps": best.value, "ms": {w: ms[q] for q, w in enumerate((1, 2, 4, 8))}}


def autotune_shape(settings: Settings, n_points: Optional[int] = None, series=None,
                   cross: bool = False) -> dict:
    """The full tile-shape search (rqa_autotune_shape): strip width, columns
    per lane and row-band height; records the winner for the class.
    Returns {"warps", "cols", "band_scale", "ms"}."""
    P = ctypes.POINTER(ctypes.c_double)
    if series is not None:
        s = _f64(series)
        ptr, n_points = s.ctypes.data_as(P), len(s)
    else:
        ptr = None
    cs = _cs(settings)
    w, c, b = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    ms = ctypes.c_float()
    rc = load().rqa_autotune_shape(ctypes.byref(cs), ptr, int(n_points), 1 if cross else 0,
                                   ctypes.byref(w), ctypes.byref(c), ctypes.byref(b),
                                   ctypes.byref(ms))
    if rc:
        raise RQAError(rc, "rqa_autotune_shape", load().rqa_autotune_last_error().decode())
    return {"warps": w.value, "cols": c.value, "band_scale": b.value, "ms": ms.value}


def save_tuning_table(path: str) -> None:
    rc = load().rqa_autotune_save(path.encode())
    if rc:
        raise RQAError(rc, "rqa_autotune_save", load().rqa_autotune_last_error().decode())


def load_tuning_table(path: str) -> int:
    cnt = ctypes.c_int32()
    rc = load().rqa_autotune_load(path.encode(), ctypes.byref(cnt))
    if rc:
        raise RQAError(rc, "rqa_autotune_load", load().rqa_autotune_last_error().decode())
    return cnt.value


def tuning_table_loaded() -> bool:
    """True if the committed B300 tuning table was loaded with the library."""
    load()
    return _tuned_entries > 0


def selftest_bounded_wait():
    """Run the bounded-wait self-test: returns (status the waiting warp
    reported -- 6, RQA_ETIMEOUT, when the mechanism works -- and the SM
    cycles it waited).  Raises RQAError if the wait did not give up."""
    st = ctypes.c_int32()
    cyc = ctypes.c_int64()
    rc = load().rqa_selftest_bounded_wait(ctypes.byref(st), ctypes.byref(cyc))
    if rc:
        raise RQAError(rc, "rqa_selftest_bounded_wait")
    return st.value, cyc.value


ALU_PROBES = ("fma.f32", "fma.f32x2", "add.f32", "sub.f32x2", "max.f32")


def probe_alu() -> dict:
    """Measured FP32 operations/s of each probe kind (one per lane, two for
    the packed f32x2 forms) on the current device."""
    res = {}
    for k, name in enumerate(ALU_PROBES):
        v = ctypes.c_double()
        rc = load().rqa_probe_alu(k, ctypes.byref(v))
        if rc:
            raise RQAError(rc, "rqa_probe_alu")
        res[name] = v.value
    return res


def preload_kernels() -> int:
    """Load every kernel of the library into the current device's context
    now (once per process) instead of at first launch; returns how many.
    Servers call it at creation; a latency-sensitive caller can too."""
    n = ctypes.c_int32()
    rc = load().rqa_preload_kernels(ctypes.byref(n))
    if rc:
        raise RQAError(rc, "rqa_preload_kernels")
    return int(n.value)


def autotune_clear() -> None:
    """Forget every width the autotuner recorded."""
    load().rqa_autotune_clear()


def pack_matrix(matrix) -> np.ndarray:
    """Pack a 2-D 0/1 array into the library's bit layout: (rows,
    ceil(cols/32)) uint32 words, bit b of word w = column 32 w + b."""
    a = np.asarray(matrix) != 0
    if a.ndim != 2:
        raise ValueError("matrix must be two-dimensional")
    rows, cols = a.shape
    wpr = (cols + 31) // 32
    padded = np.zeros((rows, wpr * 32), dtype=bool)
    padded[:, :cols] = a
    b = np.packbits(padded, axis=1, bitorder="little")
    return np.ascontiguousarray(b).view(np.uint32).reshape(rows, wpr)


def write_pgm(path: str, plot) -> None:
    """Write a 0/1 recurrence plot as a binary PGM image (recurrences black,
    row 0 at the top), the headless form of the paper's plot image."""
    img = np.where(np.asarray(plot, dtype=bool), 0, 255).astype(np.uint8)
    with open(path, "wb") as f:
        f.write(b"P5\n%d %d\n255\n" % (img.shape[1], img.shape[0]))
        f.write(img.tobytes())
