"""FP64 CPU oracle for the RQA hot path -- TEST INFRASTRUCTURE ONLY.

The arithmetic lives in ``rqa_oracle.c`` (plain C, FP64, built with
``-ffp-contract=off``); this module compiles it with gcc and marshals numpy
arrays through ctypes.  It shares no code with the CUDA library under
``paper_2402_16853_b300/`` and must never be imported by it: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.

What it computes (PyRQA paper, Sect. 2 and Sect. 7.2; measures as in
Table 3, defined after Marwan et al. 2007): the full n x n recurrence matrix
of a time-delay embedded series under the L1 / L2 / L-infinity norm with a
fixed radius and a Theiler window, the histograms of diagonal, vertical and
white vertical line lengths over that full matrix, and the measures derived
from them; the same for the cross-recurrence matrix of two series (Sect. 3.3)
and for a precomputed binary matrix (Sect. 9).  Readings of points the paper
leaves open are listed at the top of ``rqa_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
# RQA_ORACLE_SRC lets the mutant tests build a copy of the source with a
# planted mistake; by default the committed source is used.
_SRC = os.environ.get("RQA_ORACLE_SRC") or os.path.join(_HERE, "rqa_oracle.c")
_LIB = (os.path.join(_BUILD, "liboracle.so") if "RQA_ORACLE_SRC" not in os.environ
        else os.path.join(os.path.dirname(os.path.abspath(_SRC)), "liboracle_variant.so"))

NORM_MAX, NORM_L2, NORM_L1 = 0, 1, 2
NORMS = {"max": NORM_MAX, "linf": NORM_MAX, "l2": NORM_L2, "euclidean": NORM_L2,
         "l1": NORM_L1, "taxicab": NORM_L1}


@dataclass(frozen=True)
class Settings:
    """Analysis parameters (the paper's ``Settings``, Sect. 7.2)."""
    m: int
    tau: int
    eps: float
    norm: int = NORM_L2
    theiler: int = 1
    l_min: int = 2
    v_min: int = 2
    w_min: int = 2


class _CSettings(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("tau", ctypes.c_int32),
                ("eps", ctypes.c_double), ("norm", ctypes.c_int32),
                ("theiler", ctypes.c_int32), ("l_min", ctypes.c_int32),
                ("v_min", ctypes.c_int32), ("w_min", ctypes.c_int32)]


class _CMeasures(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("rr", "det", "l", "div", "l_entr", "lam", "tt", "v_entr", "w",
                 "w_entr")] + \
               [(k, ctypes.c_int64) for k in
                ("l_max", "v_max", "w_max", "n_vec", "recurrence_points")]


MEASURE_FIELDS = [f for f, _ in _CMeasures._fields_]


def _host_id() -> str:
    """CPU model and feature flags of this host: -march=native code built on
    one CPU may not run on another, so the library is rebuilt when they
    change (the repository is copied between machines with its build
    folder)."""
    model = flags = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if not model and line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                elif not flags and line.startswith("flags"):
                    flags = line.split(":", 1)[1].strip()
                if model and flags:
                    break
    except OSError:
        pass
    import hashlib
    return hashlib.sha256((model + "|" + flags).encode()).hexdigest()


def build(force: bool = False) -> str:
    """Compile rqa_oracle.c into a shared library (gcc -O3 -march=native,
    OpenMP, no FMA contraction, no fast-math: every FP64 operation is the
    IEEE one the source writes, in the source's order)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stamp = _LIB + ".host"
    host = _host_id()
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)
            and os.path.exists(stamp) and open(stamp).read() == host):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O3", "-march=native", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-Wall", "-Wextra", _SRC,
           "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    with open(stamp + f".{os.getpid()}.tmp", "w") as f:
        f.write(host)
    os.replace(stamp + f".{os.getpid()}.tmp", stamp)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        lib.oracle_nvec.restype = ctypes.c_int64
        lib.oracle_nvec.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32]
        lib.oracle_distance.restype = ctypes.c_double
        lib.oracle_distance.argtypes = [P(ctypes.c_double), ctypes.c_int64,
                                        ctypes.c_int64, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_int32]
        lib.oracle_matrix.restype = ctypes.c_uint64
        lib.oracle_matrix.argtypes = [P(ctypes.c_double), ctypes.c_int64,
                                      P(_CSettings), P(ctypes.c_uint8)]
        lib.oracle_histograms_from_matrix.restype = None
        lib.oracle_histograms_from_matrix.argtypes = [
            P(ctypes.c_uint8), ctypes.c_int64, P(ctypes.c_uint64),
            P(ctypes.c_uint64), P(ctypes.c_uint64)]
        lib.oracle_histograms_streaming.restype = ctypes.c_uint64
        lib.oracle_histograms_streaming.argtypes = [
            P(ctypes.c_double), ctypes.c_int64, P(_CSettings), ctypes.c_int32,
            ctypes.c_int64, P(ctypes.c_uint64), P(ctypes.c_uint64),
            P(ctypes.c_uint64), P(ctypes.c_uint64)]
        lib.oracle_cross_distance.restype = ctypes.c_double
        lib.oracle_cross_distance.argtypes = [P(ctypes.c_double), P(ctypes.c_double),
                                              ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                              ctypes.c_int32, ctypes.c_int32]
        lib.oracle_cross_histograms.restype = ctypes.c_uint64
        lib.oracle_cross_histograms.argtypes = [
            P(ctypes.c_double), ctypes.c_int64, P(ctypes.c_double), ctypes.c_int64,
            P(_CSettings), ctypes.c_int32, P(ctypes.c_uint64), P(ctypes.c_uint64),
            P(ctypes.c_uint64)]
        lib.oracle_measures_rect.restype = None
        lib.oracle_measures_rect.argtypes = [P(ctypes.c_uint64), P(ctypes.c_uint64),
                                             P(ctypes.c_uint64), ctypes.c_int64,
                                             ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
                                             P(_CSettings), P(_CMeasures)]
        lib.oracle_histograms_from_rect.restype = ctypes.c_uint64
        lib.oracle_histograms_from_rect.argtypes = [
            P(ctypes.c_uint8), ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
            P(ctypes.c_uint64), P(ctypes.c_uint64), P(ctypes.c_uint64)]
        lib.oracle_measures.restype = None
        lib.oracle_measures.argtypes = [P(ctypes.c_uint64), P(ctypes.c_uint64),
                                        P(ctypes.c_uint64), ctypes.c_int64,
                                        ctypes.c_uint64, P(_CSettings),
                                        P(_CMeasures)]
        _lib = lib
    return _lib


def _cs(st: Settings) -> _CSettings:
    return _CSettings(int(st.m), int(st.tau), float(st.eps), int(st.norm),
                      int(st.theiler), int(st.l_min), int(st.v_min),
                      int(st.w_min))


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _uptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _series(series) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(series, dtype=np.float64))


def nvec(N: int, m: int, tau: int) -> int:
    return int(_load().oracle_nvec(N, m, tau))


def distance(series, i: int, j: int, m: int, tau: int, norm: int) -> float:
    s = _series(series)
    return float(_load().oracle_distance(_dptr(s), i, j, m, tau, norm))


def matrix(series, st: Settings):
    """Full n x n recurrence matrix (uint8) and its number of recurrence points."""
    s = _series(series)
    n = nvec(len(s), st.m, st.tau)
    R = np.zeros((n, n), dtype=np.uint8)
    cs = _cs(st)
    rp = _load().oracle_matrix(_dptr(s), len(s), ctypes.byref(cs),
                               R.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return R, int(rp)


def histograms_from_matrix(R: np.ndarray):
    R = np.ascontiguousarray(R, dtype=np.uint8)
    n = R.shape[0]
    hd, hv, hw = (np.zeros(n + 1, np.uint64) for _ in range(3))
    _load().oracle_histograms_from_matrix(
        R.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), n, _uptr(hd),
        _uptr(hv), _uptr(hw))
    return hd, hv, hw


def histograms_streaming(series, st: Settings, threads: int = 0,
                         stride: int = 1):
    """Histograms with cells computed on the fly; returns (hd, hv, hw, rp,
    cells_visited).  stride > 1 visits every stride-th diagonal and column
    only (a bounded sample for timing; the histograms are then partial)."""
    s = _series(series)
    n = nvec(len(s), st.m, st.tau)
    hd, hv, hw = (np.zeros(n + 1, np.uint64) for _ in range(3))
    rp = ctypes.c_uint64(0)
    cs = _cs(st)
    visited = _load().oracle_histograms_streaming(
        _dptr(s), len(s), ctypes.byref(cs), int(threads), int(stride),
        _uptr(hd), _uptr(hv), _uptr(hw), ctypes.byref(rp))
    return hd, hv, hw, int(rp.value), int(visited)


def measures(hd, hv, hw, n: int, rp: int, st: Settings) -> dict:
    hd, hv, hw = (np.ascontiguousarray(h, dtype=np.uint64) for h in (hd, hv, hw))
    out = _CMeasures()
    cs = _cs(st)
    _load().oracle_measures(_uptr(hd), _uptr(hv), _uptr(hw), n, rp,
                            ctypes.byref(cs), ctypes.byref(out))
    return {f: getattr(out, f) for f in MEASURE_FIELDS}


MATERIALISE_MAX_N = 4096


def rqa(series, st: Settings, mode: str = "auto", threads: int = 0):
    """Complete oracle result: dict with hd, hv, hw (uint64 arrays of length
    n + 1, index = line length), rp, n and the measures."""
    s = _series(series)
    n = nvec(len(s), st.m, st.tau)
    if mode == "auto":
        mode = "matrix" if n <= MATERIALISE_MAX_N else "streaming"
    if mode == "matrix":
        R, rp = matrix(s, st)
        hd, hv, hw = histograms_from_matrix(R)
    elif mode == "streaming":
        hd, hv, hw, rp, _ = histograms_streaming(s, st, threads=threads)
    else:
        raise ValueError(mode)
    return {"hd": hd, "hv": hv, "hw": hw, "rp": rp, "n": n,
            "measures": measures(hd, hv, hw, n, rp, st)}


def cross_distance(s1, s2, i: int, j: int, m: int, tau: int, norm: int) -> float:
    a, b = _series(s1), _series(s2)
    return float(_load().oracle_cross_distance(_dptr(a), _dptr(b), i, j, m, tau, norm))


def cross_rqa(series1, series2, st: Settings, threads: int = 0):
    """Cross recurrence: rows are the vectors of series1, columns those of
    series2.  Returns the same dict as rqa() (n = rows, plus cols)."""
    a, b = _series(series1), _series(series2)
    n1 = nvec(len(a), st.m, st.tau)
    n2 = nvec(len(b), st.m, st.tau)
    L = max(n1, n2, 0)
    hd, hv, hw = (np.zeros(L + 1, np.uint64) for _ in range(3))
    cs = _cs(st)
    rp = _load().oracle_cross_histograms(_dptr(a), len(a), _dptr(b), len(b), ctypes.byref(cs),
                                         int(threads), _uptr(hd), _uptr(hv), _uptr(hw))
    out = _CMeasures()
    _load().oracle_measures_rect(_uptr(hd), _uptr(hv), _uptr(hw), L, n1, n2, int(rp),
                                 ctypes.byref(cs), ctypes.byref(out))
    return {"hd": hd, "hv": hv, "hw": hw, "rp": int(rp), "n": n1, "cols": n2,
            "measures": {f: getattr(out, f) for f in MEASURE_FIELDS}}


def matrix_rqa(R, st: Settings):
    """Lines and measures of a precomputed rows x cols 0/1 matrix R (cells
    with |i - j| < st.theiler count as 0).  Same dict as cross_rqa()."""
    R = np.ascontiguousarray(np.asarray(R) != 0, dtype=np.uint8)
    if R.ndim != 2:
        raise ValueError("R must be two-dimensional")
    rows, cols = R.shape
    L = max(rows, cols, 0)
    hd, hv, hw = (np.zeros(L + 1, np.uint64) for _ in range(3))
    rp = _load().oracle_histograms_from_rect(R.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                             rows, cols, int(st.theiler), _uptr(hd), _uptr(hv),
                                             _uptr(hw))
    out = _CMeasures()
    cs = _cs(st)
    _load().oracle_measures_rect(_uptr(hd), _uptr(hv), _uptr(hw), L, rows, cols, int(rp),
                                 ctypes.byref(cs), ctypes.byref(out))
    return {"hd": hd, "hv": hv, "hw": hw, "rp": int(rp), "n": rows, "cols": cols,
            "measures": {f: getattr(out, f) for f in MEASURE_FIELDS}}
