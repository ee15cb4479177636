"""C-ABI checks that need no GPU: the library builds, loads, exports every
function include/rqa.h declares, and reports a missing device as an error
code (no CPU fallback)."""
import os
import re

import pytest

import paper_2402_16853_b300 as rqa_pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rqa.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|const char\*)\s+(rqa_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_paper_api():
    names = declared_functions()
    for must in ("rqa_create", "rqa_run", "rqa_run_device", "rqa_measures", "rqa_histogram",
                 "rqa_destroy", "rqa_batch_run", "rqa_server_create", "rqa_submit", "rqa_poll"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = rqa_pkg.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_run_batch_has_the_boundary_signature():
    """rqa_run_batch(const rqa_settings*, const double* const*, const int64_t*,
    int32_t count, rqa_measures_t* out, void* stream): the batched call with a
    caller's stream, declared once in the header and exported."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    m = re.search(r"int\s+rqa_run_batch\s*\(([^)]*)\)", src)
    assert m, "rqa_run_batch not declared"
    args = [re.sub(r"\s+", " ", a).strip() for a in m.group(1).split(",")]
    assert args == ["const rqa_settings* settings", "const double* const* series",
                    "const int64_t* lens", "int32_t count", "rqa_measures_t* out",
                    "void* stream"], args
    lib = rqa_pkg.load()
    assert hasattr(lib, "rqa_run_batch") and hasattr(lib, "rqa_run_batch_release")


def test_strerror_names_every_code():
    for code in range(11):
        assert rqa_pkg.strerror(code) != "unknown status"
    assert rqa_pkg.strerror(99) == "unknown status"


def test_no_device_is_an_error_not_a_fallback():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(rqa_pkg.RQAError) as ei:
        rqa_pkg.RQA(rqa_pkg.Settings(m=2, tau=1, eps=0.5))
    assert ei.value.status == 8  # RQA_ENODEV


def test_invalid_settings_rejected_before_device_lookup():
    bad = [dict(m=0), dict(tau=0), dict(eps=0.0), dict(eps=float("nan")), dict(norm=3),
           dict(theiler=-1), dict(l_min=0), dict(precision=5)]
    for kw in bad:
        base = dict(m=2, tau=1, eps=0.5)
        base.update(kw)
        with pytest.raises(rqa_pkg.RQAError) as ei:
            rqa_pkg.RQA(rqa_pkg.Settings(**base))
        assert ei.value.status == 1, kw
    with pytest.raises(rqa_pkg.RQAError) as ei:
        rqa_pkg.RQA(rqa_pkg.Settings(m=11, tau=1, eps=0.5))
    assert ei.value.status == 9  # RQA_ETOOBIG


def test_batch_marshalling_dtypes_match_the_c_structs():
    """Batch.run passes numpy arrays where the ABI wants arrays of
    rqa_settings and rqa_measures_t: their dtypes must have the structs'
    field names, offsets, sizes and types."""
    import ctypes

    import numpy as np

    from paper_2402_16853_b300 import rqa as R
    kinds = {ctypes.c_int32: np.int32, ctypes.c_int64: np.int64, ctypes.c_double: np.float64}
    for cls, dt in ((R._CSettings, R._SETTINGS_DT), (R._CMeasures, R._MEASURES_DT)):
        assert dt.itemsize == ctypes.sizeof(cls)
        assert list(dt.names) == [f for f, _ in cls._fields_]
        for f, t in cls._fields_:
            assert dt.fields[f][1] == getattr(cls, f).offset
            assert dt.fields[f][0] == np.dtype(kinds[t])
    assert list(R._MEASURES_DT.names) == R.MEASURE_FIELDS
    # a round trip through the C layout
    a = np.zeros(2, R._SETTINGS_DT)
    a["m"] = [3, 7]
    a["eps"] = [0.5, 0.25]
    c = (R._CSettings * 2).from_buffer_copy(a.tobytes())
    assert (c[0].m, c[1].m, c[0].eps, c[1].eps) == (3, 7, 0.5, 0.25)


def test_tuning_table_files(tmp_path):
    """The tuning table's text form (no GPU needed): a well-formed file is
    read with its entry count, a malformed one is refused and records
    nothing, and the committed B300 table, if present, parses."""
    import ctypes
    lib = rqa_pkg.load()
    good = tmp_path / "t.txt"
    good.write_text("# kind m norm f64 log2n warps cols band_scale\n"
                    "0 3 1 0 14 2 2 0\n0 5 0 0 17 8 4 -1\n")
    cnt = ctypes.c_int32()
    assert lib.rqa_autotune_load(str(good).encode(), ctypes.byref(cnt)) == 0
    assert cnt.value == 2
    for bad in ("0 3 1 0 14 3 4 0\n", "0 3 1 1 14 2 2 0\n", "0 3 1 0 14 2 4 2\n", "x\n"):
        p = tmp_path / "bad.txt"
        p.write_text(bad)
        assert lib.rqa_autotune_load(str(p).encode(), None) == 1, bad
    lib.rqa_autotune_clear()
    from paper_2402_16853_b300 import rqa as R
    if os.path.exists(R.TUNING_TABLE):
        assert lib.rqa_autotune_load(R.TUNING_TABLE.encode(), ctypes.byref(cnt)) == 0
        assert cnt.value > 0
        lib.rqa_autotune_clear()


def test_plot_window_limits_checked_on_the_host():
    """Windows whose byte size or origin would overflow are refused before any
    device work (so this runs without a GPU): rows x words above 4 GiB, a
    row count whose product with the words per row wraps, an origin past 2^40."""
    import ctypes
    import numpy as np
    from paper_2402_16853_b300.rqa import _cs
    lib = rqa_pkg.load()
    cs = _cs(rqa_pkg.Settings(m=2, tau=1, eps=0.5))
    s = np.linspace(0.0, 1.0, 100)
    ps = s.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    out = (ctypes.c_uint32 * 4)()
    cases = [((0, 0, 1 << 20, 1 << 20), 9),          # 128 GiB of plot
             ((0, 0, 1 << 62, 32), 9),                # 4 * rows * 1 word wraps to 0
             ((0, 0, 1 << 40, (1 << 63) - 1), 9),     # cols near INT64_MAX
             ((1 << 41, 0, 4, 4), 1), ((0, 1 << 50, 4, 4), 1),
             ((-1, 0, 4, 4), 1)]
    for (i0, j0, rows, cols), want in cases:
        rc = lib.rqa_recurrence_plot(ctypes.byref(cs), ps, len(s), i0, j0, rows, cols, out)
        assert rc == want, (i0, j0, rows, cols, rc)
