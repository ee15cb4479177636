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
