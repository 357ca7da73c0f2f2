"""The C ABI library builds, loads and exports every entry point include/sg.h
declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(sg_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1507_04769_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("sg_build_grid", "sg_solve_bvps", "sg_build_surpluses", "sg_eval_feedback"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_and_reports_errors_without_gpu(lib):
    from paper_1507_04769_gb300 import sg
    # argument validation happens before any CUDA call
    h = ctypes.c_void_p()
    lo = (ctypes.c_double * 2)(0.0, 0.0)
    hi = (ctypes.c_double * 2)(1.0, -1.0)
    rc = sg.LIB.sg_build_grid(2, 1, ctypes.cast(lo, ctypes.c_void_p), ctypes.cast(hi, ctypes.c_void_p),
                              ctypes.byref(h))
    assert rc == sg.SG_EINVAL
    assert b"lo < hi" in sg.LIB.sg_last_error()
    assert sg.LIB.sg_build_grid(9, 1, ctypes.cast(lo, ctypes.c_void_p), ctypes.cast(lo, ctypes.c_void_p),
                                ctypes.byref(h)) == sg.SG_EUNSUPPORTED


def test_workspace_size_grows_with_problem(lib):
    from paper_1507_04769_gb300 import sg
    a = sg.workspace_bytes(10, 64, sg.PREC_FP64)
    b = sg.workspace_bytes(20, 64, sg.PREC_FP64)
    c = sg.workspace_bytes(10, 64, sg.PREC_MIXED)
    # the two FP32-direction forms share the layout; an unknown precision sizes nothing
    assert sg.workspace_bytes(10, 64, sg.PREC_MIXED_PAIR) == c
    assert sg.workspace_bytes(10, 64, 7) == 0
    assert 0 < a < b and c < a
    assert sg.workspace_bytes(10, 0, 0) == 0
