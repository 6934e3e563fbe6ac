"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/tsf.h declares (no compute call: there may be no GPU)."""
import ctypes
import os
import re

import pytest

import paper_2407_12399_gb300 as tsf
from paper_2407_12399_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(tsf_[a-z0-9_]+)\s*\(", txt))
    return names


def test_header_declares_the_boundary():
    d = declared()
    for name in ("tsf_create_field", "tsf_set_signal_pairs", "tsf_compute_diagram", "tsf_solver_step",
                 "tsf_simplify"):
        assert name in d


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    for name in declared():
        assert hasattr(L, name), name


def test_binding_names_match_the_header():
    assert set(tsf.EXPORTS) <= declared()
    for name in tsf.EXPORTS:
        assert callable(getattr(tsf, name))


def test_status_strings_and_argument_checks_need_no_gpu(libpath):
    assert tsf.tsf_status_string(0) == "ok"
    assert "NaN" in tsf.tsf_status_string(tsf.TSF_ENAN)
    L = tsf.lib()
    h = ctypes.c_void_p()
    # grid below 2 per axis and null pointers are rejected before any CUDA call
    assert L.tsf_create_field(1, 4, 4, ctypes.c_void_p(1), 0, None, ctypes.byref(h)) == tsf.TSF_EINVAL
    assert L.tsf_create_field(4, 4, 4, None, 0, None, ctypes.byref(h)) == tsf.TSF_EINVAL
    assert L.tsf_solver_step(None, None, None) == tsf.TSF_EINVAL
    assert L.tsf_destroy_field(None) == 0


def test_struct_layouts():
    assert ctypes.sizeof(tsf.tsf_pair) == 40
    assert ctypes.sizeof(tsf.tsf_params) == 24
    assert ctypes.sizeof(tsf.tsf_stats) == 192
