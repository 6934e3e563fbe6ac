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


def _c_layout(struct, fields):
    """sizeof and offsetof as the C compiler sees them in include/tsf.h."""
    import shutil
    import subprocess
    import tempfile
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    body = "".join(f'  printf("%zu\\n", offsetof({struct}, {f}));\n' for f in fields)
    src = f"""#include <stddef.h>
#include <stdio.h>
#include "tsf.h"
int main(void) {{
  printf("%zu\\n", sizeof({struct}));
{body}  return 0;
}}
"""
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "l.c"), os.path.join(d, "l")
        open(c, "w").write(src)
        subprocess.run([cc, "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    return [int(x) for x in out]


@pytest.mark.parametrize("name", ["tsf_pair", "tsf_params", "tsf_stats"])
def test_struct_layouts_match_the_header(name):
    S = getattr(tsf, name)
    fields = [f for f, _ in S._fields_]
    got = _c_layout(name, fields)
    assert got[0] == ctypes.sizeof(S)
    assert got[1:] == [getattr(S, f).offset for f in fields]


def test_binding_constants_match_the_header():
    text = open(os.path.join(ROOT, "include", "tsf.h")).read()
    defs = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(TSF_\w+)\s+\(?(-?\d+)\)?", text)}
    assert tsf.INCREMENTAL_ORDER_MAX == defs["TSF_INCREMENTAL_ORDER_MAX"]
    assert tsf.TSF_NSTAGES == defs["TSF_NSTAGES"]
    for name in ("TSF_OK", "TSF_EINVAL", "TSF_ENAN", "TSF_ENOMEM", "TSF_ECUDA", "TSF_ETIMEOUT", "TSF_ENOTARGET",
                 "TSF_ECAPACITY", "TSF_EINTERNAL"):
        assert getattr(tsf, name) == defs[name], name


def test_batch_argument_checks_need_no_gpu(libpath):
    import numpy as np
    L = tsf.lib()
    out = ctypes.c_void_p()
    dims = (ctypes.c_int * 1)(4)
    vals = (ctypes.c_void_p * 1)(1)
    assert L.tsf_batch_create(0, dims, dims, dims, vals, 0, ctypes.byref(out)) == tsf.TSF_EINVAL
    assert L.tsf_batch_create(1, None, dims, dims, vals, 0, ctypes.byref(out)) == tsf.TSF_EINVAL
    assert L.tsf_batch_create(1, dims, dims, dims, None, 0, ctypes.byref(out)) == tsf.TSF_EINVAL
    assert L.tsf_batch_create(1, dims, dims, dims, vals, 0, None) == tsf.TSF_EINVAL
    assert L.tsf_batch_destroy(None) == tsf.TSF_OK
    assert L.tsf_batch_size(None) == 0
    assert L.tsf_batch_field(None, 0, ctypes.byref(out)) == tsf.TSF_EINVAL
    assert L.tsf_batch_set_signal_thresholds(None, None) == tsf.TSF_EINVAL
    p = tsf.params()
    assert L.tsf_batch_step(None, ctypes.byref(p), None) == tsf.TSF_EINVAL
    assert L.tsf_batch_simplify(None, ctypes.byref(p), None) == tsf.TSF_EINVAL
    with pytest.raises(ValueError):
        tsf.Batch([np.zeros((4, 4), np.float32)])


def test_params_carry_the_assignment_precision():
    p = tsf.params(assignment_precision=0.01)
    assert abs(p.assignment_precision - 0.01) < 1e-9
    assert tsf.params().assignment_precision == 0.0
    assert "assign_rounds" in dict(tsf.tsf_stats._fields_)


def test_warm_start_and_knob_entry_points_check_arguments_without_a_gpu(libpath):
    """The network's parameter count agrees between the header, the library
    and the layer list; the new entry points reject bad arguments before any
    CUDA call; the schedule knobs round-trip and refuse unknown ids."""
    import numpy as np
    L = tsf.lib()
    text = open(os.path.join(ROOT, "include", "tsf.h")).read()
    n = int(re.search(r"#define\s+TSF_UNET_NPARAMS\s+(\d+)", text).group(1))
    assert tsf.TSF_UNET_NPARAMS == n == tsf.tsf_unet_num_params()
    assert sum(int(np.prod(ws)) + nb for _, ws, nb in tsf.unet_layer_shapes()) == n
    h = ctypes.c_void_p()
    buf = np.zeros(4, np.float32)
    assert L.tsf_unet_create(buf.ctypes.data, 4, None, ctypes.byref(h)) == tsf.TSF_EINVAL
    assert L.tsf_unet_create(None, n, None, ctypes.byref(h)) == tsf.TSF_EINVAL
    assert L.tsf_unet_destroy(None) == tsf.TSF_OK
    assert L.tsf_unet_forward(None, 8, 8, 8, buf.ctypes.data, ctypes.c_float(0.1), buf.ctypes.data, 0) == tsf.TSF_EINVAL
    assert L.tsf_unet_get_params(None, buf.ctypes.data, n) == tsf.TSF_EINVAL
    assert L.tsf_set_start_field(None, buf.ctypes.data, 0) == tsf.TSF_EINVAL
    c = ctypes.c_int(0)
    assert L.tsf_batch_autotune(None, ctypes.byref(c), None, 0) == tsf.TSF_EINVAL
    assert tsf.tsf_debug_set(99, 1) == -1
    for knob in (1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12):
        old = tsf.tsf_debug_set(knob, 5)
        assert tsf.tsf_debug_set(knob, old) == 5
