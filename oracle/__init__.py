"""CPU oracle for the topological simplification solver (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path
(package ``paper_2407_12399_gb300``) never imports this package, and the two
share no code.  See ``oracle.c`` for what each function follows in the paper.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile liboracle.so next to the sources (gcc, no FMA contraction)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    try:
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    finally:
        if os.path.exists(tmp):
            os.unlink(tmp)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        L.or_diagram_compute.restype = P
        L.or_diagram_compute.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, ctypes.POINTER(ctypes.c_int)]
        L.or_diagram_count.restype = I64
        L.or_diagram_count.argtypes = [P, ctypes.c_int]
        L.or_diagram_get.argtypes = [P, ctypes.c_int, P, P, P, P, P, P]
        L.or_diagram_filtration.argtypes = [P, P]
        L.or_diagram_ranks.argtypes = [P, P]
        L.or_diagram_free.argtypes = [P]
        L.or_solver_create.restype = P
        L.or_solver_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, ctypes.c_float,
                                       ctypes.POINTER(ctypes.c_int)]
        L.or_solver_create_targets.restype = P
        L.or_solver_create_targets.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, I64, P, P, P, P, P, P,
                                               ctypes.POINTER(ctypes.c_int)]
        L.or_solver_iterate.restype = ctypes.c_int
        L.or_solver_iterate.argtypes = [P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                        ctypes.c_int]
        L.or_solver_done.restype = ctypes.c_int
        L.or_solver_done.argtypes = [P, ctypes.c_float, ctypes.c_float, ctypes.c_int]
        L.or_solver_set_fast_assignment.restype = None
        L.or_solver_set_fast_assignment.argtypes = [P, ctypes.c_int]
        L.or_solver_set_assignment_precision.restype = None
        L.or_solver_set_assignment_precision.argtypes = [P, ctypes.c_double]
        L.or_solver_loss_grad.restype = ctypes.c_int
        L.or_solver_loss_grad.argtypes = [P, P, P, P]
        L.or_solver_field.argtypes = [P, P]
        L.or_solver_set_start.restype = ctypes.c_int
        L.or_solver_set_start.argtypes = [P, P]
        L.or_solver_num_points.restype = I64
        L.or_solver_num_points.argtypes = [P]
        L.or_solver_num_targets.restype = I64
        L.or_solver_num_targets.argtypes = [P]
        L.or_solver_points.argtypes = [P] + [P] * 10
        L.or_solver_targets.argtypes = [P] + [P] * 6
        L.or_solver_stats.argtypes = [P, P, P]
        L.or_solver_free.argtypes = [P]
        L.or_assign.restype = ctypes.c_double
        L.or_assign.argtypes = [I64, P, P, I64, P, P, P]
        L.or_assign_prec.restype = ctypes.c_double
        L.or_assign_prec.argtypes = [I64, P, P, I64, P, P, ctypes.c_double, P]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _field(f):
    f = np.ascontiguousarray(np.asarray(f, dtype=np.float32))
    if f.ndim != 3:
        raise ValueError("field must be (Lz, Ly, Lx)")
    lz, ly, lx = f.shape
    return f, lx, ly, lz


def _get_pairs(L, h, which):
    n = L.or_diagram_count(h, which)
    out = {
        "dim": np.zeros(n, np.int32), "essential": np.zeros(n, np.int32),
        "vb": np.zeros(n, np.uint32), "vd": np.zeros(n, np.uint32),
        "cb": np.zeros(n, np.uint64), "cd": np.zeros(n, np.uint64),
    }
    if n:
        L.or_diagram_get(h, which, *(_ptr(out[k]) for k in ("dim", "essential", "vb", "vd", "cb", "cd")))
    return out


def diagram(f, with_zero: bool = False, with_filtration: bool = False):
    """Persistence pairs of the lexicographic filtration of f (plain reduction).

    Returns a dict with "pairs" (v_b != v_d, plus the essential class) and,
    on request, "zero" (v_b == v_d pairs), "filtration" (cell ids in order)
    and "rank" (vertex ranks).
    """
    L = lib()
    f, lx, ly, lz = _field(f)
    st = ctypes.c_int(0)
    h = L.or_diagram_compute(lx, ly, lz, _ptr(f), ctypes.byref(st))
    if not h:
        raise ValueError(f"oracle diagram failed (status {st.value})")
    try:
        res = {"pairs": _get_pairs(L, h, 0)}
        if with_zero:
            res["zero"] = _get_pairs(L, h, 1)
        if with_filtration:
            n = L.or_diagram_count(h, 2)
            cells = np.zeros(n, np.uint64)
            L.or_diagram_filtration(h, _ptr(cells))
            res["filtration"] = cells
            rank = np.zeros(lx * ly * lz, np.uint32)
            L.or_diagram_ranks(h, _ptr(rank))
            res["rank"] = rank
        return res
    finally:
        L.or_diagram_free(h)


def _prec(p):
    """The precision as the solver sees it: a float32 parameter widened to fp64."""
    return float(np.float32(p))


def assign(pb, pd, tb, td, precision=0.0):
    """Reduced assignment of one finite group, exact (precision 0) or by the
    auction at that relative precision; returns (targets, W2^2)."""
    L = lib()
    pb = np.ascontiguousarray(pb, np.float32)
    pd = np.ascontiguousarray(pd, np.float32)
    tb = np.ascontiguousarray(tb, np.float32)
    td = np.ascontiguousarray(td, np.float32)
    out = np.zeros(len(pb), np.int32)
    cost = L.or_assign_prec(len(pb), _ptr(pb), _ptr(pd), len(tb), _ptr(tb), _ptr(td), ctypes.c_double(_prec(precision)),
                            _ptr(out))
    if cost < 0:
        raise RuntimeError("oracle auction did not finish")
    return out, cost


class Solver:
    """Algorithm 1 with Sections 4.1 and 4.3, on the CPU, one iteration at a time."""

    def __init__(self, f0, tau=None, targets=None, fast_assignment=True, assignment_precision=0.0):
        L = lib()
        f0, lx, ly, lz = _field(f0)
        self.shape = f0.shape
        st = ctypes.c_int(0)
        if targets is None:
            h = L.or_solver_create(lx, ly, lz, _ptr(f0), ctypes.c_float(tau), ctypes.byref(st))
        else:
            t = {k: np.ascontiguousarray(v) for k, v in targets.items()}
            n = len(t["vb"])
            h = L.or_solver_create_targets(
                lx, ly, lz, _ptr(f0), n, _ptr(t["dim"].astype(np.int32)), _ptr(t["essential"].astype(np.int32)),
                _ptr(t["vb"].astype(np.uint32)), _ptr(t["vd"].astype(np.uint32)),
                _ptr(t["birth"].astype(np.float32)), _ptr(t["death"].astype(np.float32)), ctypes.byref(st))
        if not h:
            raise ValueError(f"oracle solver failed (status {st.value})")
        self._h = h
        L.or_solver_set_fast_assignment(h, 1 if fast_assignment else 0)
        L.or_solver_set_assignment_precision(h, ctypes.c_double(_prec(assignment_precision)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_solver_free(h)
            self._h = None

    def iterate(self, alpha_b=0.5, alpha_d=0.5, stop_s=0.01, cancel_eps=0.0, max_iters=1000):
        r = lib().or_solver_iterate(self._h, ctypes.c_float(alpha_b), ctypes.c_float(alpha_d),
                                    ctypes.c_float(stop_s), ctypes.c_float(cancel_eps), max_iters)
        if r < 0:
            raise RuntimeError(f"oracle iterate failed ({r})")
        return bool(r)

    def done(self, stop_s=0.01, cancel_eps=0.0, max_iters=1000):
        return bool(lib().or_solver_done(self._h, ctypes.c_float(stop_s), ctypes.c_float(cancel_eps), max_iters))

    def field(self):
        out = np.zeros(self.shape, np.float32)
        lib().or_solver_field(self._h, _ptr(out))
        return out

    def points(self):
        L = lib()
        n = L.or_solver_num_points(self._h)
        out = {
            "dim": np.zeros(n, np.int32), "essential": np.zeros(n, np.int32),
            "vb": np.zeros(n, np.uint32), "vd": np.zeros(n, np.uint32),
            "birth": np.zeros(n, np.float32), "death": np.zeros(n, np.float32),
            "tgt": np.zeros(n, np.int32), "still": np.zeros(n, np.int32),
            "cb": np.zeros(n, np.uint64), "cd": np.zeros(n, np.uint64),
        }
        L.or_solver_points(self._h, *(_ptr(out[k]) for k in
                                      ("dim", "essential", "vb", "vd", "birth", "death", "tgt", "still", "cb", "cd")))
        return out

    def targets(self):
        L = lib()
        n = L.or_solver_num_targets(self._h)
        out = {
            "dim": np.zeros(n, np.int32), "essential": np.zeros(n, np.int32),
            "vb": np.zeros(n, np.uint32), "vd": np.zeros(n, np.uint32),
            "birth": np.zeros(n, np.float32), "death": np.zeros(n, np.float32),
        }
        L.or_solver_targets(self._h, *(_ptr(out[k]) for k in ("dim", "essential", "vb", "vd", "birth", "death")))
        return out

    def stats(self):
        st = np.zeros(5, np.int64)
        loss = np.zeros(2, np.float64)
        lib().or_solver_stats(self._h, _ptr(st), _ptr(loss))
        return {"iter": int(st[0]), "uncancelled": int(st[1]), "still": int(st[2]), "updated": int(st[3]),
                "nonstill_matched": int(st[4]), "loss": float(loss[0]), "loss0": float(loss[1])}

    def loss_grad(self, values):
        """(loss, dL/df as float64 of the field's shape) of `values` against the
        target diagram, every point matched by the exact solver."""
        v = np.ascontiguousarray(values, np.float32)
        assert v.shape == self.shape
        loss = np.zeros(1, np.float64)
        grad = np.zeros(self.shape, np.float64)
        r = lib().or_solver_loss_grad(self._h, _ptr(v), _ptr(loss), _ptr(grad))
        if r < 0:
            raise ValueError(f"oracle loss failed ({r})")
        return float(loss[0]), grad

    def set_start(self, values):
        """Continue from the start field `values` (warm start): same targets
        and loss_0, its diagram matched as after a step, j back to 0."""
        v = np.ascontiguousarray(values, np.float32)
        assert v.shape == self.shape
        r = lib().or_solver_set_start(self._h, _ptr(v))
        if r < 0:
            raise ValueError(f"oracle set_start failed ({r})")

    def run(self, alpha_b=0.5, alpha_d=0.5, stop_s=0.01, cancel_eps=0.0, max_iters=1000):
        while not self.done(stop_s, cancel_eps, max_iters):
            self.iterate(alpha_b, alpha_d, stop_s, cancel_eps, max_iters)
        return self.field()
