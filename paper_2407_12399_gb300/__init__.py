"""Python binding of libtsf.so, the GB300 topological simplification solver.

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  The functions keep the C ABI's names and arguments
(include/tsf.h); ``Field`` wraps them for numpy arrays and torch tensors.
Importing this package needs no GPU; the first call that touches the
library loads it and fails loudly if it has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtsf.so")

TSF_OK = 0
TSF_EINVAL = -1
TSF_ENAN = -2
TSF_ENOMEM = -3
TSF_ECUDA = -4
TSF_ETIMEOUT = -5
TSF_ENOTARGET = -6
TSF_ECAPACITY = -7
TSF_EINTERNAL = -8


class tsf_pair(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("essential", ctypes.c_int32), ("v_birth", ctypes.c_uint32),
                ("v_death", ctypes.c_uint32), ("cell_birth", ctypes.c_uint64), ("cell_death", ctypes.c_uint64),
                ("birth", ctypes.c_float), ("death", ctypes.c_float)]


PAIR_DTYPE = np.dtype([("dim", np.int32), ("essential", np.int32), ("v_birth", np.uint32), ("v_death", np.uint32),
                       ("cell_birth", np.uint64), ("cell_death", np.uint64), ("birth", np.float32),
                       ("death", np.float32)])
assert PAIR_DTYPE.itemsize == ctypes.sizeof(tsf_pair) == 40


class tsf_params(ctypes.Structure):
    _fields_ = [("alpha_b", ctypes.c_float), ("alpha_d", ctypes.c_float), ("stop_s", ctypes.c_float),
                ("cancel_eps", ctypes.c_float), ("max_iters", ctypes.c_int32),
                ("fast_gradient_update", ctypes.c_int32), ("fast_assignment_update", ctypes.c_int32),
                ("assignment_precision", ctypes.c_float)]


class tsf_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("done", ctypes.c_int32), ("loss0", ctypes.c_double),
                ("loss", ctypes.c_double), ("n_points", ctypes.c_int64), ("n_pairs", ctypes.c_int64 * 3),
                ("n_critical", ctypes.c_int64 * 4), ("n_uncancelled", ctypes.c_int64), ("n_still", ctypes.c_int64),
                ("n_nonstill_matched", ctypes.c_int64), ("n_updated_vertices", ctypes.c_int64),
                ("n_gradient_vertices", ctypes.c_int64), ("d1_columns", ctypes.c_int64),
                ("d1_blocks_total", ctypes.c_int64), ("d1_blocks_max", ctypes.c_int64),
                ("d1_rounds_total", ctypes.c_int64), ("d1_rounds_max", ctypes.c_int64),
                ("d1_star_updates", ctypes.c_int64), ("ms_diagram", ctypes.c_double),
                ("ms_assign", ctypes.c_double), ("ms_step", ctypes.c_double), ("assign_rounds", ctypes.c_int64),
                ("assign_phases", ctypes.c_int64), ("assign_checks", ctypes.c_int64),
                ("d1_reduce_rounds", ctypes.c_int64), ("d1_reduce_merged", ctypes.c_int64),
                ("d1_reduce_longest", ctypes.c_int64), ("d1_reduce_big_rounds", ctypes.c_int64),
                ("d1_reduce_big_cycles", ctypes.c_int64), ("d1_reduce_cycles", ctypes.c_int64),
                ("d1_chain_adds", ctypes.c_int64), ("d1_chain_longest", ctypes.c_int64),
                ("d1_chain_rounds", ctypes.c_int64), ("d1_chain_cycles", ctypes.c_int64)]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, ctypes.Array) else v
        return out


EXPORTS = ("tsf_create_field", "tsf_destroy_field", "tsf_compute_diagram", "tsf_set_signal_threshold",
           "tsf_set_signal_pairs", "tsf_solver_step", "tsf_simplify", "tsf_get_field", "tsf_set_field",
           "tsf_get_assignment", "tsf_get_targets", "tsf_zero_pairs", "tsf_status_string", "tsf_profile_enable",
           "tsf_profile_read", "tsf_stage_name", "tsf_kernel_launches", "tsf_zero_pairs_static",
           "tsf_loss_and_gradient", "tsf_batch_create", "tsf_batch_destroy", "tsf_batch_size", "tsf_batch_field",
           "tsf_batch_set_signal_thresholds", "tsf_batch_step", "tsf_batch_simplify", "tsf_unet_num_params", "tsf_set_start_field", "tsf_debug_set", "tsf_batch_autotune",
           "tsf_unet_create", "tsf_unet_destroy", "tsf_unet_get_params", "tsf_unet_forward", "tsf_unet_gradients",
           "tsf_unet_train_step", "tsf_unet_debug")
TSF_UNET_NPARAMS = 353713
TSF_NSTAGES = 12
INCREMENTAL_ORDER_MAX = 8192  # TSF_INCREMENTAL_ORDER_MAX

_lib = None


def lib():
    """The loaded library; raises if the CUDA extension was not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2407_12399_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        I = ctypes.c_int
        I64 = ctypes.c_int64
        sig = {
            "tsf_create_field": [I, I, I, P, I, P, ctypes.POINTER(P)],
            "tsf_destroy_field": [P],
            "tsf_compute_diagram": [P, P, I64, ctypes.POINTER(I64), I],
            "tsf_set_signal_threshold": [P, ctypes.c_float],
            "tsf_set_signal_pairs": [P, P, I64],
            "tsf_solver_step": [P, ctypes.POINTER(tsf_params), ctypes.POINTER(tsf_stats)],
            "tsf_simplify": [P, ctypes.POINTER(tsf_params), P, I, ctypes.POINTER(tsf_stats)],
            "tsf_get_field": [P, P, I],
            "tsf_set_field": [P, P, I],
            "tsf_get_assignment": [P, P, P, I64, ctypes.POINTER(I64)],
            "tsf_get_targets": [P, P, I64, ctypes.POINTER(I64)],
            "tsf_zero_pairs": [P, P, I64, ctypes.POINTER(I64)],
            "tsf_zero_pairs_static": [I, I, I, P, P, I64, ctypes.POINTER(I64), P],
            "tsf_loss_and_gradient": [P, P, I, ctypes.POINTER(ctypes.c_double), P, I],
            "tsf_batch_create": [I, P, P, P, P, I, ctypes.POINTER(P)],
            "tsf_batch_destroy": [P],
            "tsf_batch_size": [P],
            "tsf_batch_field": [P, I, ctypes.POINTER(P)],
            "tsf_batch_set_signal_thresholds": [P, P],
            "tsf_batch_step": [P, ctypes.POINTER(tsf_params), P],
            "tsf_batch_simplify": [P, ctypes.POINTER(tsf_params), P],
            "tsf_batch_autotune": [P, ctypes.POINTER(I), P, I],
            "tsf_set_start_field": [P, P, I],
            "tsf_unet_create": [P, I64, P, ctypes.POINTER(P)],
            "tsf_unet_destroy": [P],
            "tsf_unet_get_params": [P, P, I64],
            "tsf_unet_forward": [P, I, I, I, P, ctypes.c_float, P, I],
            "tsf_unet_gradients": [P, I, I, I, P, P, I, ctypes.c_float, P, ctypes.POINTER(ctypes.c_double)],
            "tsf_unet_train_step": [P, I, I, I, P, P, I, ctypes.c_float, ctypes.c_float,
                                    ctypes.POINTER(ctypes.c_double)],
            "tsf_unet_debug": [P, I, I, I, P, P, ctypes.c_float, P, I64, P, I64],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.tsf_status_string.argtypes = [ctypes.c_int]
        L.tsf_status_string.restype = ctypes.c_char_p
        L.tsf_profile_enable.argtypes = [P, I]
        L.tsf_profile_enable.restype = I
        L.tsf_profile_read.argtypes = [P, P, P, I]
        L.tsf_profile_read.restype = I
        L.tsf_stage_name.argtypes = [I]
        L.tsf_stage_name.restype = ctypes.c_char_p
        L.tsf_kernel_launches.argtypes = []
        L.tsf_kernel_launches.restype = ctypes.c_int64
        L.tsf_debug_set.argtypes = [I, ctypes.c_int64]
        L.tsf_debug_set.restype = ctypes.c_int64
        L.tsf_unet_num_params.argtypes = []
        L.tsf_unet_num_params.restype = ctypes.c_int64
        _lib = L
    return _lib


class TsfError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {tsf_status_string(code)} ({code})")


def tsf_status_string(code: int) -> str:
    return lib().tsf_status_string(code).decode()


def _check(code, where):
    if code != TSF_OK:
        raise TsfError(code, where)


# --- thin wrappers with the C names (pointers as ints, sizes as ints) -------
def tsf_create_field(lx, ly, lz, values_ptr, values_on_device, cuda_stream=0):
    h = ctypes.c_void_p()
    _check(lib().tsf_create_field(lx, ly, lz, values_ptr, values_on_device, cuda_stream or None, ctypes.byref(h)),
           "tsf_create_field")
    return h


def tsf_destroy_field(h):
    return lib().tsf_destroy_field(h)


def tsf_compute_diagram(h, out_ptr, cap, out_on_device=0):
    n = ctypes.c_int64(0)
    r = lib().tsf_compute_diagram(h, out_ptr, cap, ctypes.byref(n), out_on_device)
    return r, n.value


def tsf_set_signal_threshold(h, fraction):
    _check(lib().tsf_set_signal_threshold(h, fraction), "tsf_set_signal_threshold")


def tsf_set_signal_pairs(h, pairs_ptr, n):
    _check(lib().tsf_set_signal_pairs(h, pairs_ptr, n), "tsf_set_signal_pairs")


def tsf_solver_step(h, params, stats=None):
    st = stats if stats is not None else tsf_stats()
    _check(lib().tsf_solver_step(h, ctypes.byref(params), ctypes.byref(st)), "tsf_solver_step")
    return st


def tsf_simplify(h, params, out_ptr=None, out_on_device=0, stats=None):
    st = stats if stats is not None else tsf_stats()
    _check(lib().tsf_simplify(h, ctypes.byref(params), out_ptr, out_on_device, ctypes.byref(st)), "tsf_simplify")
    return st


def tsf_get_field(h, out_ptr, out_on_device=0):
    _check(lib().tsf_get_field(h, out_ptr, out_on_device), "tsf_get_field")


def tsf_set_start_field(h, values_ptr, values_on_device=0):
    _check(lib().tsf_set_start_field(h, values_ptr, values_on_device), "tsf_set_start_field")


def tsf_set_field(h, values_ptr, values_on_device=0):
    _check(lib().tsf_set_field(h, values_ptr, values_on_device), "tsf_set_field")


def tsf_get_assignment(h, target_ptr, still_ptr, cap):
    n = ctypes.c_int64(0)
    r = lib().tsf_get_assignment(h, target_ptr, still_ptr, cap, ctypes.byref(n))
    return r, n.value


def tsf_get_targets(h, out_ptr, cap):
    n = ctypes.c_int64(0)
    r = lib().tsf_get_targets(h, out_ptr, cap, ctypes.byref(n))
    return r, n.value


def tsf_zero_pairs(h, out_ptr, cap):
    n = ctypes.c_int64(0)
    r = lib().tsf_zero_pairs(h, out_ptr, cap, ctypes.byref(n))
    return r, n.value


def tsf_zero_pairs_static(lx, ly, lz, values_ptr, out_ptr, cap, cuda_stream=0):
    """No-allocation variant of tsf_zero_pairs (device pointers in and out)."""
    n = ctypes.c_int64(0)
    r = lib().tsf_zero_pairs_static(lx, ly, lz, values_ptr, out_ptr, cap, ctypes.byref(n), cuda_stream or None)
    return r, n.value


def tsf_loss_and_gradient(h, values_ptr, values_on_device, grad_ptr, grad_on_device):
    """Loss of the values at values_ptr against the target diagram; dL/df
    (float64) written at grad_ptr (may be None)."""
    loss = ctypes.c_double(0.0)
    _check(lib().tsf_loss_and_gradient(h, values_ptr, values_on_device, ctypes.byref(loss), grad_ptr, grad_on_device),
           "tsf_loss_and_gradient")
    return loss.value


def tsf_batch_create(shapes, values_ptrs, values_on_device):
    """shapes: (Lz, Ly, Lx) per field; values_ptrs: one pointer per field."""
    n = len(shapes)
    lx = (ctypes.c_int * n)(*[s[2] for s in shapes])
    ly = (ctypes.c_int * n)(*[s[1] for s in shapes])
    lz = (ctypes.c_int * n)(*[s[0] for s in shapes])
    vp = (ctypes.c_void_p * n)(*values_ptrs)
    h = ctypes.c_void_p()
    _check(lib().tsf_batch_create(n, lx, ly, lz, vp, values_on_device, ctypes.byref(h)), "tsf_batch_create")
    return h


def tsf_batch_destroy(h):
    return lib().tsf_batch_destroy(h)


def tsf_batch_size(h):
    return lib().tsf_batch_size(h)


def tsf_batch_field(h, i):
    f = ctypes.c_void_p()
    _check(lib().tsf_batch_field(h, i, ctypes.byref(f)), "tsf_batch_field")
    return f


def tsf_batch_set_signal_thresholds(h, fractions):
    a = np.ascontiguousarray(fractions, np.float32)
    _check(lib().tsf_batch_set_signal_thresholds(h, a.ctypes.data), "tsf_batch_set_signal_thresholds")


def tsf_batch_step(h, params, n):
    st = (tsf_stats * n)()
    _check(lib().tsf_batch_step(h, ctypes.byref(params), st), "tsf_batch_step")
    return [s.as_dict() for s in st]


def tsf_batch_simplify(h, params, n):
    st = (tsf_stats * n)()
    _check(lib().tsf_batch_simplify(h, ctypes.byref(params), st), "tsf_batch_simplify")
    return [s.as_dict() for s in st]


def tsf_batch_autotune(h, ncand=4):
    """Chooses the D1 phase-A schedule for the batch; returns (choice, ms per candidate)."""
    c = ctypes.c_int(0)
    ms = np.zeros(ncand, np.float64)
    _check(lib().tsf_batch_autotune(h, ctypes.byref(c), ms.ctypes.data, ncand), "tsf_batch_autotune")
    return c.value, ms.tolist()


def tsf_profile_enable(h, enable=1):
    _check(lib().tsf_profile_enable(h, enable), "tsf_profile_enable")


def tsf_profile_read(h):
    ms = np.zeros(TSF_NSTAGES, np.float64)
    calls = np.zeros(TSF_NSTAGES, np.int64)
    _check(lib().tsf_profile_read(h, ms.ctypes.data, calls.ctypes.data, TSF_NSTAGES), "tsf_profile_read")
    return {tsf_stage_name(i): (float(ms[i]), int(calls[i])) for i in range(TSF_NSTAGES)}


def tsf_stage_name(i):
    return lib().tsf_stage_name(i).decode()


def tsf_debug_set(what, value):
    """Test and tuning knob (include/tsf.h); returns the previous value."""
    return int(lib().tsf_debug_set(what, value))


def tsf_kernel_launches():
    return int(lib().tsf_kernel_launches())


def params(alpha_b=0.5, alpha_d=0.5, stop_s=0.01, cancel_eps=0.0, max_iters=1000, fast_gradient_update=1,
           fast_assignment_update=1, assignment_precision=0.0):
    return tsf_params(alpha_b, alpha_d, stop_s, cancel_eps, max_iters, fast_gradient_update, fast_assignment_update,
                      assignment_precision)


def _ptr_of(a):
    """(pointer, on_device) of a numpy array or a torch tensor."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data, 0
    try:
        import torch
        if isinstance(a, torch.Tensor):
            return a.data_ptr(), 1 if a.is_cuda else 0
    except ImportError:  # pragma: no cover
        pass
    raise TypeError(type(a))


class Field:
    """A field on the GPU.  values: (Lz, Ly, Lx) float32 numpy array or tensor."""

    def __init__(self, values, stream=None):
        shape = tuple(values.shape)
        if len(shape) != 3:
            raise ValueError("values must be (Lz, Ly, Lx)")
        if isinstance(values, np.ndarray):
            values = np.ascontiguousarray(values, dtype=np.float32)
        else:
            values = values.contiguous()
        self.shape = shape
        lz, ly, lx = shape
        p, dev = _ptr_of(values)
        s = 0
        if stream is not None:
            s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self._h = tsf_create_field(lx, ly, lz, p, dev, s)

    def close(self):
        if getattr(self, "_h", None):
            tsf_destroy_field(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def diagram(self):
        r, n = tsf_compute_diagram(self._h, None, 0)
        if r not in (TSF_OK, TSF_ECAPACITY):
            _check(r, "tsf_compute_diagram")
        out = np.zeros(n, PAIR_DTYPE)
        r, n = tsf_compute_diagram(self._h, out.ctypes.data, n)
        _check(r, "tsf_compute_diagram")
        return out

    def set_threshold(self, fraction):
        tsf_set_signal_threshold(self._h, fraction)

    def set_targets(self, pairs):
        pairs = np.ascontiguousarray(pairs, PAIR_DTYPE)
        tsf_set_signal_pairs(self._h, pairs.ctypes.data, len(pairs))

    def step(self, **kw):
        return tsf_solver_step(self._h, params(**kw)).as_dict()

    def simplify(self, **kw):
        out = np.zeros(self.shape, np.float32)
        st = tsf_simplify(self._h, params(**kw), out.ctypes.data, 0)
        return out, st.as_dict()

    def values(self):
        out = np.zeros(self.shape, np.float32)
        tsf_get_field(self._h, out.ctypes.data, 0)
        return out

    def loss_and_grad(self, values, grad_out=None):
        """Topological loss of `values` (numpy array or tensor of the field's
        shape) against the target diagram, and dL/df into `grad_out` (float64
        numpy array or tensor of the same shape, host or device; allocated on
        the host when None).  The values become the field's values."""
        if isinstance(values, np.ndarray):
            values = np.ascontiguousarray(values, np.float32)
        else:
            values = values.contiguous()
        vp, von = _ptr_of(values)
        if grad_out is None:
            grad_out = np.zeros(self.shape, np.float64)
        gp, gon = _ptr_of(grad_out)
        return tsf_loss_and_gradient(self._h, vp, von, gp, gon), grad_out

    def assignment(self):
        r, n = tsf_get_assignment(self._h, None, None, 0)
        tgt = np.zeros(n, np.int32)
        still = np.zeros(n, np.int32)
        r, n = tsf_get_assignment(self._h, tgt.ctypes.data, still.ctypes.data, n)
        _check(r, "tsf_get_assignment")
        return tgt, still

    def targets(self):
        r, n = tsf_get_targets(self._h, None, 0)
        out = np.zeros(n, PAIR_DTYPE)
        r, n = tsf_get_targets(self._h, out.ctypes.data, n)
        _check(r, "tsf_get_targets")
        return out

    def zero_pairs(self):
        r, n = tsf_zero_pairs(self._h, None, 0)
        out = np.zeros(2 * max(n, 1), np.uint64)
        r, n = tsf_zero_pairs(self._h, out.ctypes.data, n)
        _check(r, "tsf_zero_pairs")
        return out[: 2 * n].reshape(-1, 2)


class _BatchMember(Field):
    """A field owned by a Batch: the single-field calls work on it, but the
    batch frees it."""

    def __init__(self, h, shape):
        self._h = h
        self.shape = shape

    def close(self):
        self._h = None


class Batch:
    """Independent fields solved together (one stream and one host worker
    per field, all fields' kernels in flight at once).  fields: sequence of
    (Lz, Ly, Lx) float32 arrays or tensors, all on the host or all on the
    device.  A field's trajectory is the one it has when solved alone."""

    def __init__(self, fields):
        shapes, ptrs, on_dev = [], [], set()
        keep = []
        for v in fields:
            if len(v.shape) != 3:
                raise ValueError("values must be (Lz, Ly, Lx)")
            v = np.ascontiguousarray(v, np.float32) if isinstance(v, np.ndarray) else v.contiguous()
            p, dev = _ptr_of(v)
            keep.append(v)
            shapes.append(tuple(v.shape))
            ptrs.append(p)
            on_dev.add(dev)
        if len(on_dev) != 1:
            raise ValueError("batch fields must be all on the host or all on the device")
        self.shapes = shapes
        self._h = tsf_batch_create(shapes, ptrs, on_dev.pop())
        self.fields = [_BatchMember(tsf_batch_field(self._h, i), s) for i, s in enumerate(shapes)]

    def __len__(self):
        return len(self.shapes)

    def close(self):
        if getattr(self, "_h", None):
            for f in self.fields:
                f.close()
            tsf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self):
        """Before set_thresholds: time each candidate D1 tile on the batch and
        keep the fastest; returns (choice, ms per candidate)."""
        return tsf_batch_autotune(self._h)

    def set_thresholds(self, fractions):
        tsf_batch_set_signal_thresholds(self._h, fractions)

    def step(self, **kw):
        return tsf_batch_step(self._h, params(**kw), len(self))

    def simplify(self, **kw):
        return tsf_batch_simplify(self._h, params(**kw), len(self))

    def values(self):
        return [f.values() for f in self.fields]


# --- learned warm start (tsf_unet_*) --------------------------------------
def tsf_unet_num_params():
    return int(lib().tsf_unet_num_params())


def tsf_unet_create(params_ptr, n, cuda_stream=0):
    h = ctypes.c_void_p()
    _check(lib().tsf_unet_create(params_ptr, n, cuda_stream or None, ctypes.byref(h)), "tsf_unet_create")
    return h


def tsf_unet_destroy(h):
    return lib().tsf_unet_destroy(h)


def tsf_unet_get_params(h, out_ptr, n):
    _check(lib().tsf_unet_get_params(h, out_ptr, n), "tsf_unet_get_params")


def tsf_unet_forward(h, lx, ly, lz, f_ptr, tau, g0_ptr, on_device):
    _check(lib().tsf_unet_forward(h, lx, ly, lz, f_ptr, tau, g0_ptr, on_device), "tsf_unet_forward")


def tsf_unet_gradients(h, lx, ly, lz, f_ptr, g_ptr, on_device, tau, grad_ptr):
    loss = ctypes.c_double(0.0)
    _check(lib().tsf_unet_gradients(h, lx, ly, lz, f_ptr, g_ptr, on_device, tau, grad_ptr, ctypes.byref(loss)),
           "tsf_unet_gradients")
    return loss.value


def tsf_unet_train_step(h, lx, ly, lz, f_ptr, g_ptr, on_device, tau, lr):
    loss = ctypes.c_double(0.0)
    _check(lib().tsf_unet_train_step(h, lx, ly, lz, f_ptr, g_ptr, on_device, tau, lr, ctypes.byref(loss)),
           "tsf_unet_train_step")
    return loss.value


def tsf_unet_debug(h, lx, ly, lz, f_ptr, g_ptr, tau, acts_ptr, acts_cap, gz_ptr, gz_cap):
    _check(lib().tsf_unet_debug(h, lx, ly, lz, f_ptr, g_ptr, tau, acts_ptr, acts_cap, gz_ptr, gz_cap),
           "tsf_unet_debug")


UNET_CHANNELS = (16, 32, 64)


def unet_layer_shapes():
    """(name, weight shape, bias length) of every layer, in parameter order
    (the order tsf.h states)."""
    c1, c2, c3 = UNET_CHANNELS
    convs = [("e1a", c1, 2), ("e1b", c1, c1), ("e2a", c2, c1), ("e2b", c2, c2), ("e3a", c3, c2), ("e3b", c3, c3),
             ("d2a", c2, c3 + c2), ("d2b", c2, c2), ("d1a", c1, c2 + c1), ("d1b", c1, c1)]
    return [(n, (co, ci, 3, 3, 3), co) for n, co, ci in convs] + [("head", (1, c1), 1)]


def unet_flatten(p):
    """Parameter dict {name.w, name.b} -> the flat float32 vector."""
    return np.concatenate([np.asarray(p[n + k], np.float64).ravel() for n, _, _ in unet_layer_shapes()
                           for k in (".w", ".b")]).astype(np.float32)


def unet_unflatten(flat):
    out, o = {}, 0
    for n, ws, nb in unet_layer_shapes():
        k = int(np.prod(ws))
        out[n + ".w"] = np.asarray(flat[o:o + k]).reshape(ws)
        out[n + ".b"] = np.asarray(flat[o + k:o + k + nb])
        o += k + nb
    return out


def unet_init(seed=0):
    """He-normal weights (std sqrt(2 / fan_in)), zero biases, a zero head (the
    untrained network returns f), as a flat float32 vector."""
    rng = np.random.default_rng(seed)
    p = {}
    for n, ws, nb in unet_layer_shapes():
        fan_in = int(np.prod(ws[1:]))
        p[n + ".w"] = np.zeros(ws) if n == "head" else rng.normal(0.0, np.sqrt(2.0 / fan_in), ws)
        p[n + ".b"] = np.zeros(nb)
    return unet_flatten(p)


class UNet:
    """The warm-start network on the current CUDA device."""

    def __init__(self, params=None, seed=0, stream=None):
        flat = unet_init(seed) if params is None else np.ascontiguousarray(params, np.float32)
        assert flat.size == TSF_UNET_NPARAMS
        self._h = tsf_unet_create(flat.ctypes.data, flat.size, stream.cuda_stream if stream is not None else 0)

    def close(self):
        if getattr(self, "_h", None):
            tsf_unet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        out = np.empty(TSF_UNET_NPARAMS, np.float32)
        tsf_unet_get_params(self._h, out.ctypes.data, out.size)
        return out

    def forward(self, f, tau):
        """g0 for f: a torch CUDA tensor (returns one) or a numpy array."""
        if hasattr(f, "data_ptr"):
            import torch
            g0 = torch.empty_like(f)
            lz, ly, lx = f.shape
            tsf_unet_forward(self._h, lx, ly, lz, f.data_ptr(), tau, g0.data_ptr(), 1)
            return g0
        f = np.ascontiguousarray(f, np.float32)
        g0 = np.empty_like(f)
        lz, ly, lx = f.shape
        tsf_unet_forward(self._h, lx, ly, lz, f.ctypes.data, tau, g0.ctypes.data, 0)
        return g0

    def gradients(self, f, g, tau):
        f = np.ascontiguousarray(f, np.float32)
        g = np.ascontiguousarray(g, np.float32)
        grad = np.empty(TSF_UNET_NPARAMS, np.float32)
        lz, ly, lx = f.shape
        loss = tsf_unet_gradients(self._h, lx, ly, lz, f.ctypes.data, g.ctypes.data, 0, tau, grad.ctypes.data)
        return loss, grad

    def train_step(self, f, g, tau, lr):
        """One Adam step on the pair (f, g): torch CUDA tensors or numpy arrays."""
        lz, ly, lx = f.shape
        if hasattr(f, "data_ptr"):
            return tsf_unet_train_step(self._h, lx, ly, lz, f.data_ptr(), g.data_ptr(), 1, tau, lr)
        f = np.ascontiguousarray(f, np.float32)
        g = np.ascontiguousarray(g, np.float32)
        return tsf_unet_train_step(self._h, lx, ly, lz, f.ctypes.data, g.ctypes.data, 0, tau, lr)

    ACT_KEYS = (("x", 2, 1), ("e1a", 16, 1), ("e1b", 16, 1), ("e2a", 32, 2), ("e2b", 32, 2), ("e3a", 64, 4),
                ("e3b", 64, 4), ("d2a", 32, 2), ("d2b", 32, 2), ("d1a", 16, 1), ("d1b", 16, 1), ("g0", 1, 1))
    GZ_KEYS = (("d1b", 16, 1), ("d1a", 16, 1), ("d2b", 32, 2), ("d2a", 32, 2), ("e3b", 64, 4), ("e3a", 64, 4),
               ("e2b", 32, 2), ("e2a", 32, 2), ("e1b", 16, 1), ("e1a", 16, 1))

    def debug(self, f, tau, g=None):
        """Every stored activation (and, with g, every pre-activation
        gradient) as float32 arrays (C, z, y, x) keyed by layer."""
        f = np.ascontiguousarray(f, np.float32)
        lz, ly, lx = f.shape

        def layout(keys):
            out, o = [], 0
            for k, c, s in keys:
                shape = (c, lz // s, ly // s, lx // s)
                out.append((k, o, shape))
                o += int(np.prod(shape))
            return out, o

        al, an = layout(self.ACT_KEYS)
        gl, gn = layout(self.GZ_KEYS)
        acts = np.empty(an, np.float32)
        gz = np.empty(gn, np.float32) if g is not None else None
        gp = np.ascontiguousarray(g, np.float32) if g is not None else None
        tsf_unet_debug(self._h, lx, ly, lz, f.ctypes.data, gp.ctypes.data if gp is not None else None, tau,
                       acts.ctypes.data, an, gz.ctypes.data if gz is not None else None, gn if gz is not None else 0)
        A = {k: acts[o:o + int(np.prod(sh))].reshape(sh) for k, o, sh in al}
        A["g0"] = A["g0"][0]
        G = {k: gz[o:o + int(np.prod(sh))].reshape(sh) for k, o, sh in gl} if gz is not None else None
        return A, G
