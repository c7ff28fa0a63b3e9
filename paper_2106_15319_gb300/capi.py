"""Thin ctypes binding of libserial_emd.so (the C ABI in include/serial_emd.h).

Argument marshalling only: every step of Serial-EMD runs in the library's CUDA
kernels. Functions keep the C names; tensors are torch CUDA tensors whose data
pointers are passed through. There is no CPU fallback: loading fails loudly if
the library is missing, and the calls raise when the C ABI returns an error.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

SEMD_OK, SEMD_PENDING = 0, 1
SEMD_EINVAL, SEMD_ENOMEM, SEMD_EBUDGET, SEMD_ECUDA = -1, -2, -3, -4
SEMD_ETIMEOUT, SEMD_ECANCELED, SEMD_EUNSUPPORTED = -5, -6, -7
ORDER_ROWS, ORDER_COLS = 0, 1
STOP_FIXED, STOP_SD, STOP_SNUMBER = 0, 1, 2
BOUNDARY_MIRROR, BOUNDARY_ENDPOINTS = 0, 1
SPLINE_NATURAL, SPLINE_NOT_A_KNOT = 0, 1
FP64, FP32_MIXED = 0, 1

_STATUS = {0: "OK", 1: "PENDING", -1: "EINVAL", -2: "ENOMEM", -3: "EBUDGET", -4: "ECUDA",
           -5: "ETIMEOUT", -6: "ECANCELED", -7: "EUNSUPPORTED"}


class SemdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class semd_params(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("order", ctypes.c_int32),
                ("transition_len", ctypes.c_int32), ("max_imfs", ctypes.c_int32),
                ("stop", ctypes.c_int32), ("fixed_sifts", ctypes.c_int32),
                ("max_sifts", ctypes.c_int32), ("sd_threshold", ctypes.c_double),
                ("boundary", ctypes.c_int32), ("mirror_knots", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("ensemble_trials", ctypes.c_int32),
                ("noise_rel_std", ctypes.c_double), ("s_number", ctypes.c_int32),
                ("spline_end", ctypes.c_int32)]


class semd_instance(ctypes.Structure):
    _fields_ = [("d_x", ctypes.c_void_p), ("rows", ctypes.c_int64), ("cols", ctypes.c_int64),
                ("d_imfs", ctypes.c_void_p), ("d_residue", ctypes.c_void_p)]


class semd_request(ctypes.Structure):
    _fields_ = [("d_x", ctypes.c_void_p), ("rows", ctypes.c_int64), ("cols", ctypes.c_int64),
                ("order", ctypes.c_int32), ("_reserved", ctypes.c_int32),
                ("d_imfs", ctypes.c_void_p), ("d_residue", ctypes.c_void_p)]


class semd_stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_int64), ("pass_launches", ctypes.c_int64),
                ("pass_ms", ctypes.c_double), ("reduce_launches", ctypes.c_int64),
                ("reduce_ms", ctypes.c_double), ("sample_sifts", ctypes.c_int64),
                ("pass_bytes", ctypes.c_int64), ("used_graph", ctypes.c_int32),
                ("_reserved", ctypes.c_int32)]


class semd_tune_result(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("ms", ctypes.c_double), ("ms_default", ctypes.c_double),
                ("candidates", ctypes.c_int32), ("variant", ctypes.c_int32)]


class semd_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("n_imfs", ctypes.c_int32),
                ("sifts", ctypes.c_int64), ("queue_ms", ctypes.c_double),
                ("run_ms", ctypes.c_double)]


# name -> (restype, argtypes); every symbol the header declares
SIGNATURES = {
    "serial_emd_default_params": (None, [ctypes.POINTER(semd_params)]),
    "serial_emd_plan": (ctypes.c_int, [ctypes.POINTER(semd_params), ctypes.c_int, ctypes.c_size_t,
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "serial_emd_plan_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "serial_emd_decompose": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]),
    "serial_emd_plan_set_noise_seed": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "serial_emd_decompose_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int,
                                                  ctypes.POINTER(semd_instance),
                                                  ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]),
    "serial_emd_decompose_slices": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p,
                                                   ctypes.c_int64, ctypes.c_int64,
                                                   ctypes.c_void_p, ctypes.c_void_p,
                                                   ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]),
    "serial_emd_ceemdan": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]),
    "serial_emd_eemd_trial": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "serial_emd_plan_counts": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_int)]),
    "serial_emd_extrema": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_int64),
                                          ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]),
    "serial_emd_sift": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "serial_emd_sift_noalloc": (ctypes.c_int, [ctypes.POINTER(semd_params), ctypes.c_void_p,
                                               ctypes.c_int64, ctypes.c_void_p,
                                               ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "serial_emd_plan_set_tile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "serial_emd_plan_get_tile": (ctypes.c_int, [ctypes.c_void_p]),
    "serial_emd_plan_set_pass_ctas": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "serial_emd_plan_get_pass_ctas": (ctypes.c_int, [ctypes.c_void_p]),
    "serial_emd_plan_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int,
                                                ctypes.POINTER(semd_instance), ctypes.c_void_p,
                                                ctypes.c_int, ctypes.POINTER(semd_tune_result),
                                                ctypes.c_void_p]),
    "serial_emd_tune_lookup": (ctypes.c_int, [ctypes.POINTER(semd_params), ctypes.c_int64,
                                              ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_int)]),
    "serial_emd_plan_set_pass_variant": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "serial_emd_plan_get_pass_variant": (ctypes.c_int, [ctypes.c_void_p]),
    "serial_emd_tune_clear": (None, []),
    "serial_emd_tune_save": (ctypes.c_int, [ctypes.c_char_p]),
    "serial_emd_tune_load": (ctypes.c_int, [ctypes.c_char_p]),
    "serial_emd_tune_last_error": (ctypes.c_char_p, []),
    "serial_emd_plan_set_options": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "serial_emd_plan_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(semd_stats)]),
    "serial_emd_plan_launch_times": (ctypes.c_int64, [ctypes.c_void_p, ctypes.c_int,
                                                      ctypes.POINTER(ctypes.c_float),
                                                      ctypes.c_int64]),
    "serial_emd_fma_rate": (ctypes.c_int, [ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "serial_emd_interface_solve_shape": (ctypes.c_int, [ctypes.c_int, ctypes.c_int,
                                                        ctypes.POINTER(ctypes.c_int),
                                                        ctypes.POINTER(ctypes.c_int64),
                                                        ctypes.POINTER(ctypes.c_int64)]),
    "serial_emd_destroy": (None, [ctypes.c_void_p]),
    "serial_emd_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "serial_emd_server_create": (ctypes.c_int, [ctypes.POINTER(semd_params), ctypes.c_size_t,
                                                ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "serial_emd_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(semd_request),
                                         ctypes.POINTER(ctypes.c_uint64)]),
    "serial_emd_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64,
                                       ctypes.POINTER(semd_result)]),
    "serial_emd_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_double,
                                       ctypes.POINTER(semd_result)]),
    "serial_emd_server_destroy": (None, [ctypes.c_void_p]),
    "serial_emd_server_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Loads the in-tree library (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libserial_emd.so not found at {path}; run build() first")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


# handle -> the plan's parameters, for the argument checks below
_PLAN_PARAMS: dict = {}

_TORCH_DTYPES = None


def _dtype_of(precision: int):
    global _TORCH_DTYPES
    if _TORCH_DTYPES is None:
        import torch
        _TORCH_DTYPES = {FP64: torch.float64, FP32_MIXED: torch.float32, "int32": torch.int32}
    return _TORCH_DTYPES[precision]


_NO_DEVICE = object()


def _current_device():
    """The current CUDA device index, or a marker when no device is present (the device
    check is then skipped: nothing can run anyway)."""
    import torch
    return torch.cuda.current_device() if torch.cuda.is_available() else _NO_DEVICE


def _need(t, what: str, dtype, numel: int | None = None, optional: bool = False, dev=None):
    """Refuses (SEMD_EINVAL, before any library call) a buffer the C ABI would read or write
    out of bounds or misinterpret: it must be a contiguous CUDA tensor on the current
    device, of the element type the call uses, with at least `numel` elements. dev: the
    current device, when the caller checks many tensors (looked up here otherwise)."""
    if t is None:
        if optional:
            return
        raise SemdError(SEMD_EINVAL, f"{what}: a CUDA tensor is required")
    if isinstance(t, int):  # a raw device pointer: the caller vouches for it
        return
    if not getattr(t, "is_cuda", False):
        raise SemdError(SEMD_EINVAL, f"{what}: not a CUDA tensor")
    if dev is None:
        dev = _current_device()
    if dev is not _NO_DEVICE and t.device.index != dev:
        raise SemdError(SEMD_EINVAL, f"{what}: on cuda:{t.device.index}, not on the current "
                                     f"device cuda:{dev}")
    if not t.is_contiguous():
        raise SemdError(SEMD_EINVAL, f"{what}: not contiguous")
    want = _dtype_of(dtype)
    if t.dtype is not want:
        raise SemdError(SEMD_EINVAL, f"{what}: dtype {t.dtype}, the call needs {want}")
    if numel is not None and t.numel() < numel:
        raise SemdError(SEMD_EINVAL, f"{what}: {t.numel()} elements, the call needs {numel}")


def _plan_precision(plan: int):
    p = _PLAN_PARAMS.get(plan)
    return p.precision if p is not None else None


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(rc: int, handle, err_fn="serial_emd_last_error"):
    if rc < 0:
        msg = getattr(load(), err_fn)(handle)
        raise SemdError(rc, msg.decode() if msg else "")
    return rc


# ------------------------------------------------------------------ C-named wrappers

def serial_emd_default_params(**overrides) -> semd_params:
    p = semd_params()
    load().serial_emd_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def serial_emd_plan(params: semd_params, max_batch: int = 1, mem_budget: int = 0) -> int:
    h = ctypes.c_void_p()
    rc = load().serial_emd_plan(ctypes.byref(params), max_batch, mem_budget, ctypes.byref(h))
    _check(rc, None)
    kept = semd_params()
    ctypes.pointer(kept)[0] = params
    _PLAN_PARAMS[h.value] = kept
    return h.value


def serial_emd_plan_bytes(plan: int) -> int:
    return int(load().serial_emd_plan_bytes(plan))


def _serial_len(p, rows: int, cols: int) -> int:
    M, N = (cols, rows) if p.order == ORDER_ROWS else (rows, cols)
    D = int(round(0.2 * M)) if p.transition_len < 0 else p.transition_len
    return M * N if N == 1 else M * N + D * N - D


def _need_decompose(plan: int, x, noise, imfs, residue, ensemble_needs_noise: bool):
    p = _PLAN_PARAMS.get(plan)
    if p is None:
        return
    rc = p.rows * p.cols
    _need(x, "x", p.precision, rc)
    _need(imfs, "imfs", p.precision, p.max_imfs * rc)
    _need(residue, "residue", FP64, rc, optional=True)
    if p.ensemble_trials > 1 and (ensemble_needs_noise or noise is not None):
        _need(noise, "noise", p.precision, p.ensemble_trials * _serial_len(p, p.rows, p.cols))


def serial_emd_decompose(plan: int, x, noise, imfs, residue, stream=None, wait: bool = True):
    """noise: the EEMD realizations, or None to let the library draw them (EEMD plans)."""
    _need_decompose(plan, x, noise, imfs, residue, False)
    n = ctypes.c_int(-1)
    rc = load().serial_emd_decompose(plan, _ptr(x), _ptr(noise), _ptr(imfs), _ptr(residue),
                                     ctypes.byref(n) if wait else None, _stream(stream))
    _check(rc, plan)
    return n.value if wait else None


def serial_emd_plan_set_noise_seed(plan: int, seed: int) -> None:
    _check(load().serial_emd_plan_set_noise_seed(plan, seed), plan)


_INSTANCE_DTYPE = None


def _instance_array(items, p):
    """The semd_instance array of a batch, built with vectorized numpy (a batch may hold
    thousands of inputs), after the per-item buffer checks."""
    global _INSTANCE_DTYPE
    import numpy as np
    if _INSTANCE_DTYPE is None:
        _INSTANCE_DTYPE = np.dtype([("x", "<u8"), ("rows", "<i8"), ("cols", "<i8"),
                                    ("imfs", "<u8"), ("res", "<u8")], align=True)
        assert _INSTANCE_DTYPE.itemsize == ctypes.sizeof(semd_instance)
    n = len(items)
    if p is not None:
        dev = _current_device()
        want, wres = _dtype_of(p.precision), _dtype_of(FP64)
        for i, (x, imfs, res) in enumerate(items):
            rc = x.shape[0] * x.shape[1]
            if isinstance(x, int) or isinstance(imfs, int) or not (
                    x.is_cuda and imfs.is_cuda and x.dtype is want and imfs.dtype is want
                    and x.is_contiguous() and imfs.is_contiguous()
                    and imfs.numel() >= p.max_imfs * rc
                    and (res is None or (res.is_cuda and res.dtype is wres
                                         and res.is_contiguous() and res.numel() >= rc))
                    and (i > 0 or dev is _NO_DEVICE or x.device.index == dev)):
                _need(x, "items[%d].x" % i, p.precision, rc, dev=dev)
                _need(imfs, "items[%d].imfs" % i, p.precision, p.max_imfs * rc, dev=dev)
                _need(res, "items[%d].residue" % i, FP64, rc, optional=True, dev=dev)
    a = np.zeros(n, _INSTANCE_DTYPE)
    a["x"] = [_ptr(x) for x, _, _ in items]
    a["rows"] = [x.shape[0] for x, _, _ in items]
    a["cols"] = [x.shape[1] for x, _, _ in items]
    a["imfs"] = [_ptr(m) for _, m, _ in items]
    a["res"] = [_ptr(r) or 0 for _, _, r in items]
    return a


def serial_emd_decompose_batch(plan: int, items, stream=None, wait: bool = True):
    """items: list of (x, imfs, residue) CUDA tensors, x 2D (rows, cols)."""
    a = _instance_array(items, _PLAN_PARAMS.get(plan))
    n = (ctypes.c_int * len(items))()
    rc = load().serial_emd_decompose_batch(
        plan, len(items), a.ctypes.data_as(ctypes.POINTER(semd_instance)), n if wait else None,
        _stream(stream))
    _check(rc, plan)
    return list(n) if wait else None


def _packed_instance_array(plan: int, x, shapes, imfs, residue):
    """The semd_instance array of a packed batch: instance i's (rows_i, cols_i) input at
    element offset o_i = sum of the earlier rows * cols in x, its K IMFs at K o_i in imfs
    and its residue at o_i in residue, with one buffer check per tensor."""
    global _INSTANCE_DTYPE
    import numpy as np
    p = _PLAN_PARAMS.get(plan)
    if p is None:
        raise SemdError(SEMD_EINVAL, "a packed batch needs a plan created by this binding")
    sh = np.asarray(shapes, dtype=np.int64).reshape(-1, 2)
    if sh.shape[0] < 1 or (sh < 1).any():
        raise SemdError(SEMD_EINVAL, "shapes: one (rows, cols) pair of positive sizes per input")
    size = sh[:, 0] * sh[:, 1]
    off = np.concatenate(([0], np.cumsum(size)[:-1]))
    total = int(size.sum())
    dev = _current_device()
    _need(x, "x", p.precision, total, dev=dev)
    _need(imfs, "imfs", p.precision, p.max_imfs * total, dev=dev)
    _need(residue, "residue", FP64, total, optional=True, dev=dev)
    if _INSTANCE_DTYPE is None:
        _INSTANCE_DTYPE = np.dtype([("x", "<u8"), ("rows", "<i8"), ("cols", "<i8"),
                                    ("imfs", "<u8"), ("res", "<u8")], align=True)
    elem = 8 if p.precision == FP64 else 4
    a = np.zeros(sh.shape[0], _INSTANCE_DTYPE)
    a["x"] = np.uint64(_ptr(x)) + (off * elem).astype(np.uint64)
    a["rows"] = sh[:, 0]
    a["cols"] = sh[:, 1]
    a["imfs"] = np.uint64(_ptr(imfs)) + (off * (p.max_imfs * elem)).astype(np.uint64)
    if residue is not None:
        a["res"] = np.uint64(_ptr(residue)) + (off * 8).astype(np.uint64)
    return a


def serial_emd_decompose_packed(plan: int, x, shapes, imfs, residue=None, stream=None,
                                wait: bool = True):
    """serial_emd_decompose_batch of inputs stored back to back in one tensor: x holds
    input i, (rows_i, cols_i) row-major, at element offset o_i (the sum of the earlier
    inputs' sizes); its K IMFs are written at K o_i in imfs (K x rows_i x cols_i) and its
    residue at o_i in residue. The per-input pointers are computed from the offsets, so a
    batch of thousands of inputs costs one buffer check per tensor instead of three per
    input."""
    a = _packed_instance_array(plan, x, shapes, imfs, residue)
    n = (ctypes.c_int * len(a))()
    rc = load().serial_emd_decompose_batch(
        plan, len(a), a.ctypes.data_as(ctypes.POINTER(semd_instance)), n if wait else None,
        _stream(stream))
    _check(rc, plan)
    return list(n) if wait else None


def serial_emd_decompose_slices(plan: int, x, imfs, residue, stream=None, wait: bool = True):
    """Slice-wise standard EMD of every row of x (rows, cols); imfs (K, rows, cols)."""
    rows, cols = x.shape
    p = _PLAN_PARAMS.get(plan)
    if p is not None:
        _need(x, "x", p.precision, rows * cols)
        _need(imfs, "imfs", p.precision, p.max_imfs * rows * cols)
        _need(residue, "residue", FP64, rows * cols, optional=True)
    n = (ctypes.c_int * rows)()
    rc = load().serial_emd_decompose_slices(plan, _ptr(x), rows, cols, _ptr(imfs), _ptr(residue),
                                            n if wait else None, _stream(stream))
    _check(rc, plan)
    return list(n) if wait else None


def serial_emd_ceemdan(plan: int, x, noise, modes, residue, stream=None, wait: bool = True):
    """Serial-CEEMDAN (Sec. 2.2 Steps 1-4 inside Sec. 3) of x with the noise (trials, L)."""
    _need_decompose(plan, x, noise, modes, residue, True)
    n = ctypes.c_int(-1)
    rc = load().serial_emd_ceemdan(plan, _ptr(x), _ptr(noise), _ptr(modes), _ptr(residue),
                                   ctypes.byref(n) if wait else None, _stream(stream))
    _check(rc, plan)
    return n.value if wait else None


def serial_emd_eemd_trial(plan: int, trial: int, imfs, residue=None, stream=None):
    """Realization `trial` of the plan's last EEMD call: fills imfs (K, rows, cols) and
    residue; returns (its IMF count, beta of the call)."""
    p = _PLAN_PARAMS.get(plan)
    if p is not None:
        _need(imfs, "imfs", p.precision, p.max_imfs * p.rows * p.cols)
        _need(residue, "residue", FP64, p.rows * p.cols, optional=True)
    n, beta = ctypes.c_int(-1), ctypes.c_double()
    rc = load().serial_emd_eemd_trial(plan, trial, _ptr(imfs), _ptr(residue), ctypes.byref(n),
                                      ctypes.byref(beta), _stream(stream))
    _check(rc, plan)
    return n.value, beta.value


def serial_emd_plan_counts(plan: int, count: int, max_imfs: int):
    n = (ctypes.c_int * count)()
    s = (ctypes.c_int * (count * max_imfs))()
    _check(load().serial_emd_plan_counts(plan, count, n, s), plan)
    return list(n), [list(s[i * max_imfs:(i + 1) * max_imfs]) for i in range(count)]


def serial_emd_extrema(plan: int, h, tmax, tmin, stream=None):
    prec = _plan_precision(plan)
    if prec is not None:
        _need(h, "h", prec)
        n = h.numel() // 2 + 1 if not isinstance(h, int) else None
        _need(tmax, "tmax", "int32", n)
        _need(tmin, "tmin", "int32", n)
    a, b = ctypes.c_int64(), ctypes.c_int64()
    rc = load().serial_emd_extrema(plan, _ptr(h), h.numel(), _ptr(tmax), _ptr(tmin),
                                   ctypes.byref(a), ctypes.byref(b), _stream(stream))
    _check(rc, plan)
    return a.value, b.value


def serial_emd_sift(plan: int, h, out, stream=None):
    prec = _plan_precision(plan)
    if prec is not None:
        _need(h, "h", prec)
        _need(out, "out", prec, h.numel())
    a, b = ctypes.c_double(), ctypes.c_double()
    rc = load().serial_emd_sift(plan, _ptr(h), h.numel(), _ptr(out), ctypes.byref(a),
                                ctypes.byref(b), _stream(stream))
    _check(rc, plan)
    return a.value, b.value


def serial_emd_sift_noalloc(params: semd_params, h, out, stream=None):
    """Allocation-free single sift (no plan); returns (sum (h - h')^2, sum h^2)."""
    if params.precision not in (FP64, FP32_MIXED):
        raise SemdError(SEMD_EINVAL, "precision must be FP64 or FP32_MIXED")
    _need(h, "h", params.precision)
    _need(out, "out", params.precision, h.numel())
    a, b = ctypes.c_double(), ctypes.c_double()
    rc = load().serial_emd_sift_noalloc(ctypes.byref(params), _ptr(h), h.numel(), _ptr(out),
                                        ctypes.byref(a), ctypes.byref(b), _stream(stream))
    _check(rc, None)
    return a.value, b.value


def serial_emd_plan_set_tile(plan: int, tile: int) -> None:
    _check(load().serial_emd_plan_set_tile(plan, tile), plan)


def serial_emd_plan_get_tile(plan: int) -> int:
    return int(load().serial_emd_plan_get_tile(plan))


def serial_emd_plan_set_options(plan: int, use_graphs: bool = True, profile: bool = False):
    _check(load().serial_emd_plan_set_options(plan, int(use_graphs), int(profile)), plan)


def serial_emd_plan_set_pass_ctas(plan: int, ctas_per_sm: int) -> None:
    _check(load().serial_emd_plan_set_pass_ctas(plan, ctas_per_sm), plan)


def serial_emd_plan_get_pass_ctas(plan: int) -> int:
    return int(load().serial_emd_plan_get_pass_ctas(plan))


def serial_emd_plan_autotune(plan: int, items, noise=None, repeats: int = 3,
                             stream=None) -> semd_tune_result:
    """Times every pass-kernel shape on the inputs (list of (x, imfs, residue) tensors,
    as decompose_batch takes them; one item plus noise for an ensemble plan), keeps the
    fastest on the plan and in the process-wide tuning table."""
    arr = (semd_instance * len(items))()
    for i, (x, imfs, res) in enumerate(items):
        arr[i] = semd_instance(_ptr(x), x.shape[0], x.shape[1], _ptr(imfs), _ptr(res))
    out = semd_tune_result()
    rc = load().serial_emd_plan_autotune(plan, len(items), arr, _ptr(noise), repeats,
                                         ctypes.byref(out), _stream(stream))
    _check(rc, plan)
    return out


def serial_emd_tune_lookup(params: semd_params, L: int, ninst: int):
    """(tile, ctas_per_sm, variant) of the tuning table's entry, or None."""
    t, c, v = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    rc = load().serial_emd_tune_lookup(ctypes.byref(params), L, ninst, ctypes.byref(t),
                                       ctypes.byref(c), ctypes.byref(v))
    if rc == SEMD_PENDING:
        return None
    if rc != 0:
        raise SemdError(rc, "bad arguments")
    return t.value, c.value, v.value


def serial_emd_plan_set_pass_variant(plan: int, variant: int) -> None:
    _check(load().serial_emd_plan_set_pass_variant(plan, variant), plan)


def serial_emd_plan_get_pass_variant(plan: int) -> int:
    return int(load().serial_emd_plan_get_pass_variant(plan))


def serial_emd_tune_clear() -> None:
    load().serial_emd_tune_clear()


def serial_emd_tune_save(path: str) -> None:
    rc = load().serial_emd_tune_save(path.encode())
    if rc != 0:
        raise SemdError(rc, load().serial_emd_tune_last_error().decode())


def serial_emd_tune_load(path: str) -> None:
    rc = load().serial_emd_tune_load(path.encode())
    if rc != 0:
        raise SemdError(rc, load().serial_emd_tune_last_error().decode())


def serial_emd_plan_stats(plan: int) -> semd_stats:
    st = semd_stats()
    _check(load().serial_emd_plan_stats(plan, ctypes.byref(st)), plan)
    return st


def serial_emd_plan_launch_times(plan: int, kind: int) -> list[float]:
    """Per-launch device times (ms) of the last profiled call: kind 0 passes, 1 solves."""
    n = int(load().serial_emd_plan_launch_times(plan, kind, None, 0))
    if n < 0:
        raise SemdError(SEMD_EINVAL, "bad plan or kind")
    buf = (ctypes.c_float * max(1, n))()
    load().serial_emd_plan_launch_times(plan, kind, buf, n)
    return list(buf[:n])


def serial_emd_fma_rate(precision: int, iters: int = 4096, stream=None) -> float:
    """Measured FMA throughput (GFLOP/s) of the current GPU in FP64 or FP32."""
    g = ctypes.c_double()
    rc = load().serial_emd_fma_rate(precision, iters, ctypes.byref(g), _stream(stream))
    if rc != 0:
        raise SemdError(rc, "fma rate probe failed")
    return g.value


def serial_emd_interface_solve_shape(precision: int, spline_end: int = 0) -> tuple:
    """(cluster CTAs per envelope, min tiles, max tiles) of the cluster interface solve on
    the current GPU; cluster 0 when it is not used."""
    c, lo, hi = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
    rc = load().serial_emd_interface_solve_shape(precision, spline_end, ctypes.byref(c),
                                                 ctypes.byref(lo), ctypes.byref(hi))
    if rc != 0:
        raise SemdError(rc, "interface solve shape query failed")
    return c.value, lo.value, hi.value


def serial_emd_destroy(plan: int) -> None:
    if plan:
        _PLAN_PARAMS.pop(plan, None)
        load().serial_emd_destroy(plan)


def serial_emd_last_error(plan) -> str:
    m = load().serial_emd_last_error(plan)
    return m.decode() if m else ""


def serial_emd_server_create(params: semd_params, mem_budget: int, max_inflight: int) -> int:
    h = ctypes.c_void_p()
    rc = load().serial_emd_server_create(ctypes.byref(params), mem_budget, max_inflight,
                                         ctypes.byref(h))
    if rc < 0:
        raise SemdError(rc, serial_emd_server_last_error(None))
    kept = semd_params()
    ctypes.pointer(kept)[0] = params
    _PLAN_PARAMS[("server", h.value)] = kept
    return h.value


def serial_emd_submit(server: int, x, imfs, residue, order: int = ORDER_ROWS) -> int:
    p = _PLAN_PARAMS.get(("server", server))
    if p is not None:
        rc = x.shape[0] * x.shape[1]
        _need(x, "x", p.precision, rc)
        _need(imfs, "imfs", p.precision, p.max_imfs * rc)
        _need(residue, "residue", FP64, rc, optional=True)
    req = semd_request(_ptr(x), x.shape[0], x.shape[1], order, 0, _ptr(imfs), _ptr(residue))
    t = ctypes.c_uint64()
    rc = load().serial_emd_submit(server, ctypes.byref(req), ctypes.byref(t))
    _check(rc, server, "serial_emd_server_last_error")
    return t.value


def serial_emd_poll(server: int, ticket: int):
    """Returns None while pending, else the semd_result."""
    r = semd_result()
    rc = load().serial_emd_poll(server, ticket, ctypes.byref(r))
    if rc == SEMD_PENDING:
        return None
    _check(rc, server, "serial_emd_server_last_error")
    return r


def serial_emd_wait(server: int, ticket: int, timeout_ms: float):
    """Waits up to timeout_ms for the request; returns its semd_result, or None when the
    limit ran out (SEMD_ETIMEOUT: the request is still pending)."""
    r = semd_result()
    rc = load().serial_emd_wait(server, ticket, float(timeout_ms), ctypes.byref(r))
    if rc == SEMD_ETIMEOUT:
        return None
    _check(rc, server, "serial_emd_server_last_error")
    return r


def serial_emd_server_destroy(server: int) -> None:
    if server:
        _PLAN_PARAMS.pop(("server", server), None)
        load().serial_emd_server_destroy(server)


def serial_emd_server_last_error(server) -> str:
    m = load().serial_emd_server_last_error(server)
    return m.decode() if m else ""
