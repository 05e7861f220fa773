"""Thin ctypes binding of the C ABI in include/fw_seg.h.

Functions carry the C names and only marshal arguments: numpy arrays become
host pointers, results come back as numpy arrays.  Every step of the
segmentation runs in the CUDA library; there is no Python or CPU fallback --
a missing library raises `FwError` at the first call.
"""
from __future__ import annotations

import ctypes
import math
import os
from ctypes import POINTER, c_double, c_int32, c_int64, c_size_t, c_uint8, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libfwseg.so")

FW_OK, FW_NOT_CONVERGED, FW_PENDING = 0, 1, 2
FW_ERR_INVALID_ARG, FW_ERR_GRAPH, FW_ERR_ISOLATED, FW_ERR_NO_MEMORY = -1, -2, -3, -4
FW_ERR_CUDA, FW_ERR_NUMERIC, FW_ERR_TIMEOUT, FW_ERR_UNSUPPORTED = -5, -6, -7, -8
WEIGHTS = {"f32": 0, "bf16": 1, "f64": 2}
LAPLACIAN = {"sym": 0, "comb": 1}
ORACLE = {"greedy": 0, "full": 1}
STEP = {"exact": 0, "armijo": 1}
TOL = {"abs": 0, "rel": 1}


class FwError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"fw status {status}: {msg}")
        self.status = status


class fw_seg_opts(ctypes.Structure):
    _fields_ = [("eps", c_double), ("omega0", c_double), ("gap_tol", c_double),
                ("max_iters", c_int32), ("tol_mode", c_int32), ("weight_dtype", c_int32),
                ("laplacian", c_int32), ("oracle", c_int32), ("step_rule", c_int32),
                ("refresh_every", c_int32), ("iters_per_launch", c_int32),
                ("lanes_per_row", c_int32), ("reserved", c_int32), ("cuda_stream", c_void_p)]


class fw_seg_stats(ctypes.Structure):
    _fields_ = [("iters", c_int32), ("status", c_int32), ("active_rows", c_int32),
                ("launches", c_int32), ("gap", c_double), ("gap0", c_double), ("q", c_double),
                ("alpha", c_double), ("objective", c_double), ("ms", c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None

_SIGS = {
    "fw_seg_last_error": (ctypes.c_char_p, []),
    "fw_seg_default_opts": (c_int32, [POINTER(fw_seg_opts)]),
    "fw_seg_footprint": (c_size_t, [c_int64, c_int64, c_int32, c_int32]),
    "fw_seg_create": (c_int32, [POINTER(c_void_p), c_int64, c_void_p, c_void_p, c_void_p, c_int32,
                                c_void_p, POINTER(fw_seg_opts)]),
    "fw_seg_solve": (c_int32, [c_void_p, POINTER(fw_seg_stats)]),
    "fw_seg_step": (c_int32, [c_void_p, c_int32, POINTER(fw_seg_stats)]),
    "fw_seg_labels": (c_int32, [c_void_p, c_void_p]),
    "fw_seg_get_U": (c_int32, [c_void_p, c_void_p]),
    "fw_seg_set_U": (c_int32, [c_void_p, c_void_p]),
    "fw_seg_get_grad": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "fw_seg_objective": (c_int32, [c_void_p, POINTER(c_double)]),
    "fw_seg_refresh": (c_int32, [c_void_p]),
    "fw_seg_get_stats": (c_int32, [c_void_p, POINTER(fw_seg_stats)]),
    "fw_seg_reset": (c_int32, [c_void_p]),
    "fw_seg_profile": (c_int32, [c_void_p, c_int32, POINTER(c_double), POINTER(c_double)]),
    "fw_seg_destroy": (None, [c_void_p]),
}

# symbols every build of the library must export (checked by the CPU tests)
EXPORTED = list(_SIGS)


def lib():
    """The loaded CUDA library (raises FwError if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise FwError(FW_ERR_CUDA, f"CUDA library missing at {LIB_PATH}; "
                          "build it with paper_2508_09738_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int) -> int:
    if status < 0:
        raise FwError(status, fw_seg_last_error())
    return status


def _ptr(a):
    return c_void_p(a.ctypes.data) if a is not None else None


def fw_seg_last_error() -> str:
    return lib().fw_seg_last_error().decode()


def fw_seg_default_opts(**kw) -> fw_seg_opts:
    """Default options (eps 50, omega0 1000, ...) with keyword overrides.

    String values are accepted for weight_dtype ('f32','bf16','f64'),
    laplacian ('sym','comb'), oracle ('greedy','full'), step_rule
    ('exact','armijo') and tol_mode ('abs','rel')."""
    o = fw_seg_opts()
    _check(lib().fw_seg_default_opts(ctypes.byref(o)))
    maps = dict(weight_dtype=WEIGHTS, laplacian=LAPLACIAN, oracle=ORACLE, step_rule=STEP,
                tol_mode=TOL)
    for k, v in kw.items():
        if k in maps and isinstance(v, str):
            v = maps[k][v]
        if k == "cuda_stream" and v is not None and not isinstance(v, int):
            v = int(getattr(v, "cuda_stream", v))
        setattr(o, k, v)
    return o


def fw_seg_footprint(n: int, nnz: int, K: int, weight_dtype="f32") -> int:
    wd = WEIGHTS[weight_dtype] if isinstance(weight_dtype, str) else weight_dtype
    return int(lib().fw_seg_footprint(n, nnz, K, wd))


class Handle:
    """An fw_seg* plus the sizes the binding needs to shape outputs."""

    def __init__(self, ptr: c_void_p, n: int, K: int):
        self.ptr, self.n, self.K = ptr, n, K

    def __bool__(self):
        return bool(self.ptr)


def fw_seg_create(n, row_ptr, col, w, K, labels, opts: fw_seg_opts = None) -> Handle:
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    ww = np.ascontiguousarray(w, dtype=np.float64)
    lb = np.ascontiguousarray(labels, dtype=np.int32)
    out = c_void_p()
    _check(lib().fw_seg_create(ctypes.byref(out), int(n), _ptr(rp), _ptr(cl), _ptr(ww), int(K),
                               _ptr(lb), ctypes.byref(opts) if opts is not None else None))
    return Handle(out, int(n), int(K))


def fw_seg_solve(h: Handle) -> fw_seg_stats:
    s = fw_seg_stats()
    s.status = _check(lib().fw_seg_solve(h.ptr, ctypes.byref(s)))
    return s


def fw_seg_step(h: Handle, iters: int) -> fw_seg_stats:
    s = fw_seg_stats()
    _check(lib().fw_seg_step(h.ptr, int(iters), ctypes.byref(s)))
    return s


def fw_seg_labels(h: Handle, out: np.ndarray = None) -> np.ndarray:
    if out is None:
        out = np.empty(h.n, dtype=np.int32)
    _check(lib().fw_seg_labels(h.ptr, _ptr(out)))
    return out


def fw_seg_get_U(h: Handle) -> np.ndarray:
    U = np.empty((h.n, h.K), dtype=np.float64)
    _check(lib().fw_seg_get_U(h.ptr, _ptr(U)))
    return U


def fw_seg_set_U(h: Handle, U) -> None:
    U = np.ascontiguousarray(U, dtype=np.float64)
    assert U.shape == (h.n, h.K)
    _check(lib().fw_seg_set_U(h.ptr, _ptr(U)))


def fw_seg_get_grad(h: Handle):
    """(G', choice, active) at the current iterate, as the kernels compute them."""
    G = np.empty((h.n, h.K), dtype=np.float64)
    ch = np.empty(h.n, dtype=np.int32)
    act = np.empty(h.n, dtype=np.uint8)
    _check(lib().fw_seg_get_grad(h.ptr, _ptr(G), _ptr(ch), _ptr(act)))
    return G, ch, act.astype(bool)


def fw_seg_objective(h: Handle) -> float:
    E = c_double()
    _check(lib().fw_seg_objective(h.ptr, ctypes.byref(E)))
    return E.value


def fw_seg_refresh(h: Handle) -> None:
    _check(lib().fw_seg_refresh(h.ptr))


def fw_seg_get_stats(h: Handle) -> fw_seg_stats:
    s = fw_seg_stats()
    _check(lib().fw_seg_get_stats(h.ptr, ctypes.byref(s)))
    return s


def fw_seg_reset(h: Handle) -> None:
    _check(lib().fw_seg_reset(h.ptr))


def fw_seg_profile(h: Handle, iters: int):
    """Mean device ms of (pass A, pass B) over `iters` separately launched iterations."""
    a, b = c_double(), c_double()
    _check(lib().fw_seg_profile(h.ptr, int(iters), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def fw_seg_destroy(h: Handle) -> None:
    if h and h.ptr:
        lib().fw_seg_destroy(h.ptr)
        h.ptr = c_void_p()


class Segmenter:
    """Context-managed handle for a `workloads.Graph`-like object."""

    def __init__(self, g, **opts):
        self.g = g
        self.opts = fw_seg_default_opts(**opts)
        self.h = fw_seg_create(g.n, g.row_ptr, g.col, g.w, g.K, g.labels, self.opts)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def close(self):
        fw_seg_destroy(self.h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self):
        return fw_seg_solve(self.h)

    def step(self, iters=1):
        return fw_seg_step(self.h, iters)

    def labels(self):
        return fw_seg_labels(self.h)

    def U(self):
        return fw_seg_get_U(self.h)

    def set_U(self, U):
        fw_seg_set_U(self.h, U)

    def grad(self):
        return fw_seg_get_grad(self.h)

    def objective(self):
        return fw_seg_objective(self.h)

    def stats(self):
        return fw_seg_get_stats(self.h)

    def refresh(self):
        fw_seg_refresh(self.h)

    def reset(self):
        fw_seg_reset(self.h)

    def profile(self, iters):
        return fw_seg_profile(self.h, iters)
