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
                ("lanes_per_row", c_int32), ("index_width", c_int32), ("class_table", c_int32),
                ("reserved", c_int32), ("cuda_stream", c_void_p)]


class fw_seg_forms(ctypes.Structure):
    _fields_ = [("lanes_per_row", c_int32), ("index_width", c_int32), ("class_table", c_int32),
                ("table_blocks", c_int32), ("tiles", c_int32), ("tile_rows", c_int32),
                ("kmax", c_int32), ("reserved", c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class fw_seg_stats(ctypes.Structure):
    _fields_ = [("iters", c_int32), ("status", c_int32), ("active_rows", c_int32),
                ("launches", c_int32), ("gap", c_double), ("gap0", c_double), ("q", c_double),
                ("alpha", c_double), ("objective", c_double), ("ms", c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class fw_graph(ctypes.Structure):
    _fields_ = [("n", c_int64), ("row_ptr_host", c_void_p), ("col_host", c_void_p),
                ("w_host", c_void_p), ("K", c_int32), ("reserved", c_int32),
                ("labels_host", c_void_p)]


class fw_batch_opts(ctypes.Structure):
    _fields_ = [("weight_dtype", c_int32), ("blocks_per_sm", c_int32), ("schedule", c_int32),
                ("iters_per_launch", c_int32), ("use_graph", c_int32),
                ("spin_budget_ms", c_int32), ("test_barrier_extra", c_int32),
                ("lanes_per_row", c_int32), ("tune_cache", ctypes.c_char_p),
                ("cuda_stream", c_void_p)]


class fw_batch_info(ctypes.Structure):
    _fields_ = [("grid", c_int32), ("blocks_per_sm", c_int32), ("schedule", c_int32),
                ("graph_captured", c_int32), ("tuned", c_int32), ("kmax", c_int32),
                ("lanes_per_row", c_int32), ("iters_per_launch", c_int32),
                ("graph_error", c_int32), ("reserved", c_int32),
                ("tune_ms", c_double), ("pool_bytes", c_size_t)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class fw_srv_opts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", c_size_t), ("max_slots", c_int32), ("max_K", c_int32),
                ("weight_dtype", c_int32), ("iters_per_epoch", c_int32),
                ("blocks_per_sm", c_int32), ("schedule", c_int32), ("spin_budget_ms", c_int32),
                ("reserved", c_int32), ("cuda_stream", c_void_p)]


class fw_srv_info(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64),
                ("rejected", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("epochs", ctypes.c_uint64),
                ("resident", c_int32), ("queued", c_int32), ("pool_bytes", c_size_t),
                ("pool_used", c_size_t)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


SCHED = {"auto": 0, "static": 1, "dynamic": 2, "items": 3}
TABLE = {"auto": 0, "off": 1, "on": 2}
GRAPH = {"off": 0, "required": 1, "preferred": 2}

_lib = None

_SIGS = {
    "fw_seg_last_error": (ctypes.c_char_p, []),
    "fw_seg_default_opts": (c_int32, [POINTER(fw_seg_opts)]),
    "fw_seg_footprint": (c_size_t, [c_int64, c_int64, c_int32, c_int32]),
    "fw_seg_create": (c_int32, [POINTER(c_void_p), c_int64, c_void_p, c_void_p, c_void_p, c_int32,
                                c_void_p, POINTER(fw_seg_opts)]),
    "fw_seg_solve": (c_int32, [c_void_p, POINTER(fw_seg_stats)]),
    "fw_seg_get_forms": (c_int32, [c_void_p, POINTER(fw_seg_forms)]),
    "fw_seg_step": (c_int32, [c_void_p, c_int32, POINTER(fw_seg_stats)]),
    "fw_seg_labels": (c_int32, [c_void_p, c_void_p]),
    "fw_seg_oneshot": (c_int32, [c_void_p, c_void_p, POINTER(c_double)]),
    "fw_seg_get_U": (c_int32, [c_void_p, c_void_p]),
    "fw_seg_set_U": (c_int32, [c_void_p, c_void_p]),
    "fw_seg_get_grad": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "fw_seg_objective": (c_int32, [c_void_p, POINTER(c_double)]),
    "fw_seg_refresh": (c_int32, [c_void_p]),
    "fw_seg_lmo_gap": (c_int32, [c_void_p, POINTER(c_double)]),
    "fw_seg_get_stats": (c_int32, [c_void_p, POINTER(fw_seg_stats)]),
    "fw_seg_reset": (c_int32, [c_void_p]),
    "fw_seg_profile": (c_int32, [c_void_p, c_int32, POINTER(c_double), POINTER(c_double),
                                 POINTER(c_double), POINTER(c_double), POINTER(c_int32)]),
    "fw_seg_destroy": (None, [c_void_p]),
    "fw_batch_default_opts": (c_int32, [POINTER(fw_batch_opts)]),
    "fw_batch_create": (c_int32, [POINTER(c_void_p), c_int32, POINTER(fw_graph),
                                  POINTER(fw_seg_opts), POINTER(fw_batch_opts)]),
    "fw_batch_solve": (c_int32, [c_void_p, POINTER(fw_seg_stats)]),
    "fw_batch_reset": (c_int32, [c_void_p]),
    "fw_batch_labels": (c_int32, [c_void_p, c_int32, c_void_p]),
    "fw_batch_get_U": (c_int32, [c_void_p, c_int32, c_void_p]),
    "fw_batch_get_info": (c_int32, [c_void_p, POINTER(fw_batch_info)]),
    "fw_batch_destroy": (None, [c_void_p]),
    "fw_srv_default_opts": (c_int32, [POINTER(fw_srv_opts)]),
    "fw_srv_create": (c_int32, [POINTER(c_void_p), POINTER(fw_srv_opts)]),
    "fw_srv_submit": (c_int32, [c_void_p, POINTER(fw_graph), POINTER(fw_seg_opts),
                                POINTER(ctypes.c_uint64)]),
    "fw_srv_poll": (c_int32, [c_void_p, ctypes.c_uint64, c_void_p, POINTER(fw_seg_stats)]),
    "fw_srv_wait": (c_int32, [c_void_p, ctypes.c_uint64, c_int32, c_void_p,
                              POINTER(fw_seg_stats)]),
    "fw_srv_wait_any": (c_int32, [c_void_p, c_int32, POINTER(ctypes.c_uint64)]),
    "fw_srv_get_info": (c_int32, [c_void_p, POINTER(fw_srv_info)]),
    "fw_srv_destroy": (None, [c_void_p]),
    "fw_energy_noalloc": (c_int32, [c_int64, c_int32, c_void_p, c_void_p, c_void_p, c_int64,
                                    c_void_p, c_int64, c_void_p, c_double, c_double, c_int32,
                                    c_void_p, POINTER(c_double)]),
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
    ('exact','armijo'), tol_mode ('abs','rel') and class_table
    ('auto','off','on')."""
    o = fw_seg_opts()
    _check(lib().fw_seg_default_opts(ctypes.byref(o)))
    maps = dict(weight_dtype=WEIGHTS, laplacian=LAPLACIAN, oracle=ORACLE, step_rule=STEP,
                tol_mode=TOL, class_table=TABLE)
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


def fw_seg_oneshot(h: Handle, with_labels: bool = True):
    """One-Shot Frank-Wolfe labels (Alg. 4) and the kernel's device ms."""
    out = np.empty(h.n, dtype=np.int32) if with_labels else None
    ms = c_double()
    _check(lib().fw_seg_oneshot(h.ptr, _ptr(out), ctypes.byref(ms)))
    return out, ms.value


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


def fw_seg_lmo_gap(h: Handle) -> float:
    """Classic (full-LMO) FW gap at the current iterate (stationarity measure)."""
    g = c_double()
    _check(lib().fw_seg_lmo_gap(h.ptr, ctypes.byref(g)))
    return g.value


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


def fw_seg_get_forms(h: Handle) -> fw_seg_forms:
    f = fw_seg_forms()
    _check(lib().fw_seg_get_forms(h.ptr, ctypes.byref(f)))
    return f


def fw_seg_reset(h: Handle) -> None:
    _check(lib().fw_seg_reset(h.ptr))


def fw_seg_profile(h: Handle, iters: int) -> dict:
    """Device ms of the iteration kernels as the solve runs them: per
    iteration of a graph of `iters` fused iterations (per_iter), per launch of
    graphs of `iters` back-to-back launches of pass A (pass_a) and of pass B
    (pass_b), and one finishing kernel (finish); in_graph = 0 when the stream
    could not be captured.  The iterate advances by iters + 1 iterations."""
    a, b, f, t = c_double(), c_double(), c_double(), c_double()
    g = c_int32()
    _check(lib().fw_seg_profile(h.ptr, int(iters), ctypes.byref(a), ctypes.byref(b),
                                ctypes.byref(f), ctypes.byref(t), ctypes.byref(g)))
    return dict(pass_a=a.value, pass_b=b.value, finish=f.value, per_iter=t.value,
                in_graph=int(g.value))


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

    def oneshot(self, with_labels=True):
        """(labels, kernel ms) of One-Shot Frank-Wolfe (Alg. 4) from U_hat."""
        return fw_seg_oneshot(self.h, with_labels)

    def labels(self):
        return fw_seg_labels(self.h)

    def U(self):
        return fw_seg_get_U(self.h)

    def set_U(self, U):
        fw_seg_set_U(self.h, U)

    def grad(self):
        return fw_seg_get_grad(self.h)

    def lmo_gap(self):
        return fw_seg_lmo_gap(self.h)

    def objective(self):
        return fw_seg_objective(self.h)

    def stats(self):
        return fw_seg_get_stats(self.h)

    def forms(self):
        return fw_seg_get_forms(self.h)

    def refresh(self):
        fw_seg_refresh(self.h)

    def reset(self):
        fw_seg_reset(self.h)

    def profile(self, iters):
        return fw_seg_profile(self.h, iters)


# ------------------------------------------------------------------ batches --

def _graph_struct(g, keep: list) -> fw_graph:
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int32)
    cl = np.ascontiguousarray(g.col, dtype=np.int32)
    ww = np.ascontiguousarray(g.w, dtype=np.float64)
    lb = np.ascontiguousarray(g.labels, dtype=np.int32)
    keep += [rp, cl, ww, lb]
    return fw_graph(int(g.n), rp.ctypes.data, cl.ctypes.data, ww.ctypes.data, int(g.K), 0,
                    lb.ctypes.data)


def fw_batch_default_opts(**kw) -> fw_batch_opts:
    o = fw_batch_opts()
    _check(lib().fw_batch_default_opts(ctypes.byref(o)))
    for k, v in kw.items():
        if k == "weight_dtype" and isinstance(v, str):
            v = WEIGHTS[v]
        if k == "schedule" and isinstance(v, str):
            v = SCHED[v]
        if k == "use_graph" and isinstance(v, str):
            v = GRAPH[v]
        if k == "tune_cache" and isinstance(v, str):
            v = v.encode()
        if k == "cuda_stream" and v is not None and not isinstance(v, int):
            v = int(getattr(v, "cuda_stream", v))
        setattr(o, k, v)
    return o


class BatchHandle:
    def __init__(self, ptr, graphs):
        self.ptr = ptr
        self.sizes = [(int(g.n), int(g.K)) for g in graphs]


def fw_batch_create(graphs, opts, bopts: fw_batch_opts = None) -> BatchHandle:
    """graphs: sequence of Graph-like objects; opts: one fw_seg_opts or one per graph."""
    P = len(graphs)
    keep = []
    garr = (fw_graph * P)(*[_graph_struct(g, keep) for g in graphs])
    if isinstance(opts, fw_seg_opts):
        opts = [opts] * P
    oarr = (fw_seg_opts * P)(*opts)
    out = c_void_p()
    _check(lib().fw_batch_create(ctypes.byref(out), P, garr, oarr,
                                 ctypes.byref(bopts) if bopts is not None else None))
    return BatchHandle(out, graphs)


def fw_batch_solve(b: BatchHandle):
    P = len(b.sizes)
    st = (fw_seg_stats * P)()
    _check(lib().fw_batch_solve(b.ptr, st))
    return list(st)


def fw_batch_reset(b: BatchHandle) -> None:
    _check(lib().fw_batch_reset(b.ptr))


def fw_batch_labels(b: BatchHandle, p: int) -> np.ndarray:
    out = np.empty(b.sizes[p][0], dtype=np.int32)
    _check(lib().fw_batch_labels(b.ptr, int(p), _ptr(out)))
    return out


def fw_batch_get_U(b: BatchHandle, p: int) -> np.ndarray:
    n, K = b.sizes[p]
    U = np.empty((n, K), dtype=np.float64)
    _check(lib().fw_batch_get_U(b.ptr, int(p), _ptr(U)))
    return U


def fw_batch_get_info(b: BatchHandle) -> fw_batch_info:
    i = fw_batch_info()
    _check(lib().fw_batch_get_info(b.ptr, ctypes.byref(i)))
    return i


def fw_batch_destroy(b: BatchHandle) -> None:
    if b and b.ptr:
        lib().fw_batch_destroy(b.ptr)
        b.ptr = c_void_p()


class Batch:
    """Context-managed batch of independent problems, iterated together
    (per-item launches or one persistent launch, autotuned)."""

    def __init__(self, graphs, opts=None, **bopts):
        if opts is None:
            opts = fw_seg_default_opts()
        elif isinstance(opts, dict):
            opts = fw_seg_default_opts(**opts)
        elif isinstance(opts, (list, tuple)):
            opts = [fw_seg_default_opts(**o) if isinstance(o, dict) else o for o in opts]
        self.b = fw_batch_create(graphs, opts, fw_batch_default_opts(**bopts))

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def close(self):
        fw_batch_destroy(self.b)

    def solve(self):
        return fw_batch_solve(self.b)

    def reset(self):
        fw_batch_reset(self.b)

    def labels(self, p):
        return fw_batch_labels(self.b, p)

    def U(self, p):
        return fw_batch_get_U(self.b, p)

    def info(self):
        return fw_batch_get_info(self.b)


# ------------------------------------------------------------------ serving --

def fw_srv_default_opts(**kw) -> fw_srv_opts:
    o = fw_srv_opts()
    _check(lib().fw_srv_default_opts(ctypes.byref(o)))
    for k, v in kw.items():
        if k == "weight_dtype" and isinstance(v, str):
            v = WEIGHTS[v]
        if k == "schedule" and isinstance(v, str):
            v = SCHED[v]
        if k == "use_graph" and isinstance(v, str):
            v = GRAPH[v]
        if k == "cuda_stream" and v is not None and not isinstance(v, int):
            v = int(getattr(v, "cuda_stream", v))
        setattr(o, k, v)
    return o


def fw_srv_create(opts: fw_srv_opts = None):
    out = c_void_p()
    _check(lib().fw_srv_create(ctypes.byref(out), ctypes.byref(opts) if opts is not None else None))
    return out


def fw_srv_submit(s, g, opts: fw_seg_opts = None) -> int:
    keep = []
    gs = _graph_struct(g, keep)
    t = ctypes.c_uint64()
    _check(lib().fw_srv_submit(s, ctypes.byref(gs), ctypes.byref(opts) if opts is not None else None,
                               ctypes.byref(t)))
    return int(t.value)


def fw_srv_poll(s, ticket: int, n: int):
    """(status, labels or None, stats); status FW_PENDING while not finished."""
    lab = np.empty(n, dtype=np.int32)
    st = fw_seg_stats()
    rc = lib().fw_srv_poll(s, ctypes.c_uint64(ticket), _ptr(lab), ctypes.byref(st))
    if rc == FW_PENDING:
        return rc, None, None
    return rc, lab, st


def fw_srv_wait(s, ticket: int, n: int, timeout_ms: int = -1):
    lab = np.empty(n, dtype=np.int32)
    st = fw_seg_stats()
    rc = lib().fw_srv_wait(s, ctypes.c_uint64(ticket), int(timeout_ms), _ptr(lab), ctypes.byref(st))
    if rc == FW_PENDING:
        return rc, None, None
    return rc, lab, st


def fw_srv_wait_any(s, timeout_ms: int = -1):
    """(FW_OK, ticket) of a finished request not reported before, or
    (FW_PENDING, None) when timeout_ms ran out."""
    t = ctypes.c_uint64()
    rc = _check(lib().fw_srv_wait_any(s, int(timeout_ms), ctypes.byref(t)))
    return (rc, int(t.value)) if rc == FW_OK else (rc, None)


def fw_srv_get_info(s) -> fw_srv_info:
    i = fw_srv_info()
    _check(lib().fw_srv_get_info(s, ctypes.byref(i)))
    return i


def fw_srv_destroy(s) -> None:
    if s:
        lib().fw_srv_destroy(s)


class Server:
    """Context-managed continuous-batching server."""

    def __init__(self, **opts):
        self.s = fw_srv_create(fw_srv_default_opts(**opts))

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def close(self):
        if self.s:
            fw_srv_destroy(self.s)
            self.s = None

    def submit(self, g, **opts) -> int:
        return fw_srv_submit(self.s, g, fw_seg_default_opts(**opts))

    def poll(self, ticket, n):
        return fw_srv_poll(self.s, ticket, n)

    def wait(self, ticket, n, timeout_ms=-1):
        return fw_srv_wait(self.s, ticket, n, timeout_ms)

    def wait_any(self, timeout_ms=-1):
        return fw_srv_wait_any(self.s, timeout_ms)

    def info(self):
        return fw_srv_get_info(self.s)


# ------------------------------------------------- allocation-free energy --

FW_NOALLOC_MAX_N = 1048576


def fw_energy_noalloc(n, K, row_ptr_dev, col_dev, w_dev, nnz, U_dev, ldu, labels_dev, eps,
                      omega0, laplacian="sym", cuda_stream=None) -> float:
    """E(U) for a graph and iterate already on the device (integer device
    addresses, e.g. ``tensor.data_ptr()``; labels_dev may be 0/None)."""
    lap = LAPLACIAN[laplacian] if isinstance(laplacian, str) else int(laplacian)
    if cuda_stream is not None and not isinstance(cuda_stream, int):
        cuda_stream = int(getattr(cuda_stream, "cuda_stream", cuda_stream))
    E = c_double()
    _check(lib().fw_energy_noalloc(int(n), int(K), c_void_p(row_ptr_dev), c_void_p(col_dev),
                                   c_void_p(w_dev), int(nnz), c_void_p(U_dev), int(ldu),
                                   c_void_p(labels_dev or None), float(eps), float(omega0), lap,
                                   c_void_p(cuda_stream or None), ctypes.byref(E)))
    return E.value
