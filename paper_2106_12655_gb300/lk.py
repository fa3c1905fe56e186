"""Python binding of the C ABI in ``include/lk.h`` (argument marshalling only).

Every function has the C name and forwards to ``_build/liblk.so``; all of the
linking-number work runs in that library's CUDA kernels.  Arrays may be numpy
arrays (host memory) or torch tensors (host or CUDA memory); pointers are
passed through unchanged.  There is no fallback: if the library is missing,
loading it raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LK_OK = 0
LK_ERR_ARG = 1
LK_ERR_ZERO_SEGMENT = 2
LK_ERR_INTERSECT = 3
LK_ERR_NONINTEGER = 4
LK_ERR_OOM = 5
LK_ERR_TIMEOUT = 6
LK_ERR_CUDA = 7
LK_ERR_BUSY = 8
LK_F32 = 0
LK_F64 = 1
LK_MIXED = 0
LK_ALL_F64 = 1
LK_METHOD_DS = 0
LK_METHOD_CC = 1
LK_CC_SEARCH_AUTO = 0
LK_CC_SEARCH_SWEEP = 1
LK_CC_SEARCH_BINNED = 2

STATUS_NAMES = {0: "LK_OK", 1: "LK_ERR_ARG", 2: "LK_ERR_ZERO_SEGMENT", 3: "LK_ERR_INTERSECT",
                4: "LK_ERR_NONINTEGER", 5: "LK_ERR_OOM", 6: "LK_ERR_TIMEOUT", 7: "LK_ERR_CUDA",
                8: "LK_ERR_BUSY"}

EXPORTED = ["lk_default_options", "lk_create", "lk_update", "lk_verify", "lk_sync", "lk_get_stats", "lk_get_options",
            "lk_destroy", "lk_last_error", "lk_plan_create", "lk_plan_run", "lk_plan_destroy",
            "lk_verify_noalloc", "lk_verify_expected", "lk_autotune", "lk_tune_get", "lk_tune_set", "lk_server_default_options", "lk_server_create", "lk_server_stream",
            "lk_server_submit", "lk_server_submit_geometry", "lk_server_step", "lk_server_poll",
            "lk_server_poll_pairs", "lk_server_completed", "lk_measure_fp32_peak",
            "lk_server_get_stats", "lk_server_last_error", "lk_server_destroy", "lk_candidates"]


class lk_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("near_ratio", ctypes.c_double),
                ("int_tol", ctypes.c_double), ("mem_budget", ctypes.c_size_t),
                ("tile_rows", ctypes.c_int), ("near_capacity", ctypes.c_int),
                ("timing", ctypes.c_int), ("chunk_capacity", ctypes.c_int),
                ("accurate_threshold", ctypes.c_int64), ("method", ctypes.c_int),
                ("cc_capacity", ctypes.c_int), ("cc_search", ctypes.c_int), ("precise_tol", ctypes.c_double)]


class lk_stats(ctypes.Structure):
    _fields_ = [("n_pairs", ctypes.c_int64), ("n_items", ctypes.c_int64),
                ("segment_pairs", ctypes.c_int64), ("fp64_pairs", ctypes.c_int64),
                ("near_overflow", ctypes.c_int64), ("tile_rows", ctypes.c_int32),
                ("tile_cols", ctypes.c_int32), ("careful_items", ctypes.c_int64),
                ("sweep_ms", ctypes.c_double), ("careful_chunks", ctypes.c_int64),
                ("cc_candidates", ctypes.c_int64), ("cc_fallback_pairs", ctypes.c_int64),
                ("precise_pairs", ctypes.c_int64)]


class lk_server_options(ctypes.Structure):
    _fields_ = [("max_requests", ctypes.c_int), ("arena_bytes", ctypes.c_size_t),
                ("host_bytes", ctypes.c_size_t), ("wave_items", ctypes.c_int64),
                ("near_capacity", ctypes.c_int), ("max_queue", ctypes.c_int), ("wave_order", ctypes.c_int),
                ("pack_on_device", ctypes.c_int)]


class lk_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "admitted", "completed", "queued", "running",
                                               "waves", "waves_in_flight", "items_launched",
                                               "max_requests_per_wave", "arena_used", "near_overflow",
                                               "careful_items", "careful_chunks", "geometry_requests",
                                               "candidate_pairs")]


class LkError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load liblk.so (built by ``build.build()``); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise ImportError("liblk.so not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    vp, i64, i32p = ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p
    lib.lk_default_options.restype = None
    lib.lk_default_options.argtypes = [ctypes.POINTER(lk_options)]
    lib.lk_create.restype = ctypes.c_int
    lib.lk_create.argtypes = [ctypes.POINTER(vp), vp, ctypes.c_int, i64, vp, i64,
                              ctypes.POINTER(lk_options), vp]
    lib.lk_update.restype = ctypes.c_int
    lib.lk_update.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, vp]
    lib.lk_verify.restype = ctypes.c_int
    lib.lk_verify.argtypes = [vp, i32p, i64, vp, vp, vp, vp]
    lib.lk_sync.restype = ctypes.c_int
    lib.lk_sync.argtypes = [vp, vp]
    lib.lk_candidates.restype = ctypes.c_int
    lib.lk_candidates.argtypes = [vp, vp, i64, ctypes.POINTER(i64), vp]
    lib.lk_get_stats.restype = ctypes.c_int
    lib.lk_get_stats.argtypes = [vp, ctypes.POINTER(lk_stats)]
    lib.lk_get_error_estimates.restype = ctypes.c_int
    lib.lk_get_error_estimates.argtypes = [vp, vp, i64, vp]
    lib.lk_get_options.restype = ctypes.c_int
    lib.lk_get_options.argtypes = [vp, ctypes.POINTER(lk_options)]
    lib.lk_destroy.restype = None
    lib.lk_destroy.argtypes = [vp]
    lib.lk_last_error.restype = ctypes.c_char_p
    lib.lk_last_error.argtypes = [vp]
    lib.lk_plan_create.restype = ctypes.c_int
    lib.lk_plan_create.argtypes = [vp, i32p, i64, ctypes.POINTER(vp), vp]
    lib.lk_plan_run.restype = ctypes.c_int
    lib.lk_plan_run.argtypes = [vp, vp, vp, vp, vp]
    lib.lk_plan_destroy.restype = None
    lib.lk_plan_destroy.argtypes = [vp]
    lib.lk_server_default_options.restype = None
    lib.lk_server_default_options.argtypes = [ctypes.POINTER(lk_server_options)]
    lib.lk_server_create.restype = ctypes.c_int
    lib.lk_server_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(lk_server_options)]
    lib.lk_server_stream.restype = vp
    lib.lk_server_stream.argtypes = [vp]
    lib.lk_server_submit.restype = ctypes.c_int
    lib.lk_server_submit.argtypes = [vp, vp, i32p, i64, ctypes.POINTER(ctypes.c_int64)]
    lib.lk_server_submit_geometry.restype = ctypes.c_int
    lib.lk_server_submit_geometry.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int64)]
    lib.lk_server_poll_pairs.restype = ctypes.c_int
    lib.lk_server_poll_pairs.argtypes = [vp, i64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64), vp,
                                         i64, vp, vp, vp]
    lib.lk_measure_fp32_peak.restype = ctypes.c_int
    lib.lk_measure_fp32_peak.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), vp]
    lib.lk_server_step.restype = ctypes.c_int
    lib.lk_server_step.argtypes = [vp, ctypes.c_int]
    lib.lk_server_poll.restype = ctypes.c_int
    lib.lk_server_poll.argtypes = [vp, i64, ctypes.POINTER(ctypes.c_int), vp, vp, vp]
    lib.lk_server_completed.restype = ctypes.c_int
    lib.lk_server_completed.argtypes = [vp, vp, i64, ctypes.POINTER(i64)]
    lib.lk_server_get_stats.restype = ctypes.c_int
    lib.lk_server_get_stats.argtypes = [vp, ctypes.POINTER(lk_server_stats)]
    lib.lk_server_last_error.restype = ctypes.c_char_p
    lib.lk_server_last_error.argtypes = [vp]
    lib.lk_server_destroy.restype = None
    lib.lk_server_destroy.argtypes = [vp]
    lib.lk_verify_expected.restype = ctypes.c_int
    lib.lk_verify_expected.argtypes = [vp, i32p, vp, i64, i64, ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_int64), vp, vp, vp, vp]
    lib.lk_autotune.restype = ctypes.c_int
    lib.lk_autotune.argtypes = [vp, i32p, i64, vp]
    lib.lk_tune_get.restype = ctypes.c_int
    lib.lk_tune_get.argtypes = [vp, vp, i64, ctypes.POINTER(ctypes.c_int64)]
    lib.lk_tune_set.restype = ctypes.c_int
    lib.lk_tune_set.argtypes = [vp, vp, i64]
    lib.lk_verify_noalloc.restype = ctypes.c_int
    lib.lk_verify_noalloc.argtypes = [vp, ctypes.c_int, i64, vp, i64, i32p, i64, vp, vp, vp, vp]
    _lib = lib
    return lib


# ----------------------------------------------------------------------------- marshalling

def _ptr(x):
    """Address of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError("expected a numpy array or torch tensor, got %r" % type(x))


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dtype_code(x):
    dt = str(getattr(x, "dtype", ""))
    if dt.endswith("float32"):
        return LK_F32
    if dt.endswith("float64"):
        return LK_F64
    raise TypeError("vertices must be float32 or float64, got %s" % dt)


def _check(status, ctx=None):
    if status != LK_OK:
        msg = load().lk_last_error(ctx)
        raise LkError(status, msg.decode() if msg else "")


# ----------------------------------------------------------------------------- C functions

def lk_default_options() -> lk_options:
    o = lk_options()
    load().lk_default_options(ctypes.byref(o))
    return o


def lk_create(vertices, loop_offsets, options: lk_options | None = None, stream=None):
    """Returns the context handle (an int).  vertices [N,3] float32/float64;
    loop_offsets int64 [L+1]."""
    n = int(vertices.shape[0])
    if len(vertices.shape) != 2 or vertices.shape[1] != 3:
        raise ValueError("vertices must be [N,3]")
    if str(loop_offsets.dtype).split(".")[-1] != "int64":
        raise TypeError("loop_offsets must be int64")
    out = ctypes.c_void_p()
    st = load().lk_create(ctypes.byref(out), _ptr(vertices), _dtype_code(vertices), n,
                          _ptr(loop_offsets), int(loop_offsets.shape[0]) - 1,
                          ctypes.byref(options) if options is not None else None, _stream(stream))
    _check(st)
    return out.value


def lk_update(ctx, data, is_delta: bool, stream=None):
    _check(load().lk_update(ctx, _ptr(data), _dtype_code(data), 1 if is_delta else 0, _stream(stream)), ctx)


def lk_candidates(ctx, pairs_out=None, stream=None):
    """Potential link search on the device.  With pairs_out (int32 [capacity, 2],
    host or device) writes the first min(n, capacity) pairs and returns n;
    without it returns a new int32 numpy array [n, 2] of all candidate pairs."""
    n = ctypes.c_int64(0)
    if pairs_out is not None:
        cap = int(pairs_out.shape[0]) if len(pairs_out.shape) > 0 else 0
        _check(load().lk_candidates(ctx, _ptr(pairs_out) if cap else None, cap, ctypes.byref(n), _stream(stream)), ctx)
        return int(n.value)
    _check(load().lk_candidates(ctx, None, 0, ctypes.byref(n), _stream(stream)), ctx)
    out = np.zeros((int(n.value), 2), np.int32)
    if out.shape[0]:
        _check(load().lk_candidates(ctx, _ptr(out), out.shape[0], ctypes.byref(n), _stream(stream)), ctx)
    return out


def lk_verify(ctx, loop_pairs, lk_out=None, raw_out=None, status_out=None, stream=None):
    """loop_pairs int32 [P,2]; outputs int32/float64/int32 [P] (host or device)."""
    if str(loop_pairs.dtype).split(".")[-1] != "int32":
        raise TypeError("loop_pairs must be int32")
    n = int(loop_pairs.shape[0]) if len(loop_pairs.shape) > 0 else 0
    _check(load().lk_verify(ctx, _ptr(loop_pairs), n, _ptr(lk_out), _ptr(raw_out), _ptr(status_out),
                            _stream(stream)), ctx)


def lk_sync(ctx, stream=None):
    _check(load().lk_sync(ctx, _stream(stream)), ctx)


def lk_get_stats(ctx) -> dict:
    s = lk_stats()
    _check(load().lk_get_stats(ctx, ctypes.byref(s)), ctx)
    return {k: getattr(s, k) for k, _ in lk_stats._fields_}


def lk_get_error_estimates(ctx, err_out, stream=None):
    """err_out float64 [P] (host or device): the last verify's per-pair error estimates."""
    n = int(err_out.shape[0]) if len(err_out.shape) > 0 else 0
    _check(load().lk_get_error_estimates(ctx, _ptr(err_out), n, _stream(stream)), ctx)


def lk_get_options(ctx) -> lk_options:
    o = lk_options()
    _check(load().lk_get_options(ctx, ctypes.byref(o)), ctx)
    return o


def lk_destroy(ctx):
    if ctx:
        load().lk_destroy(ctx)


def lk_last_error(ctx=None) -> str:
    m = load().lk_last_error(ctx)
    return m.decode() if m else ""


def lk_plan_create(ctx, loop_pairs, stream=None):
    if str(loop_pairs.dtype).split(".")[-1] != "int32":
        raise TypeError("loop_pairs must be int32")
    out = ctypes.c_void_p()
    _check(load().lk_plan_create(ctx, _ptr(loop_pairs), int(loop_pairs.shape[0]), ctypes.byref(out),
                                 _stream(stream)), ctx)
    return out.value


def lk_plan_run(plan, lk_out=None, raw_out=None, status_out=None, stream=None, ctx=None):
    _check(load().lk_plan_run(plan, _ptr(lk_out), _ptr(raw_out), _ptr(status_out), _stream(stream)), ctx)


def lk_plan_destroy(plan):
    if plan:
        load().lk_plan_destroy(plan)


def lk_verify_noalloc(vertices, loop_offsets, loop_pairs, lk_out=None, raw_out=None, status_out=None,
                      stream=None):
    """Allocation-free verify: all work buffers in the library's static device
    array.  loop_offsets (int64) and loop_pairs (int32) must be host arrays."""
    if str(loop_pairs.dtype).split(".")[-1] != "int32":
        raise TypeError("loop_pairs must be int32")
    if str(loop_offsets.dtype).split(".")[-1] != "int64":
        raise TypeError("loop_offsets must be int64")
    _check(load().lk_verify_noalloc(_ptr(vertices), _dtype_code(vertices), int(vertices.shape[0]),
                                    _ptr(loop_offsets), int(loop_offsets.shape[0]) - 1, _ptr(loop_pairs),
                                    int(loop_pairs.shape[0]), _ptr(lk_out), _ptr(raw_out), _ptr(status_out),
                                    _stream(stream)))


def lk_verify_expected(ctx, loop_pairs, expected, batch_segment_pairs=0, lk_out=None, raw_out=None,
                       status_out=None, stream=None):
    """Returns (first_mismatch or -1, pairs checked)."""
    if str(loop_pairs.dtype).split(".")[-1] != "int32" or str(expected.dtype).split(".")[-1] != "int32":
        raise TypeError("loop_pairs and expected must be int32")
    fm, nc = ctypes.c_int64(), ctypes.c_int64()
    _check(load().lk_verify_expected(ctx, _ptr(loop_pairs), _ptr(expected), int(loop_pairs.shape[0]),
                                     int(batch_segment_pairs), ctypes.byref(fm), ctypes.byref(nc), _ptr(lk_out),
                                     _ptr(raw_out), _ptr(status_out), _stream(stream)), ctx)
    return fm.value, nc.value


def lk_autotune(ctx, loop_pairs, stream=None):
    if str(loop_pairs.dtype).split(".")[-1] != "int32":
        raise TypeError("loop_pairs must be int32")
    _check(load().lk_autotune(ctx, _ptr(loop_pairs), int(loop_pairs.shape[0]), _stream(stream)), ctx)


def lk_tune_get(ctx) -> np.ndarray:
    """The tuning table as an int32 [n, 3] array (row class, column class, rows per item)."""
    n = ctypes.c_int64()
    _check(load().lk_tune_get(ctx, None, 0, ctypes.byref(n)), ctx)
    out = np.zeros((n.value, 3), np.int32)
    if n.value:
        _check(load().lk_tune_get(ctx, out.ctypes.data, n.value, ctypes.byref(n)), ctx)
    return out


def lk_tune_set(ctx, entries):
    e = np.ascontiguousarray(np.asarray(entries, np.int32).reshape(-1, 3))
    _check(load().lk_tune_set(ctx, e.ctypes.data if e.size else None, e.shape[0]), ctx)


def _check_srv(status, srv):
    if status != LK_OK:
        msg = load().lk_server_last_error(srv)
        raise LkError(status, msg.decode() if msg else "")


def lk_server_default_options() -> lk_server_options:
    o = lk_server_options()
    load().lk_server_default_options(ctypes.byref(o))
    return o


def lk_server_create(options: lk_server_options | None = None):
    out = ctypes.c_void_p()
    _check_srv(load().lk_server_create(ctypes.byref(out), ctypes.byref(options) if options is not None else None),
               None)
    return out.value


def lk_server_stream(srv) -> int:
    return load().lk_server_stream(srv) or 0


def lk_server_submit(srv, ctx, loop_pairs) -> int:
    if str(loop_pairs.dtype).split(".")[-1] != "int32":
        raise TypeError("loop_pairs must be int32")
    t = ctypes.c_int64()
    _check_srv(load().lk_server_submit(srv, ctx, _ptr(loop_pairs), int(loop_pairs.shape[0]), ctypes.byref(t)), srv)
    return t.value


def lk_server_submit_geometry(srv, ctx) -> int:
    t = ctypes.c_int64()
    _check_srv(load().lk_server_submit_geometry(srv, ctx, ctypes.byref(t)), srv)
    return t.value


def lk_server_poll_pairs(srv, ticket, pairs_out=None, lk_out=None, raw_out=None, status_out=None,
                         capacity: int = 0):
    """(done, n_pairs); the outputs are filled (and the ticket released) only
    when capacity >= n_pairs."""
    d = ctypes.c_int()
    n = ctypes.c_int64()
    _check_srv(load().lk_server_poll_pairs(srv, ticket, ctypes.byref(d), ctypes.byref(n), _ptr(pairs_out), capacity,
                                           _ptr(lk_out), _ptr(raw_out), _ptr(status_out)), srv)
    return bool(d.value), n.value


def lk_measure_fp32_peak(stream=None):
    """(TFLOP/s, ms of one launch) of the packed FP32 FMA peak kernel."""
    t = ctypes.c_double()
    m = ctypes.c_double()
    st = load().lk_measure_fp32_peak(ctypes.byref(t), ctypes.byref(m), _stream(stream))
    if st != LK_OK:
        raise LkError(st, "lk_measure_fp32_peak failed")
    return t.value, m.value


def lk_server_step(srv, wait: bool = False):
    _check_srv(load().lk_server_step(srv, 1 if wait else 0), srv)


def lk_server_poll(srv, ticket, lk_out=None, raw_out=None, status_out=None) -> bool:
    d = ctypes.c_int()
    _check_srv(load().lk_server_poll(srv, ticket, ctypes.byref(d), _ptr(lk_out), _ptr(raw_out), _ptr(status_out)),
               srv)
    return bool(d.value)


_completed_buf = np.zeros(4096, np.int64)


def lk_server_completed(srv) -> list:
    """Tickets finished since the last call, in completion order."""
    out = []
    n = ctypes.c_int64(0)
    while True:
        _check_srv(load().lk_server_completed(srv, _completed_buf.ctypes.data, _completed_buf.shape[0],
                                              ctypes.byref(n)), srv)
        out.extend(_completed_buf[: n.value].tolist())
        if n.value < _completed_buf.shape[0]:
            return out


def lk_server_get_stats(srv) -> dict:
    s = lk_server_stats()
    _check_srv(load().lk_server_get_stats(srv, ctypes.byref(s)), srv)
    return {k: getattr(s, k) for k, _ in lk_server_stats._fields_}


def lk_server_last_error(srv=None) -> str:
    m = load().lk_server_last_error(srv)
    return m.decode() if m else ""


def lk_server_destroy(srv):
    if srv:
        load().lk_server_destroy(srv)


# ----------------------------------------------------------------------------- convenience

class Linker:
    """Owns one context; ``verify(pairs)`` returns (lk, raw, status) numpy arrays."""

    def __init__(self, vertices, loop_offsets, precision=LK_MIXED, stream=None, **opts):
        o = lk_default_options()
        o.precision = precision
        for k, v in opts.items():
            setattr(o, k, v)
        self.stream = stream
        self.ctx = lk_create(vertices, loop_offsets, o, stream)

    def verify(self, pairs):
        pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        n = pairs.shape[0]
        lk = np.zeros(n, np.int32)
        raw = np.zeros(n, np.float64)
        st = np.zeros(n, np.int32)
        lk_verify(self.ctx, pairs, lk, raw, st, self.stream)
        return lk, raw, st

    def update(self, data, is_delta=True):
        lk_update(self.ctx, data, is_delta, self.stream)

    def stats(self):
        return lk_get_stats(self.ctx)

    def close(self):
        if self.ctx:
            lk_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def server_take_pairs(srv, ticket):
    """None while the request runs; then (pairs [n, 2], lk, raw, status), the
    ticket released."""
    done, n = lk_server_poll_pairs(srv, ticket)
    if not done:
        return None
    pairs = np.zeros((n, 2), np.int32)
    lk = np.zeros(n, np.int32)
    raw = np.zeros(n, np.float64)
    st = np.zeros(n, np.int32)
    if n > 0:            # with no pairs the first call has released the ticket
        lk_server_poll_pairs(srv, ticket, pairs, lk, raw, st, capacity=n)
    return pairs, lk, raw, st
