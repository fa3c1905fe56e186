"""Oracle for the linking-number direct sum -- TEST INFRASTRUCTURE ONLY.

Thin ctypes wrapper over ``lk_oracle.c``: a plain FP64 CPU direct summation of
the Gauss linking number of closed polylines, evaluating the closed-form
segment-pair term of Eq. 4 (Qu & James 2021, Sec. 2.1) as written, summed over
every segment pair (Eq. 3; Sec. 3.4.2, Algorithm 5), and the potential link
search of Sec. 3.2 (Algorithm 2) as its plain all-pairs box-overlap definition.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s ``cpu_baseline``
and ``--impl reference`` legs may import this module.  The CUDA library never
calls it; the two share no code.

Integer rounding (a reading: the paper does not say how the raw sum becomes an
integer): ``lk = round-half-away-from-zero(raw)``; the raw sum of a closed
polyline pair is an integer in exact arithmetic (Eq. 3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lk_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblk_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no fast-math) if needed."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-shared",
               "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _bind(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    i64 = ctypes.c_int64
    i64p = ctypes.POINTER(ctypes.c_int64)
    i32p = ctypes.POINTER(ctypes.c_int32)
    lib.lko_term.restype = ctypes.c_double
    lib.lko_term.argtypes = [dp, dp, dp, dp]
    lib.lko_block.restype = ctypes.c_int
    lib.lko_block.argtypes = [dp, i64, dp, i64, i64, i64, i64, i64, ctypes.c_int, dp]
    lib.lko_link.restype = ctypes.c_int
    lib.lko_link.argtypes = [dp, i64, dp, i64, ctypes.c_int, dp]
    lib.lko_link_rows.restype = ctypes.c_int
    lib.lko_link_rows.argtypes = [dp, i64, dp, i64, i64p, i64, ctypes.c_int, dp]
    lib.lko_link_pairs.restype = ctypes.c_int
    lib.lko_link_pairs.argtypes = [dp, i64p, i64, i32p, i64, ctypes.c_int, dp]
    lib.lko_candidates.restype = ctypes.c_int
    lib.lko_candidates.argtypes = [dp, i64p, i64, i32p, i64, i64p]
    lib.lko_max_threads.restype = ctypes.c_int
    lib.lko_max_threads.argtypes = []
    return lib


def load_library(path: str):
    """Load an oracle build from ``path`` (tests load deliberately broken builds to
    check that the pins catch them)."""
    return _bind(ctypes.CDLL(path))


def compile_source(src_text: str, out_path: str) -> str:
    """Compile oracle C source text to a shared library at ``out_path``."""
    c_path = out_path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-shared",
                    "-fPIC", "-o", out_path, c_path, "-lm"], check=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _f64(a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if a.ndim != 2 or a.shape[1] != 3:
        raise ValueError("expected an [N,3] vertex array")
    return a


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def max_threads() -> int:
    return int(_load().lko_max_threads())


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def term(lj, lj1, ki, ki1, lib=None) -> float:
    """lambda_ji of Eq. 4 for segment l_j->l_{j+1} of loop 1 and k_i->k_{i+1} of loop 2."""
    pts = [np.ascontiguousarray(np.asarray(p, dtype=np.float64).reshape(3)) for p in (lj, lj1, ki, ki1)]
    return float((lib or _load()).lko_term(*[_dp(p) for p in pts]))


def link(l, k, threads: int | None = None, lib=None) -> float:
    """Raw FP64 sum of lambda_ji over all segment pairs of closed polylines l, k (Eq. 3)."""
    l, k = _f64(l), _f64(k)
    out = ctypes.c_double()
    rc = (lib or _load()).lko_link(_dp(l), l.shape[0], _dp(k), k.shape[0], threads or default_threads(),
                          ctypes.byref(out))
    if rc:
        raise ValueError("oracle: invalid loops (need >= 3 vertices each)")
    return out.value


def block(l, k, j0, j1, i0, i1, threads: int | None = None) -> float:
    """Sum of lambda_ji over j in [j0,j1), i in [i0,i1) (a sub-rectangle of Eq. 3's sum)."""
    l, k = _f64(l), _f64(k)
    out = ctypes.c_double()
    rc = _load().lko_block(_dp(l), l.shape[0], _dp(k), k.shape[0], j0, j1, i0, i1,
                           threads or default_threads(), ctypes.byref(out))
    if rc:
        raise ValueError("oracle: invalid block")
    return out.value


def link_rows(l, k, rows, threads: int | None = None) -> np.ndarray:
    """out[r] = sum_j lambda_{j,rows[r]} (row sums of Eq. 3's double sum)."""
    l, k = _f64(l), _f64(k)
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    out = np.zeros(rows.shape[0], dtype=np.float64)
    rc = _load().lko_link_rows(_dp(l), l.shape[0], _dp(k), k.shape[0],
                               rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), rows.shape[0],
                               threads or default_threads(), _dp(out))
    if rc:
        raise ValueError("oracle: invalid rows")
    return out


def link_pairs(vertices, offsets, pairs, threads: int | None = None, lib=None) -> np.ndarray:
    """Raw sums for every (a, b) in ``pairs`` of a CSR geometry (Algorithm 1's loop over P)."""
    v = _f64(vertices)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    out = np.zeros(pr.shape[0], dtype=np.float64)
    if pr.shape[0] == 0:
        return out
    rc = (lib or _load()).lko_link_pairs(_dp(v), off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                off.shape[0] - 1, pr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                pr.shape[0], threads or default_threads(), _dp(out))
    if rc:
        raise ValueError("oracle: invalid pairs or loops")
    return out


def round_lk(raw) -> np.ndarray:
    """Nearest integer, halves away from zero (the rounding reading used throughout)."""
    raw = np.asarray(raw, dtype=np.float64)
    return (np.sign(raw) * np.floor(np.abs(raw) + 0.5)).astype(np.int64)


def candidates(vertices, offsets, lib=None) -> np.ndarray:
    """Potential link search (Sec. 3.2, Algorithm 2) as its plain definition:
    int32 [n, 2] pairs (i, j), i < j, in (i, j) order, of loops whose closed
    axis-aligned bounding boxes overlap on all three axes."""
    lib = lib or _load()
    v = _f64(vertices)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    nloops = off.shape[0] - 1
    n = ctypes.c_int64(0)
    i64p = ctypes.POINTER(ctypes.c_int64)
    i32p = ctypes.POINTER(ctypes.c_int32)
    offp = off.ctypes.data_as(i64p)
    if lib.lko_candidates(_dp(v), offp, nloops, None, 0, ctypes.byref(n)):
        raise ValueError("oracle: invalid arguments")
    out = np.zeros((int(n.value), 2), np.int32)
    if out.shape[0]:
        if lib.lko_candidates(_dp(v), offp, nloops, out.ctypes.data_as(i32p), out.shape[0], ctypes.byref(n)):
            raise ValueError("oracle: invalid arguments")
    return out
