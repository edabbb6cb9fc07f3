"""CPU oracle for semiring matrix multiplication -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
library (``paper_1911_05328_gb300``) never imports it, and it imports
nothing from the library.

The arithmetic lives in ``mm_oracle.c`` (plain C, FP64 / int64, OpenMP over
independent rows).  This module compiles it with gcc on first use and wraps
each entry point for numpy arrays.  Every function computes the plain
definition ``C[i][j] = (+)_t A[i][t] (x) B[t][j]`` (Section 2, closed-semiring
MM) with ``t`` ascending; ``rows`` selects which rows of C to compute.

Parity pins: see ``tests/test_oracle_pins.py``.  All functions here are
pinned (identity/zero invariants, closed forms, brute force, exact rationals,
library routines, Strassen/Winograd agreement, Floyd-Warshall closure,
closures against scipy's graph search and the power series on tiny inputs).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

INF = 1 << 30  # +infinity of the (min,+) semiring on [0, 2^30]


def build(force: bool = False) -> str:
    """Compile mm_oracle.c into liboracle.so next to it (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, vp = ctypes.c_int64, ctypes.c_void_p
            for name in ("oracle_mm_f64", "oracle_mm_i64", "oracle_mm_minplus", "oracle_mm_orand"):
                f = getattr(lib, name)
                f.argtypes = [i64, i64, i64, vp, vp, vp, vp, i64]
                f.restype = ctypes.c_int
            lib.oracle_strassen_i64.argtypes = [ctypes.c_int, ctypes.c_int, i64, i64, i64, vp, vp, vp]
            lib.oracle_strassen_i64.restype = ctypes.c_int
            lib.oracle_floyd_warshall.argtypes = [i64, vp]
            lib.oracle_floyd_warshall.restype = ctypes.c_int
            lib.oracle_closure_minplus_rows.argtypes = [i64, vp, i64, vp, vp]
            lib.oracle_closure_minplus_rows.restype = ctypes.c_int
            for name in ("oracle_closure_minplus", "oracle_closure_orand"):
                getattr(lib, name).argtypes = [i64, vp]
                getattr(lib, name).restype = ctypes.c_int
            lib.oracle_num_threads.argtypes = []
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


def _rows(rows, m):
    if rows is None:
        return None, m
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    return r, int(r.shape[0])


def _call(fname, A, B, out_dtype, rows, in_dtype):
    A = np.ascontiguousarray(A, dtype=in_dtype)
    B = np.ascontiguousarray(B, dtype=in_dtype)
    if A.ndim != 2 or B.ndim != 2 or A.shape[1] != B.shape[0]:
        raise ValueError("shape mismatch: A %s, B %s" % (A.shape, B.shape))
    m, k = A.shape
    n = B.shape[1]
    r, nrows = _rows(rows, m)
    C = np.empty((nrows, n), dtype=out_dtype)
    rc = getattr(_load(), fname)(m, n, k, _ptr(A), _ptr(B), _ptr(C),
                                 _ptr(r) if r is not None else None, nrows)
    if rc != 0:
        raise RuntimeError("%s failed with %d" % (fname, rc))
    return C


def mm_f64(A, B, rows=None) -> np.ndarray:
    """(+,x) over the reals in FP64; float32 inputs are widened exactly."""
    return _call("oracle_mm_f64", A, B, np.float64, rows, np.float64)


def mm_i64(A, B, rows=None) -> np.ndarray:
    """(+,x) over the integers, exact int64."""
    return _call("oracle_mm_i64", A, B, np.int64, rows, np.int64)


def mm_minplus(A, B, rows=None) -> np.ndarray:
    """(min,+) on [0, 2^30] with 2^30 = +inf; int64 sums, clamped result."""
    return _call("oracle_mm_minplus", A, B, np.int32, rows, np.int32)


def mm_orand(A, B, rows=None) -> np.ndarray:
    """Boolean (or, and); nonzero input bytes are true, output is 0/1."""
    return _call("oracle_mm_orand", A, B, np.uint8, rows, np.uint8)


def strassen_i64(A, B, levels: int, variant: str = "strassen") -> np.ndarray:
    """Exact int64 Strassen ('strassen', the paper's formulas) or
    Strassen-Winograd ('winograd') recursion, ``levels`` deep."""
    A = np.ascontiguousarray(A, dtype=np.int64)
    B = np.ascontiguousarray(B, dtype=np.int64)
    m, k = A.shape
    n = B.shape[1]
    C = np.empty((m, n), dtype=np.int64)
    v = {"strassen": 0, "winograd": 1}[variant]
    rc = _load().oracle_strassen_i64(v, levels, m, n, k, _ptr(A), _ptr(B), _ptr(C))
    if rc != 0:
        raise RuntimeError("oracle_strassen_i64 failed with %d" % rc)
    return C


def floyd_warshall(D) -> np.ndarray:
    """All-pairs shortest paths (int64, INF = 2^30 means no edge)."""
    D = np.array(D, dtype=np.int64, copy=True, order="C")
    rc = _load().oracle_floyd_warshall(D.shape[0], _ptr(D))
    if rc != 0:
        raise RuntimeError("oracle_floyd_warshall failed with %d" % rc)
    return D


def closure_minplus(A) -> np.ndarray:
    """(min,+) closure A* = 1 (+) A (+) A^2 (+) ... (all-pairs shortest paths,
    diagonal 0, sentinel 2^30 = unreachable) of a square int matrix, as int64."""
    D = np.array(A, dtype=np.int64, copy=True, order="C")
    rc = _load().oracle_closure_minplus(D.shape[0], _ptr(D))
    if rc != 0:
        raise RuntimeError("oracle_closure_minplus failed with %d" % rc)
    return D


def closure_minplus_rows(A, rows) -> np.ndarray:
    """Rows of the (min,+) closure by one dense Dijkstra per source row (int64)."""
    D = np.ascontiguousarray(A, dtype=np.int32)
    n = D.shape[0]
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    if rows.size and (rows.min() < 0 or rows.max() >= n):
        raise ValueError("row index out of range")
    out = np.empty((rows.size, n), dtype=np.int64)
    rc = _load().oracle_closure_minplus_rows(n, _ptr(D), rows.size, _ptr(rows), _ptr(out))
    if rc != 0:
        raise RuntimeError("oracle_closure_minplus_rows failed with %d" % rc)
    return out


def closure_orand(A) -> np.ndarray:
    """(or, and) closure: reflexive-transitive reachability of a square 0/1
    matrix (nonzero = arc), as uint8 0/1."""
    R = np.array(A, dtype=np.uint8, copy=True, order="C")
    rc = _load().oracle_closure_orand(R.shape[0], _ptr(R))
    if rc != 0:
        raise RuntimeError("oracle_closure_orand failed with %d" % rc)
    return R


def num_threads() -> int:
    """Host threads the oracle's OpenMP loops use."""
    return int(_load().oracle_num_threads())


def sample_rows(m: int, count: int = 512) -> np.ndarray:
    """Rows evaluated when a full product is too large for the oracle: an even
    spread plus the quadrant boundaries of up to four halvings (where a
    recursive split would put an edge)."""
    base = set(np.linspace(0, m - 1, max(count - 40, 1)).round().astype(np.int64).tolist())
    for lvl in range(1, 5):
        q = m >> lvl
        if q <= 0:
            break
        for b in range(0, m, q):
            base.update(x for x in (b - 1, b) if 0 <= x < m)
    rows = np.array(sorted(base), dtype=np.int64)
    return rows
