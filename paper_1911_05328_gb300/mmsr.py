"""Thin ctypes binding of libmmsr (include/mmsr.h) -- argument marshalling only.

Every entry point keeps its C name.  Tensor arguments may be torch CUDA
tensors (their ``data_ptr()`` is passed) or raw integer device addresses;
``stream`` may be a ``torch.cuda.Stream``, a raw ``cudaStream_t`` integer or
None (torch's current stream on the current device).  All compute happens in
the library's CUDA kernels; there is no fallback: if libmmsr.so is missing
the first call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmmsr.so")

MM_SR_PLUS_TIMES_F64 = 0
MM_SR_PLUS_TIMES_F32 = 1
MM_SR_PLUS_TIMES_F64ACC = 2
MM_SR_MIN_PLUS_I32 = 3
MM_SR_OR_AND_U8 = 4

MM_STRASSEN_PAPER = 0
MM_LEVELS_AUTO = 16
MM_STRASSEN_WINOGRAD = 1

MM_OPT_MINPLUS_PACKED = 1
MM_OPT_MINPLUS_STREAMK = 2
MM_OPT_STRASSEN_TOP_F64 = 4
MM_OPT_TEST_SKIP_SIGNAL = 5
MM_OPT_F64ACC_SLICES = 6
MM_OPT_STRASSEN_FUSED = 7
MM_OPT_F32_STREAMK = 8
MM_OPT_F64_STREAMK = 9

MM_CLOSURE_EARLY_EXIT = 1

MM_OK = 0
MM_ERR_ARG = -1
MM_ERR_UNSUPPORTED = -2
MM_ERR_WORKSPACE = -3
MM_ERR_SHAPE = -4
MM_ERR_CUDA = -5
MM_ERR_TIMEOUT = -6
MM_ERR_ALIGN = -7

INF = 1 << 30


class MMError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__("%s returned %d (%s)" % (what, status, status_string(status)))
        self.status = status


class mm_plan_t(ctypes.Structure):
    _fields_ = [("split_k", ctypes.c_int32), ("levels", ctypes.c_int32),
                ("tile_m", ctypes.c_int32), ("tile_n", ctypes.c_int32), ("tile_k", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("workspace_used", ctypes.c_int64),
                ("workspace_min", ctypes.c_int64)]


class mm_problem_t(ctypes.Structure):
    _fields_ = [("semiring", ctypes.c_int32), ("levels", ctypes.c_int32),
                ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("C", ctypes.c_void_p),
                ("split_k", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Open libmmsr.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise OSError("libmmsr.so not found at %s: run __graft_entry__.build() "
                              "(there is no CPU fallback)" % path)
            lib = ctypes.CDLL(path)
            i32, i64, vp, sz = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t
            lib.mm_semiring.argtypes = [i32, i64, i64, i64, vp, vp, vp, vp, sz, vp]
            lib.mm_minplus_noalloc.argtypes = [i64, i64, i64, vp, vp, vp, i32, vp]
            lib.mm_minplus_noalloc.restype = ctypes.c_int
            lib.mm_strassen.argtypes = [i32, i32, i32, i64, i64, i64, vp, vp, vp, vp, sz, vp]
            lib.mm_batched.argtypes = [i32, ctypes.POINTER(mm_problem_t), vp, sz, vp]
            lib.mm_batched_query.argtypes = [i32, ctypes.POINTER(mm_problem_t)]
            lib.mm_batched_query.restype = sz
            lib.mm_plan_query.argtypes = [i32, i32, i64, i64, i64, sz, ctypes.POINTER(mm_plan_t)]
            lib.mm_last_device_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
            lib.mm_status_string.argtypes = [i32]
            lib.mm_status_string.restype = ctypes.c_char_p
            lib.mm_version.argtypes = []
            lib.mm_set_option.argtypes = [i32, i32]
            lib.mm_set_option.restype = ctypes.c_int
            lib.mm_star_strassen.argtypes = [i32, i32, i32, i32, i64, i64, i64, vp, vp, vp, vp, sz, vp]
            lib.mm_star_strassen.restype = ctypes.c_int
            lib.mm_star_strassen_query.argtypes = [i32, i32, i32, i64, i64, i64, sz, ctypes.POINTER(mm_plan_t)]
            lib.mm_star_strassen_query.restype = ctypes.c_int
            lib.mm_strassen_tar.argtypes = [i32, i32, i32, i64, i64, i64, vp, vp, vp, vp, sz, vp]
            lib.mm_strassen_tar.restype = ctypes.c_int
            lib.mm_strassen_tar_query.argtypes = [i32, i32, i64, i64, i64, ctypes.POINTER(mm_plan_t)]
            lib.mm_strassen_tar_query.restype = ctypes.c_int
            lib.mm_strassen_tar_waves.argtypes = [i32, i32, ctypes.POINTER(ctypes.c_int)]
            lib.mm_strassen_tar_waves.restype = ctypes.c_int
            lib.mm_closure.argtypes = [i32, i64, vp, vp, vp, sz, i32, ctypes.POINTER(ctypes.c_int), vp]
            lib.mm_closure.restype = ctypes.c_int
            lib.mm_closure_query.argtypes = [i32, i64, sz, ctypes.POINTER(mm_plan_t)]
            lib.mm_closure_query.restype = ctypes.c_int
            for f in ("mm_semiring", "mm_strassen", "mm_batched", "mm_plan_query",
                      "mm_last_device_status", "mm_version"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def _addr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(s):
    if s is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


def _check(rc, what, check):
    if check and rc != MM_OK:
        raise MMError(rc, what)
    return rc


def status_string(status: int) -> str:
    return load().mm_status_string(int(status)).decode()


def mm_semiring(semiring, m, n, k, A, B, C, workspace=None, workspace_bytes=0, stream=None,
                check=True) -> int:
    rc = load().mm_semiring(int(semiring), int(m), int(n), int(k), _addr(A), _addr(B), _addr(C),
                            _addr(workspace), int(workspace_bytes), _stream(stream))
    return _check(rc, "mm_semiring", check)


def mm_minplus_noalloc(m, n, k, A, B, C, split_k=1, stream=None, check=True) -> int:
    """(min,+) product with split-K partials in the library's static 64 MiB
    device scratch (no workspace argument, no allocation)."""
    rc = load().mm_minplus_noalloc(int(m), int(n), int(k), _addr(A), _addr(B), _addr(C),
                                   int(split_k), _stream(stream))
    return _check(rc, "mm_minplus_noalloc", check)


def mm_strassen(levels, variant, semiring, m, n, k, A, B, C, workspace=None, workspace_bytes=0,
                stream=None, check=True) -> int:
    rc = load().mm_strassen(int(levels), int(variant), int(semiring), int(m), int(n), int(k),
                            _addr(A), _addr(B), _addr(C), _addr(workspace), int(workspace_bytes),
                            _stream(stream))
    return _check(rc, "mm_strassen", check)


def mm_closure(semiring, n, A, C, workspace=None, workspace_bytes=0, flags=0, stream=None,
               check=True):
    """C := A* by repeated squaring; returns (status, squarings run)."""
    sq = ctypes.c_int(0)
    rc = load().mm_closure(int(semiring), int(n), _addr(A), _addr(C), _addr(workspace),
                           int(workspace_bytes), int(flags), ctypes.byref(sq), _stream(stream))
    _check(rc, "mm_closure", check)
    return rc, sq.value


def mm_closure_query(semiring, n, workspace_bytes=0, check=True) -> mm_plan_t:
    plan = mm_plan_t()
    rc = load().mm_closure_query(int(semiring), int(n), int(workspace_bytes), ctypes.byref(plan))
    _check(rc, "mm_closure_query", check)
    plan.status = rc
    return plan


def mm_strassen_tar(levels, variant, semiring, m, n, k, A, B, C, workspace=None, workspace_bytes=0, stream=None,
                    check=True) -> int:
    rc = load().mm_strassen_tar(int(levels), int(variant), int(semiring), int(m), int(n), int(k), _addr(A),
                                _addr(B), _addr(C), _addr(workspace), int(workspace_bytes), _stream(stream))
    return _check(rc, "mm_strassen_tar", check)


def mm_strassen_tar_query(levels, semiring, m, n, k, check=True) -> mm_plan_t:
    plan = mm_plan_t()
    rc = load().mm_strassen_tar_query(int(levels), int(semiring), int(m), int(n), int(k), ctypes.byref(plan))
    _check(rc, "mm_strassen_tar_query", check)
    plan.status = rc
    return plan


def mm_strassen_tar_waves(levels, variant):
    """(number of waves or MM_ERR_UNSUPPORTED, [wave of leaf product p for
    p = 0 .. 7^levels - 1])."""
    w = (ctypes.c_int * (7 ** int(levels)))()
    rc = load().mm_strassen_tar_waves(int(levels), int(variant), w)
    if rc < 0 and rc != MM_ERR_UNSUPPORTED:
        raise MMError(rc, "mm_strassen_tar_waves")
    return rc, list(w)


def mm_star_strassen(classic_levels, levels, variant, semiring, m, n, k, A, B, C, workspace=None,
                     workspace_bytes=0, stream=None, check=True) -> int:
    rc = load().mm_star_strassen(int(classic_levels), int(levels), int(variant), int(semiring), int(m),
                                 int(n), int(k), _addr(A), _addr(B), _addr(C), _addr(workspace),
                                 int(workspace_bytes), _stream(stream))
    return _check(rc, "mm_star_strassen", check)


def mm_star_strassen_query(classic_levels, levels, semiring, m, n, k, workspace_bytes=0,
                           check=True) -> mm_plan_t:
    plan = mm_plan_t()
    rc = load().mm_star_strassen_query(int(classic_levels), int(levels), int(semiring), int(m), int(n),
                                       int(k), int(workspace_bytes), ctypes.byref(plan))
    _check(rc, "mm_star_strassen_query", check)
    plan.status = rc
    return plan


def _problems(problems):
    arr = (mm_problem_t * len(problems))()
    for i, p in enumerate(problems):
        sr, m, n, k, A, B, C = p[:7]
        split = int(p[7]) if len(p) > 7 else 0
        levels = int(p[8]) if len(p) > 8 else 0
        arr[i] = mm_problem_t(int(sr), levels, int(m), int(n), int(k), _addr(A), _addr(B), _addr(C), split, 0)
    return arr


def mm_batched(problems, workspace=None, workspace_bytes=0, stream=None, check=True) -> int:
    """problems: sequence of (semiring, m, n, k, A, B, C[, split_k[, levels]])."""
    arr = _problems(problems)
    rc = load().mm_batched(len(problems), arr, _addr(workspace), int(workspace_bytes),
                           _stream(stream))
    return _check(rc, "mm_batched", check)


def mm_batched_query(problems) -> int:
    arr = _problems(problems)
    return int(load().mm_batched_query(len(problems), arr))


def mm_plan_query(semiring, levels, m, n, k, workspace_bytes=0, check=True) -> mm_plan_t:
    plan = mm_plan_t()
    rc = load().mm_plan_query(int(semiring), int(levels), int(m), int(n), int(k),
                              int(workspace_bytes), ctypes.byref(plan))
    _check(rc, "mm_plan_query", check)
    plan.status = rc
    return plan


def mm_last_device_status(stream=None) -> int:
    st = ctypes.c_int(0)
    rc = load().mm_last_device_status(_stream(stream), ctypes.byref(st))
    _check(rc, "mm_last_device_status", True)
    return st.value


def mm_set_option(option, value, check=True) -> int:
    rc = load().mm_set_option(int(option), int(value))
    return _check(rc, "mm_set_option", check)


def mm_version() -> int:
    return int(load().mm_version())


def mm_strassen_tables(variant):
    """(alpha[7][4], beta[7][4], gamma[4][7]) int8 tables of one level."""
    import numpy as np

    a = (ctypes.c_int8 * 28)()
    b = (ctypes.c_int8 * 28)()
    g = (ctypes.c_int8 * 28)()
    lib = load()
    lib.mm_strassen_tables.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.mm_strassen_tables.restype = ctypes.c_int
    _check(lib.mm_strassen_tables(int(variant), ctypes.addressof(a), ctypes.addressof(b),
                                  ctypes.addressof(g)), "mm_strassen_tables", True)
    return (np.array(a[:], dtype=np.int64).reshape(7, 4), np.array(b[:], dtype=np.int64).reshape(7, 4),
            np.array(g[:], dtype=np.int64).reshape(4, 7))
