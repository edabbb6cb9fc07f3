"""Seeded synthetic inputs for every workload of the library.

This module draws random matrices and problem lists and nothing else: it
holds none of the multiplication arithmetic, so both the CUDA path and the
CPU oracle can take their inputs from it without sharing any of the method.

Generator: ``numpy.random.default_rng(seed)`` (PCG64); A is drawn first and
then B from the same generator.  The recipes (sizes, distributions, sentinel
fraction, seeds) are the workloads the library is measured on:

* FP64 classic, n=256: A, B ~ uniform[-1, 1], seed 0.
* (min,+) tropical, n=4096: integers uniform in [0, 1000]; then each entry
  independently becomes the +inf sentinel 2^30 with probability 0.1; seed 1.
* FP32 classic, n=8192: A, B ~ normal(0, 1) in float32, seed 2.
* Strassen-Winograd, n=16384 and 12288x16384x8192: uniform[-1, 1] in FP64
  (and its float32 cast), seed 3.
* Batched: 512 problems, m, n, k each log-uniform in [64, 2048], 70% FP32
  (+,x) with normal(0,1) entries and 30% (min,+) with integers in [0, 1000],
  seed 4.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

INF = 1 << 30  # +infinity sentinel of the (min,+) semiring


def uniform_f64(m, k, n, seed=0, lo=-1.0, hi=1.0):
    rng = np.random.default_rng(seed)
    A = rng.uniform(lo, hi, size=(m, k))
    B = rng.uniform(lo, hi, size=(k, n))
    return A, B


def normal_f32(m, k, n, seed=2):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal(size=(m, k), dtype=np.float32)
    B = rng.standard_normal(size=(k, n), dtype=np.float32)
    return A, B


def tropical_i32(m, k, n, seed=1, hi=1000, inf_frac=0.1):
    """(min,+) inputs: integers in [0, hi], a fraction set to the sentinel."""
    rng = np.random.default_rng(seed)
    out = []
    for shape in ((m, k), (k, n)):
        X = rng.integers(0, hi + 1, size=shape, dtype=np.int32)
        if inf_frac > 0:
            X[rng.random(size=shape) < inf_frac] = INF
        out.append(X)
    return out[0], out[1]


def small_int(m, k, n, seed=5, bound=8, dtype=np.float64):
    """Integer-valued matrices in [-bound, bound]; exact in bf16/fp16/fp32."""
    rng = np.random.default_rng(seed)
    A = rng.integers(-bound, bound + 1, size=(m, k)).astype(dtype)
    B = rng.integers(-bound, bound + 1, size=(k, n)).astype(dtype)
    return A, B


def boolean_u8(m, k, n, seed=6, density=0.05):
    rng = np.random.default_rng(seed)
    A = (rng.random(size=(m, k)) < density).astype(np.uint8)
    B = (rng.random(size=(k, n)) < density).astype(np.uint8)
    return A, B


def graph_minplus(nv, seed=7, density=0.2, hi=100):
    """Random directed graph as a (min,+) distance matrix: 0 diagonal,
    weights in [1, hi] on edges, sentinel elsewhere."""
    rng = np.random.default_rng(seed)
    D = rng.integers(1, hi + 1, size=(nv, nv), dtype=np.int32)
    D[rng.random(size=(nv, nv)) >= density] = INF
    np.fill_diagonal(D, 0)
    return D


# semiring codes shared with the C ABI header (include/mmsr.h)
SR_PLUS_TIMES_F64 = 0
SR_PLUS_TIMES_F32 = 1
SR_PLUS_TIMES_F64ACC = 2
SR_MIN_PLUS_I32 = 3
SR_OR_AND_U8 = 4


@dataclass
class Problem:
    semiring: int
    m: int
    n: int
    k: int
    A: np.ndarray
    B: np.ndarray


def batched_problems(count=512, seed=4, lo=64, hi=2048, frac_fp32=0.7, dims=None):
    """Mixed batch: shapes log-uniform in [lo, hi]; ``round(count*frac_fp32)``
    FP32 (+,x) problems (normal(0,1)) and the rest (min,+) (integers in
    [0, 1000], no sentinel), in an order drawn by a permutation."""
    rng = np.random.default_rng(seed)
    n_fp = int(round(count * frac_fp32))
    kinds = np.array([SR_PLUS_TIMES_F32] * n_fp + [SR_MIN_PLUS_I32] * (count - n_fp))
    kinds = kinds[rng.permutation(count)]
    if dims is None:
        dims = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=(count, 3)))).astype(np.int64)
    probs = []
    for p in range(count):
        m, n, k = (int(x) for x in dims[p])
        if kinds[p] == SR_PLUS_TIMES_F32:
            A = rng.standard_normal(size=(m, k), dtype=np.float32)
            B = rng.standard_normal(size=(k, n), dtype=np.float32)
        else:
            A = rng.integers(0, 1001, size=(m, k), dtype=np.int32)
            B = rng.integers(0, 1001, size=(k, n), dtype=np.int32)
        probs.append(Problem(int(kinds[p]), m, n, k, A, B))
    return probs


def batched_long_k_problems(seed=11, long_count=8, long_shape=(256, 384, 32768), short_count=56, lo=64,
                            hi=1024):
    """FP32 batch whose few long-k products would end it alone:
    ``long_count`` products of ``long_shape`` and ``short_count`` with m, n,
    k log-uniform in [lo, hi], normal(0,1) entries."""
    rng = np.random.default_rng(seed)
    dims = [tuple(long_shape)] * long_count
    dims += [tuple(int(round(math.exp(x))) for x in rng.uniform(math.log(lo), math.log(hi), size=3))
             for _ in range(short_count)]
    probs = []
    for m, n, k in dims:
        A = rng.standard_normal((m, k), dtype=np.float32)
        B = rng.standard_normal((k, n), dtype=np.float32)
        probs.append(Problem(SR_PLUS_TIMES_F32, m, n, k, A, B))
    return probs
