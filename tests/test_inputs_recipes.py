"""The seeded workload generators follow their stated recipes (sizes,
ranges, sentinel fraction, shape distribution, semiring mix) and are
reproducible from their seeds; checked on the CPU at reduced sizes where the
recipe does not depend on the size."""
import math

import numpy as np

from paper_1911_05328_gb300 import inputs, mmsr


def test_tropical_recipe():
    A, B = inputs.tropical_i32(512, 384, 256, seed=1)
    assert A.shape == (512, 384) and B.shape == (384, 256) and A.dtype == np.int32
    for X in (A, B):
        fin = X[X != inputs.INF]
        assert fin.min() >= 0 and fin.max() <= 1000
        frac = np.mean(X == inputs.INF)
        assert abs(frac - 0.1) < 0.01, frac  # independent Bernoulli(0.1) per entry
    A2, B2 = inputs.tropical_i32(512, 384, 256, seed=1)
    assert np.array_equal(A, A2) and np.array_equal(B, B2)
    assert inputs.INF == 1 << 30


def test_uniform_and_normal_recipes():
    A, B = inputs.uniform_f64(300, 200, 100, seed=0)
    assert A.dtype == np.float64 and -1 <= A.min() and A.max() < 1 and abs(A.mean()) < 0.02
    F, G = inputs.normal_f32(300, 200, 100, seed=2)
    assert F.dtype == np.float32 and abs(F.std() - 1) < 0.02 and abs(G.mean()) < 0.02


def test_batched_recipe():
    probs = inputs.batched_problems(count=512, seed=4, lo=64, hi=2048)
    kinds = [p.semiring for p in probs]
    assert len(probs) == 512 and kinds.count(mmsr.MM_SR_PLUS_TIMES_F32) == 358
    assert kinds.count(mmsr.MM_SR_MIN_PLUS_I32) == 154
    dims = np.array([(p.m, p.n, p.k) for p in probs])
    assert dims.min() >= 64 and dims.max() <= 2048
    # log-uniform: log-dimensions spread evenly over [ln 64, ln 2048]
    logs = np.log(dims.ravel())
    assert abs(logs.mean() - 0.5 * (math.log(64) + math.log(2048))) < 0.1
    for p in probs[:40]:
        assert p.A.shape == (p.m, p.k) and p.B.shape == (p.k, p.n)
        if p.semiring == mmsr.MM_SR_MIN_PLUS_I32:
            assert p.A.dtype == np.int32 and p.A.min() >= 0 and p.A.max() <= 1000  # no sentinel
        else:
            assert p.A.dtype == np.float32
    del probs
    one = inputs.batched_problems(count=24, seed=9, lo=16, hi=128)
    two = inputs.batched_problems(count=24, seed=9, lo=16, hi=128)
    assert all(a.m == b.m and a.n == b.n and a.k == b.k and np.array_equal(a.A, b.A) and np.array_equal(a.B, b.B)
               for a, b in zip(one, two))


def test_graph_recipe():
    D = inputs.graph_minplus(200, seed=1, density=0.1, hi=1000)
    assert np.all(np.diag(D) == 0)
    off = D[~np.eye(200, dtype=bool)]
    arcs = off[off != inputs.INF]
    assert arcs.min() >= 1 and arcs.max() <= 1000
    assert abs(arcs.size / off.size - 0.1) < 0.01
