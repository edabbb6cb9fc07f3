"""Closure A* by repeated squaring on the GPU vs the oracle's vertex
elimination (Floyd-Warshall for (min,+), Warshall for boolean): bit-exact."""
import numpy as np
import pytest

import oracle
from paper_1911_05328_gb300 import inputs, mmsr

from gpu_util import canary_intact, dev, empty, workspace

pytestmark = pytest.mark.gpu
MP = mmsr.MM_SR_MIN_PLUS_I32
OA = mmsr.MM_SR_OR_AND_U8


def closure(sr, A, extra_parts=0, flags=0, in_place=False):
    import torch

    n = A.shape[0]
    p = mmsr.mm_closure_query(sr, n, 0)
    budget = int(p.workspace_min) + extra_parts * n * n * 4
    ws = workspace(budget)
    dA = dev(A)
    dC = dA if in_place else empty(A.shape, dA.dtype)
    rc, t = mmsr.mm_closure(sr, n, dA, dC, ws, budget, flags=flags)
    torch.cuda.synchronize()
    assert canary_intact(ws, budget)
    assert mmsr.mm_last_device_status() == 0
    return dC.cpu().numpy(), t, p


@pytest.mark.parametrize("n", [1, 2, 3, 17, 100, 129, 300])
def test_minplus_closure_exact(n):
    D = inputs.graph_minplus(n, seed=40 + n, density=0.05, hi=1000)
    np.fill_diagonal(D, 7)  # the closure's 1 term must clear a nonzero diagonal
    C, t, p = closure(MP, D)
    assert t == p.levels
    np.testing.assert_array_equal(C.astype(np.int64), oracle.closure_minplus(D))


@pytest.mark.parametrize("parts", [0, 1, 3])
@pytest.mark.parametrize("flags", [0, mmsr.MM_CLOSURE_EARLY_EXIT])
def test_minplus_closure_budget_and_early_exit(parts, flags):
    n = 333
    D = inputs.graph_minplus(n, seed=60 + parts, density=0.03, hi=1000)
    C, t, p = closure(MP, D, extra_parts=parts, flags=flags)
    np.testing.assert_array_equal(C.astype(np.int64), oracle.closure_minplus(D))
    if flags == 0:
        assert t == p.levels
    else:
        assert 1 <= t <= p.levels


def test_minplus_closure_early_exit_stops_at_fixed_point():
    # a dense graph: every shortest path has few arcs, so the squares stop
    # changing long before ceil(log2(n-1)) squarings.
    n = 1000
    D = inputs.graph_minplus(n, seed=70, density=0.5, hi=1000)
    C, t, p = closure(MP, D, flags=mmsr.MM_CLOSURE_EARLY_EXIT)
    assert t < p.levels
    np.testing.assert_array_equal(C.astype(np.int64), oracle.closure_minplus(D))


def test_minplus_closure_long_distances_leave_packed_range():
    # a long path of heavy arcs: distances grow past the packed 16-bit range
    # between squarings, so later squarings must take the 32-bit leaf.
    n = 200
    D = np.full((n, n), mmsr.INF, dtype=np.int32)
    for i in range(n - 1):
        D[i, i + 1] = 900 + (i % 50)
    C, _, _ = closure(MP, D)
    ref = oracle.closure_minplus(D)
    assert ref[0, n - 1] > 16383
    np.testing.assert_array_equal(C.astype(np.int64), ref)


def test_minplus_closure_in_place_and_sentinel():
    n = 64
    D = np.full((n, n), mmsr.INF, dtype=np.int32)  # no arcs at all
    C, _, _ = closure(MP, D, in_place=True)
    np.testing.assert_array_equal(C.astype(np.int64), oracle.closure_minplus(D))
    D = inputs.graph_minplus(n, seed=71, density=0.1, hi=1000)
    C, _, _ = closure(MP, D, in_place=True)
    np.testing.assert_array_equal(C.astype(np.int64), oracle.closure_minplus(D))


@pytest.mark.parametrize("n", [1, 5, 33, 130, 517])
@pytest.mark.parametrize("flags", [0, mmsr.MM_CLOSURE_EARLY_EXIT])
def test_orand_closure_exact(n, flags):
    A, _ = inputs.boolean_u8(n, n, 1, seed=80 + n, density=1.5 / max(n, 1))
    A = A * 5  # nonzero = arc
    C, t, p = closure(OA, A, flags=flags)
    np.testing.assert_array_equal(C, oracle.closure_orand(A))
    if flags == 0:
        assert t == p.levels


@pytest.mark.parametrize("flags", [0, mmsr.MM_CLOSURE_EARLY_EXIT])
def test_closure_full_size_n4096_sampled_rows(flags):
    # the (min,+) product's operand as a graph: 4096 vertices, 10% arcs with
    # weights in [0, 1000]; sampled rows against one Dijkstra per source.
    import torch

    n = 4096
    rng = np.random.default_rng(1)
    D = rng.integers(0, 1001, size=(n, n)).astype(np.int32)
    D[rng.random((n, n)) >= 0.1] = mmsr.INF
    C, t, p = closure(MP, D, extra_parts=1, flags=flags)
    assert p.levels == 12 and (t == 12 if flags == 0 else 1 <= t < 12)
    rows = oracle.sample_rows(n)
    np.testing.assert_array_equal(C[rows].astype(np.int64), oracle.closure_minplus_rows(D, rows))
    torch.cuda.empty_cache()
