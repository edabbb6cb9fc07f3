"""(min,+) tropical path on the GPU vs the int64 oracle: bit-exact.

Covers the leaf kernel (k-serial in place, budget 0), split-K under every
budget of the n=4096 workload (0/1/2/4/8 extra n x n buffers) with the
min-reduction, ragged edges, tiny and empty inputs, sentinel saturation and
the workspace cap (canary bytes past the budget stay untouched)."""
import numpy as np
import pytest

import oracle
from paper_1911_05328_gb300 import inputs, mmsr

from gpu_util import canary_intact, dev, empty, workspace

pytestmark = pytest.mark.gpu
SR = mmsr.MM_SR_MIN_PLUS_I32


@pytest.fixture(params=[1, 0], ids=["packed-auto", "int32-only"])
def packed(request):
    mmsr.mm_set_option(mmsr.MM_OPT_MINPLUS_PACKED, request.param)
    yield request.param
    mmsr.mm_set_option(mmsr.MM_OPT_MINPLUS_PACKED, 1)


def run(A, B, budget=0):
    import torch

    m, k = A.shape
    n = B.shape[1]
    dA, dB = dev(A), dev(B)
    dC = empty((m, n), torch.int32)
    ws = workspace(budget)
    mmsr.mm_semiring(SR, m, n, k, dA, dB, dC, ws if budget else None, budget)
    torch.cuda.synchronize()
    assert canary_intact(ws, budget)
    return dC.cpu().numpy()


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (7, 5, 3), (64, 64, 64), (128, 128, 32), (129, 131, 67),
                                   (256, 256, 256), (130, 260, 1000), (1000, 1000, 1000), (333, 97, 4099)])
def test_leaf_matches_oracle(m, n, k, packed):
    A, B = inputs.tropical_i32(m, k, n, seed=m + n + k)
    np.testing.assert_array_equal(run(A, B), oracle.mm_minplus(A, B))


@pytest.mark.parametrize("parts", [1, 2, 3, 5, 9])
def test_split_k_budgets_bit_identical(parts, packed):
    m, n, k = 300, 260, 1440  # 45 k-blocks of 32: divisible into 1, 2, 3, 5, 9 slices
    A, B = inputs.tropical_i32(m, k, n, seed=31)
    budget = (parts - 1) * m * n * 4
    plan = mmsr.mm_plan_query(SR, -1, m, n, k, budget)
    assert plan.split_k == parts
    np.testing.assert_array_equal(run(A, B, budget), oracle.mm_minplus(A, B))


def test_budget_not_multiple_of_slice():
    m, n, k = 200, 200, 900
    A, B = inputs.tropical_i32(m, k, n, seed=32)
    budget = 2 * m * n * 4 + 1234  # 2 full buffers + change
    np.testing.assert_array_equal(run(A, B, budget), oracle.mm_minplus(A, B))


@pytest.mark.parametrize("big", [16384, 20000, (1 << 30) - 1])
def test_value_outside_packed_range_falls_back(big):
    # one finite entry above 16383 must route the call to the 32-bit leaf
    m, n, k = 200, 300, 500
    A, B = inputs.tropical_i32(m, k, n, seed=35)
    A[17, 123] = big
    B[45, 7] = big
    np.testing.assert_array_equal(run(A, B), oracle.mm_minplus(A, B))


def test_packed_range_edge_values():
    # largest packable entries: finite sums reach 32766, one below the
    # 16-bit sentinel, and must not be confused with +inf
    m, n, k = 130, 260, 70
    A = np.full((m, k), 16383, np.int32)
    B = np.full((k, n), 16383, np.int32)
    A[::3, :] = inputs.INF
    B[:, 5] = inputs.INF
    np.testing.assert_array_equal(run(A, B), oracle.mm_minplus(A, B))


def test_k_zero_is_semiring_zero():
    import torch

    dC = empty((5, 7), torch.int32)
    dC.fill_(3)
    dA = empty((5, 1), torch.int32)
    dB = empty((1, 7), torch.int32)
    mmsr.mm_semiring(SR, 5, 7, 0, dA, dB, dC)
    torch.cuda.synchronize()
    assert np.all(dC.cpu().numpy() == inputs.INF)


def test_all_sentinel_saturates():
    A = np.full((70, 90), inputs.INF, np.int32)
    B = np.full((90, 50), inputs.INF, np.int32)
    np.testing.assert_array_equal(run(A, B), np.full((70, 50), inputs.INF, np.int32))


def test_tropical_identity_and_closure():
    D = inputs.graph_minplus(200, seed=33, density=0.03)
    X = D.copy()
    for _ in range(8):
        X = run(X, X, budget=X.size * 4)
    np.testing.assert_array_equal(X.astype(np.int64), oracle.floyd_warshall(D))


def test_full_size_workload_all_budgets():
    # n = 4096, integers in [0, 1000] with 10% sentinel, seed 1: every budget
    # must reproduce the full oracle product bit for bit.
    import torch

    n = 4096
    A, B = inputs.tropical_i32(n, n, n, seed=1)
    ref = oracle.mm_minplus(A, B)
    dA, dB = dev(A), dev(B)
    dC = empty((n, n), torch.int32)
    for nb in (0, 1, 2, 4, 8):
        budget = nb * n * n * 4
        ws = workspace(budget)
        dC.fill_(-1)
        mmsr.mm_semiring(SR, n, n, n, dA, dB, dC, ws if budget else None, budget)
        torch.cuda.synchronize()
        assert canary_intact(ws, budget)
        np.testing.assert_array_equal(dC.cpu().numpy(), ref)
        del ws


@pytest.mark.parametrize("m,n,k", [(4096, 4096, 4096), (333, 97, 4099), (1000, 700, 300), (129, 257, 17), (64, 64, 5000)])
def test_streamk_zero_budget_matches(m, n, k, packed):
    # budget 0, few waves: the zero-workspace k-parallel form (register tiles
    # merged into C by atomic min) must equal the oracle bit for bit, and
    # equal the plain k-serial leaf -- for the packed 2 x 16-bit leaf and for
    # the exact 32-bit leaf
    A, B = inputs.tropical_i32(m, k, n, seed=m + 2 * n + 3 * k)
    mmsr.mm_set_option(mmsr.MM_OPT_MINPLUS_STREAMK, 1)
    C1 = run(A, B)
    mmsr.mm_set_option(mmsr.MM_OPT_MINPLUS_STREAMK, 0)
    try:
        C0 = run(A, B)
    finally:
        mmsr.mm_set_option(mmsr.MM_OPT_MINPLUS_STREAMK, 1)
    ref = oracle.mm_minplus(A, B) if m * n * k <= 2 ** 33 else None
    np.testing.assert_array_equal(C1, C0)
    if ref is not None:
        np.testing.assert_array_equal(C1, ref)
