"""Plain FP64 (+,x) path on the GPU vs the FP64 oracle (rel. Frobenius
<= 1e-12), including split-K with the fixed-order FP64 reduction and the
n=256 uniform[-1,1] workload (seed 0, budget 0) in full."""
import numpy as np
import pytest

import oracle
from paper_1911_05328_gb300 import inputs, mmsr

from gpu_util import canary_intact, dev, empty, rel_fro, workspace

pytestmark = pytest.mark.gpu
SR = mmsr.MM_SR_PLUS_TIMES_F64
TOL = 1e-12


def run(A, B, budget=0):
    import torch

    m, k = A.shape
    n = B.shape[1]
    dC = empty((m, n), torch.float64)
    ws = workspace(budget)
    mmsr.mm_semiring(SR, m, n, k, dev(A), dev(B), dC, ws if budget else None, budget)
    torch.cuda.synchronize()
    assert canary_intact(ws, budget)
    return dC.cpu().numpy()


def test_n256_workload_full():
    A, B = inputs.uniform_f64(256, 256, 256, seed=0)
    assert rel_fro(run(A, B), oracle.mm_f64(A, B)) <= TOL


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (7, 5, 3), (64, 64, 16), (65, 67, 33), (200, 130, 513), (512, 384, 1024)])
def test_shapes(m, n, k):
    A, B = inputs.uniform_f64(m, k, n, seed=m * 7 + n + k)
    assert rel_fro(run(A, B), oracle.mm_f64(A, B)) <= TOL


@pytest.mark.parametrize("parts", [2, 3, 7])
def test_split_k(parts):
    m, n, k = 192, 160, 2000
    A, B = inputs.uniform_f64(m, k, n, seed=40 + parts)
    budget = (parts - 1) * m * n * 8
    assert mmsr.mm_plan_query(SR, -1, m, n, k, budget).split_k == parts
    assert rel_fro(run(A, B, budget), oracle.mm_f64(A, B)) <= TOL


def test_small_integers_exact():
    A, B = inputs.small_int(130, 300, 70, seed=41)
    np.testing.assert_array_equal(run(A, B, 2 * 130 * 70 * 8), oracle.mm_f64(A, B))


def test_k_zero_writes_zero():
    import torch

    dC = empty((3, 4), torch.float64)
    dC.fill_(7.0)
    mmsr.mm_semiring(SR, 3, 4, 0, empty((3, 1), torch.float64), empty((1, 4), torch.float64), dC)
    torch.cuda.synchronize()
    assert np.all(dC.cpu().numpy() == 0.0)


@pytest.fixture
def sk_forced():
    # the stream-K form wherever it applies (option 2), not only where the
    # planner's rule takes it
    mmsr.mm_set_option(mmsr.MM_OPT_F64_STREAMK, 2)
    yield
    mmsr.mm_set_option(mmsr.MM_OPT_F64_STREAMK, 1)


def _streamk_budget(m, n, k):
    """Smallest budget for which the planner picks the stream-K form (the
    per-CTA partial tiles plus one counter per tile), or None when the
    product is too large or too shallow for it."""
    for b in (1 << 20, 1 << 22, 1 << 24, 1 << 26):
        p = mmsr.mm_plan_query(SR, -1, m, n, k, b)
        if p.kernel == 6:
            return int(p.workspace_used)
    return None


@pytest.mark.parametrize("m,n,k", [(256, 256, 256), (1, 1, 100), (33, 65, 77), (130, 257, 1000), (100, 40, 4096),
                                   (512, 512, 64), (600, 700, 300)])
def test_streamk_form_matches_oracle(m, n, k, sk_forced):
    # the zero-temporary k-parallel form (Fig. tar-mm): per-CTA partial tiles
    # folded in k order by the last CTA to arrive; ragged tiles and k tails
    w = _streamk_budget(m, n, k)
    assert w is not None
    A, B = inputs.uniform_f64(m, k, n, seed=m + 3 * n + 7 * k)
    C1 = run(A, B, w)
    assert rel_fro(C1, oracle.mm_f64(A, B)) <= TOL
    # fixed summation order: identical on a second run
    np.testing.assert_array_equal(run(A, B, w), C1)


def test_streamk_small_integers_exact(sk_forced):
    m, n, k = 200, 190, 3000
    A, B = inputs.small_int(m, k, n, seed=43)
    w = _streamk_budget(m, n, k)
    np.testing.assert_array_equal(run(A, B, w), oracle.mm_f64(A, B))


def test_streamk_n256_workload(sk_forced):
    # the n = 256 uniform[-1,1] workload (seed 0) in the stream-K form,
    # beside the budget-0 path of the same product
    A, B = inputs.uniform_f64(256, 256, 256, seed=0)
    w = _streamk_budget(256, 256, 256)
    assert w <= 9 << 20  # p b^2: the partial tiles of a few hundred CTAs
    ref = oracle.mm_f64(A, B)
    assert rel_fro(run(A, B, w), ref) <= TOL
    assert rel_fro(run(A, B, 0), ref) <= TOL


def test_streamk_not_taken_for_large_grids_or_small_budgets(sk_forced):
    assert mmsr.mm_plan_query(SR, -1, 4096, 4096, 4096, 1 << 30).kernel != 6
    w = _streamk_budget(256, 256, 256)
    assert mmsr.mm_plan_query(SR, -1, 256, 256, 256, w - 1).kernel != 6
    assert mmsr.mm_plan_query(SR, -1, 256, 256, 256, 0).kernel != 6


def test_streamk_planner_rule():
    # the planner's own rule (option 1): not at n = 256, whose 8 x 8 tiles
    # already balance; yes just past one wave of two 64 x 64 CTAs per SM
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert mmsr.mm_plan_query(SR, -1, 256, 256, 256, 1 << 26).kernel != 6
    tiles = 2 * sms + max(1, sms // 10)
    m, n, k = 64 * tiles, 64, 2048
    assert mmsr.mm_plan_query(SR, -1, m, n, k, 1 << 28).kernel == 6
    mmsr.mm_set_option(mmsr.MM_OPT_F64_STREAMK, 0)
    try:
        assert mmsr.mm_plan_query(SR, -1, m, n, k, 1 << 28).kernel != 6
    finally:
        mmsr.mm_set_option(mmsr.MM_OPT_F64_STREAMK, 1)