"""FP32-mode (+,x): bf16x3 split products on tcgen05 tensor cores vs the FP64
oracle.  Tolerance: relative Frobenius error <= 1e-5; integer-valued inputs
whose products and sums are exact in bf16 / fp32 must match bit for bit."""
import numpy as np
import pytest

import oracle
from paper_1911_05328_gb300 import inputs, mmsr

from gpu_util import canary_intact, dev, empty, rel_fro, workspace

pytestmark = pytest.mark.gpu
SR = mmsr.MM_SR_PLUS_TIMES_F32
TOL = 1e-5


def run(A, B, extra_parts=0):
    import torch

    m, k = A.shape
    n = B.shape[1]
    p0 = mmsr.mm_plan_query(SR, -1, m, n, k, 0)
    budget = int(p0.workspace_min) + extra_parts * m * n * 4
    ws = workspace(budget)
    dC = empty((m, n), torch.float32)
    mmsr.mm_semiring(SR, m, n, k, dev(A.astype(np.float32)), dev(B.astype(np.float32)), dC, ws, budget)
    torch.cuda.synchronize()
    assert canary_intact(ws, budget)
    assert mmsr.mm_last_device_status() == 0
    return dC.cpu().numpy()


def test_tiny_integer_tile_exact():
    A, B = inputs.small_int(128, 64, 256, seed=50, dtype=np.float32)
    np.testing.assert_array_equal(run(A, B), oracle.mm_f64(A, B).astype(np.float32))


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (128, 256, 64), (129, 257, 65), (300, 200, 1000), (256, 512, 2048),
                                   (389, 300, 500)])
def test_integer_inputs_exact(m, n, k):
    A, B = inputs.small_int(m, k, n, seed=m + n + k, bound=4, dtype=np.float32)
    np.testing.assert_array_equal(run(A, B), oracle.mm_f64(A, B).astype(np.float32))


@pytest.mark.parametrize("m,n,k", [(128, 256, 64), (200, 300, 777), (512, 512, 4096), (1000, 1100, 1200)])
def test_normal_inputs_tolerance(m, n, k):
    A, B = inputs.normal_f32(m, k, n, seed=m * 3 + k)
    err = rel_fro(run(A, B), oracle.mm_f64(A, B))
    assert err <= TOL, err


@pytest.mark.parametrize("parts", [1, 2, 5])
def test_split_k(parts):
    m, n, k = 256, 384, 2048
    A, B = inputs.normal_f32(m, k, n, seed=60 + parts)
    err = rel_fro(run(A, B, extra_parts=parts), oracle.mm_f64(A, B))
    assert err <= TOL, err


def test_workspace_below_minimum_rejected():
    import torch

    m = n = k = 256
    p = mmsr.mm_plan_query(SR, -1, m, n, k, 0)
    assert p.workspace_min == 4 * 256 * (m + n)
    ws = empty((int(p.workspace_min),), torch.uint8)
    dA = empty((m, k), torch.float32)
    rc = mmsr.mm_semiring(SR, m, n, k, dA, dA, dA, ws, int(p.workspace_min) - 16, check=False)
    assert rc == mmsr.MM_ERR_WORKSPACE


def test_k_zero_writes_zero():
    import torch

    dC = empty((3, 5), torch.float32)
    dC.fill_(9.0)
    p = mmsr.mm_plan_query(SR, -1, 3, 5, 0, 0)
    ws = empty((int(p.workspace_min),), torch.uint8)
    mmsr.mm_semiring(SR, 3, 5, 0, empty((3, 1), torch.float32), empty((1, 5), torch.float32), dC, ws,
                     int(p.workspace_min))
    torch.cuda.synchronize()
    assert np.all(dC.cpu().numpy() == 0.0)


def test_full_size_n8192_sampled_rows():
    import torch

    n = 8192
    A, B = inputs.normal_f32(n, n, n, seed=2)
    C = run(A, B)
    rows = oracle.sample_rows(n)
    ref = oracle.mm_f64(A, B, rows=rows)
    err = rel_fro(C[rows], ref)
    assert err <= TOL, err
    torch.cuda.empty_cache()


def _sk_budget(m, n, k):
    """Smallest budget for which the planner picks the FP32 stream-K form
    (kernel id 5): the split operands plus two partial tiles per CTA and one
    counter per tile."""
    base = int(mmsr.mm_plan_query(SR, -1, m, n, k, 0).workspace_min)
    for extra in (1 << 26, 1 << 28):
        p = mmsr.mm_plan_query(SR, -1, m, n, k, base + extra)
        if p.kernel == 5:
            return int(p.workspace_used)
    return None


def run_budget(A, B, budget):
    import torch

    m, k = A.shape
    n = B.shape[1]
    ws = workspace(budget)
    dC = empty((m, n), torch.float32)
    dC.fill_(float("nan"))  # every tile must be written, whole or folded
    mmsr.mm_semiring(SR, m, n, k, dev(A.astype(np.float32)), dev(B.astype(np.float32)), dC, ws, budget)
    torch.cuda.synchronize()
    assert canary_intact(ws, budget)
    assert mmsr.mm_last_device_status() == 0
    return dC.cpu().numpy()


@pytest.fixture
def f32_streamk_mode(request):
    mmsr.mm_set_option(mmsr.MM_OPT_F32_STREAMK, request.param)
    yield request.param
    mmsr.mm_set_option(mmsr.MM_OPT_F32_STREAMK, 1)


@pytest.mark.parametrize("f32_streamk_mode", [2, 3], indirect=True)
@pytest.mark.parametrize("m,n,k", [(2048, 4096, 2048), (2200, 4100, 777), (2560, 4096, 4096)])
def test_streamk_form_matches_oracle(m, n, k, f32_streamk_mode):
    # one to four waves of 128 x 256 tiles: persistent CTAs take the whole
    # waves tile by tile and split the (tile, k-block) units of the tiles left
    # over evenly; partial tiles meet in per-CTA slots, folded in k order by
    # the last CTA to arrive (sampled rows, incl. tile edges).  2200 x 4100 x
    # 777 leaves two tiles of thirteen k-blocks over three CTAs when the
    # whole waves run first (mode 3); mode 2 splits every tile's units.
    w = _sk_budget(m, n, k)
    assert w is not None
    rows = oracle.sample_rows(m, 256)
    A, B = inputs.small_int(m, k, n, seed=m + n + k, bound=4, dtype=np.float32)
    np.testing.assert_array_equal(run_budget(A, B, w)[rows], oracle.mm_f64(A, B, rows=rows).astype(np.float32))
    A, B = inputs.normal_f32(m, k, n, seed=3 * m + k)
    C1 = run_budget(A, B, w)
    assert rel_fro(C1[rows], oracle.mm_f64(A, B, rows=rows)) <= TOL
    np.testing.assert_array_equal(run_budget(A, B, w), C1)  # fixed fold order: repeatable
    # and the same product through split-K with that budget's slices
    base = int(mmsr.mm_plan_query(SR, -1, m, n, k, 0).workspace_min)
    C2 = run_budget(A, B, base + m * n * 4)
    assert rel_fro(C1[rows], C2[rows].astype(np.float64)) <= 2 * TOL


@pytest.mark.parametrize("f32_streamk_mode", [2, 3], indirect=True)
def test_streamk_whole_waves_only(f32_streamk_mode):
    # exactly two waves of 128 x 256 tiles: every CTA takes two whole tiles
    # and no stream-K range is left, so no slot is written and the result
    # equals the classic grid's bit for bit (same per-tile k order)
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    m, n, k = 128 * sms, 512, 1024
    w = _sk_budget(m, n, k)
    assert w is not None
    A, B = inputs.normal_f32(m, k, n, seed=91)
    C1 = run_budget(A, B, w)
    base = int(mmsr.mm_plan_query(SR, -1, m, n, k, 0).workspace_min)
    np.testing.assert_array_equal(C1, run_budget(A, B, base))
    rows = oracle.sample_rows(m, 256)
    assert rel_fro(C1[rows], oracle.mm_f64(A, B, rows=rows)) <= TOL


def test_streamk_planner_rule():
    # the planner's own choice (option 1): stream-K only when the classic
    # grid's last wave would be nearly empty -- 1.05 waves of 128 x 256 tiles
    # yes, 1.68 waves no (the budget then buys split-K); more than four waves:
    # the classic grid; under one wave: split-K, which the same budget always
    # buys enough slices of
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    m, k = 2048, 2048
    n_few = 256 * -(-(sms + sms // 20) // 16)  # just over one wave of 16-row columns
    assert _sk_budget(m, n_few, k) is not None
    base = int(mmsr.mm_plan_query(SR, -1, m, 4096, k, 0).workspace_min)
    if (16 * 16) % sms > 0.3 * sms:
        assert mmsr.mm_plan_query(SR, -1, m, 4096, k, base + (1 << 28)).kernel == 2
    assert mmsr.mm_plan_query(SR, -1, 8192, 8192, 8192, 1 << 34).kernel == 2
    base = int(mmsr.mm_plan_query(SR, -1, 1024, 1024, 16384, 0).workspace_min)
    p = mmsr.mm_plan_query(SR, -1, 1024, 1024, 16384, base + (1 << 28))
    assert p.kernel == 2 and p.split_k > 1
    w = _sk_budget(m, n_few, k)
    assert mmsr.mm_plan_query(SR, -1, m, n_few, k, w - 1).kernel == 2
    mmsr.mm_set_option(mmsr.MM_OPT_F32_STREAMK, 0)
    try:
        assert mmsr.mm_plan_query(SR, -1, m, n_few, k, w).kernel == 2
    finally:
        mmsr.mm_set_option(mmsr.MM_OPT_F32_STREAMK, 1)