"""STAR-Strassen-1 mixed plans (classic in-place levels over Strassen levels),
ragged Strassen shapes and the wide top-level sum, vs the oracle."""
import numpy as np
import pytest

import oracle
from paper_1911_05328_gb300 import inputs, mmsr

from error_bounds import FP32_TOL, fp32_strassen_tol
from gpu_util import canary_intact, dev, empty, rel_fro, workspace

pytestmark = pytest.mark.gpu
F32 = mmsr.MM_SR_PLUS_TIMES_F32
F64 = mmsr.MM_SR_PLUS_TIMES_F64
F64ACC = mmsr.MM_SR_PLUS_TIMES_F64ACC
VARIANTS = [mmsr.MM_STRASSEN_PAPER, mmsr.MM_STRASSEN_WINOGRAD]


def run_star(c, L, variant, sr, A, B, extra=0):
    import torch

    m, k = A.shape
    n = B.shape[1]
    p = mmsr.mm_star_strassen_query(c, L, sr, m, n, k)
    budget = int(p.workspace_min) + extra
    ws = workspace(budget)
    dt = torch.float32 if sr == F32 else torch.float64
    npdt = np.float32 if sr == F32 else np.float64
    dC = empty((m, n), dt)
    dC.fill_(float("nan"))  # the first block products must overwrite, not add
    mmsr.mm_star_strassen(c, L, variant, sr, m, n, k, dev(A.astype(npdt)), dev(B.astype(npdt)), dC, ws, budget)
    torch.cuda.synchronize()
    assert canary_intact(ws, budget)
    assert mmsr.mm_last_device_status() == 0
    return dC.cpu().numpy()


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("c,L,m,k,n", [(1, 1, 256, 256, 256), (2, 1, 512, 256, 384), (1, 2, 512, 512, 256),
                                       (1, 3, 512, 512, 512), (2, 2, 1024, 512, 512)])
def test_fp32_integer_inputs_exact(variant, c, L, m, k, n):
    A, B = inputs.small_int(m, k, n, seed=90 + 4 * c + L, bound=2, dtype=np.float32)
    C = run_star(c, L, variant, F32, A, B)
    np.testing.assert_array_equal(C, oracle.mm_f64(A, B).astype(np.float32))


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("c,L", [(1, 1), (1, 2), (2, 1)])
def test_fp64_modes(variant, c, L):
    m, k, n = 256, 512, 384
    A, B = inputs.small_int(m, k, n, seed=95 + c + L, bound=5)
    np.testing.assert_array_equal(run_star(c, L, variant, F64, A, B), oracle.mm_f64(A, B))
    A, B = inputs.uniform_f64(m, k, n, seed=3)
    ref = oracle.mm_f64(A, B)
    assert rel_fro(run_star(c, L, variant, F64, A, B), ref) <= 1e-12
    assert rel_fro(run_star(c, L, variant, F64ACC, A, B), ref) <= 1e-12


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("c,L", [(1, 1), (1, 2), (2, 2), (1, 3)])
def test_fp32_uniform_error_matches_pure_strassen_bound(variant, c, L):
    # the classic levels grow the worst-case bound by 2 per level at half the
    # inner dimension (a factor 1 in all): the tolerance is that of L
    # Strassen levels; the paper's formulas at one level meet plain 1e-5
    m, k, n = 1024, 2048, 768
    A, B = inputs.uniform_f64(m, k, n, seed=3)
    A32, B32 = A.astype(np.float32), B.astype(np.float32)
    err = rel_fro(run_star(c, L, variant, F32, A32, B32), oracle.mm_f64(A32, B32))
    print("fp32 star-strassen variant %d c %d L %d rel_fro %.3e" % (variant, c, L, err))
    assert err <= fp32_strassen_tol(variant, L), err
    if variant == mmsr.MM_STRASSEN_PAPER and L == 1:
        assert err <= FP32_TOL, err


@pytest.mark.parametrize("sr", [F32, F64])
@pytest.mark.parametrize("c,L,m,k,n", [(0, 2, 20, 28, 44), (1, 1, 52, 28, 44), (1, 2, 24, 40, 56),
                                       (2, 1, 40, 56, 24)])
def test_ragged_blocks_take_the_scalar_paths(sr, c, L, m, k, n):
    # block and leaf widths that are not multiples of the 16-byte vector
    # (odd leaves: 5, 7, 11, 3 ...), exact on small integers.
    npdt = np.float32 if sr == F32 else np.float64
    A, B = inputs.small_int(m, k, n, seed=m + k + n, bound=3, dtype=npdt)
    C = run_star(c, L, mmsr.MM_STRASSEN_WINOGRAD, sr, A, B)
    np.testing.assert_array_equal(C, oracle.mm_f64(A, B).astype(npdt))


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("L", [3, 4])
def test_double_float_top_sum_equals_fp64_sum(variant, L):
    # The top-level post-additions of FP32-mode Strassen at L >= 3 run as an
    # error-free double-float sum by default and in FP64 arithmetic with the
    # option set.  Both round the exact sum of the same FP32 products once,
    # so they agree to one unit in the last place, nearly always exactly.
    import torch

    m = k = n = 1024
    A, B = inputs.normal_f32(m, k, n, seed=5)
    p = mmsr.mm_plan_query(F32, L, m, n, k, 0)
    ws = workspace(int(p.workspace_min))
    dA, dB = dev(A), dev(B)
    out = []
    try:
        for opt in (0, 1):
            mmsr.mm_set_option(mmsr.MM_OPT_STRASSEN_TOP_F64, opt)
            dC = empty((m, n), torch.float32)
            mmsr.mm_strassen(L, variant, F32, m, n, k, dA, dB, dC, ws, int(p.workspace_min))
            torch.cuda.synchronize()
            out.append(dC.cpu().numpy())
    finally:
        mmsr.mm_set_option(mmsr.MM_OPT_STRASSEN_TOP_F64, 0)
    dd, f64 = out
    ulp = np.spacing(np.abs(f64).astype(np.float32))
    assert np.all(np.abs(dd.astype(np.float64) - f64) <= ulp)
    assert np.mean(dd == f64) >= 0.999
    ref = oracle.mm_f64(A, B)
    assert abs(rel_fro(dd, ref) - rel_fro(f64, ref)) <= 1e-3 * rel_fro(f64, ref)


def test_full_size_n16384_star_sampled_rows():
    # one classic level over one Winograd level at the full size, a quarter of
    # the workspace of Strassen at that block size times four.
    import torch

    n = 16384
    A, B = inputs.uniform_f64(n, n, n, seed=3)
    A, B = A.astype(np.float32), B.astype(np.float32)
    C = run_star(1, 1, mmsr.MM_STRASSEN_WINOGRAD, F32, A, B)
    rows = oracle.sample_rows(n, 128)
    err = rel_fro(C[rows], oracle.mm_f64(A, B, rows=rows))
    print("n16384 star c 1 L 1 winograd rel_fro %.3e" % err)
    assert err <= fp32_strassen_tol(mmsr.MM_STRASSEN_WINOGRAD, 1), err
    torch.cuda.empty_cache()
