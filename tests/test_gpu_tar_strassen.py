"""TAR-Strassen (one or two levels, leaf products added straight into the
blocks of C by the leaf epilogue in conflict-free waves; FP32 and
FP64-accuracy modes) vs the oracle."""
import numpy as np
import pytest

import oracle
from paper_1911_05328_gb300 import inputs, mmsr

from error_bounds import FP32_TOL, fp32_strassen_tol
from gpu_util import canary_intact, dev, empty, rel_fro, workspace

pytestmark = pytest.mark.gpu
F32, FA = mmsr.MM_SR_PLUS_TIMES_F32, mmsr.MM_SR_PLUS_TIMES_F64ACC
PAPER, WINO = mmsr.MM_STRASSEN_PAPER, mmsr.MM_STRASSEN_WINOGRAD
# (levels, variant): two Winograd levels are refused (a product would reach
# all sixteen blocks)
PLANS = [(1, PAPER), (1, WINO), (2, PAPER)]


def run_tar(variant, A, B, levels=1, sr=F32):
    import torch

    m, k = A.shape
    n = B.shape[1]
    p = mmsr.mm_strassen_tar_query(levels, sr, m, n, k)
    budget = int(p.workspace_min)
    ws = workspace(budget)
    dt = torch.float32 if sr == F32 else torch.float64
    npt = np.float32 if sr == F32 else np.float64
    dC = empty((m, n), dt)
    dC.fill_(float("nan"))  # every block's first writer must overwrite
    mmsr.mm_strassen_tar(levels, variant, sr, m, n, k, dev(A.astype(npt)), dev(B.astype(npt)), dC, ws, budget)
    torch.cuda.synchronize()
    assert canary_intact(ws, budget)
    assert mmsr.mm_last_device_status() == 0
    return dC.cpu().numpy()


@pytest.mark.parametrize("levels,variant", PLANS)
@pytest.mark.parametrize("m,k,n", [(256, 256, 256), (512, 384, 768), (4, 4, 4), (24, 16, 12), (132, 68, 264),
                                   (1000, 2052, 516)])
def test_integer_inputs_exact(levels, variant, m, k, n):
    A, B = inputs.small_int(m, k, n, seed=m + 3 * k + 7 * n, bound=3, dtype=np.float32)
    np.testing.assert_array_equal(run_tar(variant, A, B, levels), oracle.mm_f64(A, B).astype(np.float32))


@pytest.mark.parametrize("levels,variant", PLANS)
@pytest.mark.parametrize("m,k,n", [(256, 256, 256), (132, 68, 264), (520, 1028, 388)])
def test_f64acc_integer_inputs_exact(levels, variant, m, k, n):
    # FP64-accuracy mode: every digit product and sum exact
    A, B = inputs.small_int(m, k, n, seed=5 * m + k + n, bound=50, dtype=np.float64)
    np.testing.assert_array_equal(run_tar(variant, A, B, levels, FA), oracle.mm_f64(A, B))


@pytest.mark.parametrize("levels,variant", PLANS)
def test_uniform_error_within_bound(levels, variant):
    m, k, n = 1024, 2048, 768
    A, B = inputs.uniform_f64(m, k, n, seed=3)
    A32, B32 = A.astype(np.float32), B.astype(np.float32)
    err = rel_fro(run_tar(variant, A32, B32, levels), oracle.mm_f64(A32, B32))
    print("tar-strassen L%d variant %d rel_fro %.3e" % (levels, variant, err))
    # the paper's formulas at one level meet the plain FP32-mode tolerance;
    # otherwise the derived Strassen tolerance 1e-5 (g/2)^L
    tol = FP32_TOL if (levels, variant) == (1, PAPER) else fp32_strassen_tol(variant, levels)
    assert err <= tol, err


@pytest.mark.parametrize("levels,variant", PLANS)
def test_f64acc_uniform_error(levels, variant):
    # FP64-accuracy mode must meet 1e-12 with the products added into C
    m, k, n = 1024, 2048, 768
    A, B = inputs.uniform_f64(m, k, n, seed=4)
    err = rel_fro(run_tar(variant, A, B, levels, FA), oracle.mm_f64(A, B))
    print("tar-strassen f64acc L%d variant %d rel_fro %.3e" % (levels, variant, err))
    assert err <= 1e-12, err


def test_same_result_class_as_stored_products():
    # normal inputs: TAR and the stored-product level agree to FP32 rounding
    import torch

    m = k = n = 512
    A, B = inputs.normal_f32(m, k, n, seed=7)
    tar = run_tar(WINO, A, B)
    p = mmsr.mm_plan_query(F32, 1, m, n, k, 0)
    ws = workspace(int(p.workspace_min))
    dC = empty((m, n), torch.float32)
    mmsr.mm_strassen(1, WINO, F32, m, n, k, dev(A), dev(B), dC, ws, int(p.workspace_min))
    torch.cuda.synchronize()
    ref = oracle.mm_f64(A, B)
    tol = fp32_strassen_tol(WINO, 1)
    assert rel_fro(dC.cpu().numpy(), ref) <= tol
    assert rel_fro(tar, ref) <= tol
    # same leaf products, different summation into C: the two differ by at
    # most the sum of their bounds
    assert rel_fro(tar, dC.cpu().numpy()) <= 2 * tol


def test_two_winograd_levels_refused():
    import torch

    d = empty((64, 64), torch.float32)
    ws = workspace(1 << 20)
    rc = mmsr.mm_strassen_tar(2, WINO, F32, 64, 64, 64, d, d, d, ws, 1 << 20, check=False)
    assert rc == mmsr.MM_ERR_UNSUPPORTED


def test_full_size_n16384_sampled_rows():
    import torch

    n = 16384
    A, B = inputs.uniform_f64(n, n, n, seed=3)
    A, B = A.astype(np.float32), B.astype(np.float32)
    C = run_tar(WINO, A, B)
    rows = oracle.sample_rows(n, 128)
    err = rel_fro(C[rows], oracle.mm_f64(A, B, rows=rows))
    print("n16384 tar-strassen winograd rel_fro %.3e" % err)
    assert err <= fp32_strassen_tol(WINO, 1), err
    torch.cuda.empty_cache()


@pytest.mark.parametrize("levels,variant", [(1, WINO), (2, PAPER)])
def test_f64acc_n8192_sampled_rows(levels, variant):
    import torch

    n = 8192
    A, B = inputs.uniform_f64(n, n, n, seed=3)
    C = run_tar(variant, A, B, levels, FA)
    rows = oracle.sample_rows(n, 64)
    err = rel_fro(C[rows], oracle.mm_f64(A, B, rows=rows))
    print("n8192 tar-strassen f64acc L%d rel_fro %.3e" % (levels, err))
    assert err <= 1e-12, err
    torch.cuda.empty_cache()
