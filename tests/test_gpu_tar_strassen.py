"""TAR-Strassen (one level, products added straight into C's quadrants by
the leaf epilogue in conflict-free waves) vs the oracle."""
import numpy as np
import pytest

import oracle
from paper_1911_05328_gb300 import inputs, mmsr

from error_bounds import FP32_TOL, fp32_strassen_tol
from gpu_util import canary_intact, dev, empty, rel_fro, workspace

pytestmark = pytest.mark.gpu
F32 = mmsr.MM_SR_PLUS_TIMES_F32
VARIANTS = [mmsr.MM_STRASSEN_PAPER, mmsr.MM_STRASSEN_WINOGRAD]


def run_tar(variant, A, B):
    import torch

    m, k = A.shape
    n = B.shape[1]
    p = mmsr.mm_strassen_tar_query(F32, m, n, k)
    budget = int(p.workspace_min)
    ws = workspace(budget)
    dC = empty((m, n), torch.float32)
    dC.fill_(float("nan"))  # every quadrant's first writer must overwrite
    mmsr.mm_strassen_tar(variant, F32, m, n, k, dev(A.astype(np.float32)), dev(B.astype(np.float32)), dC, ws,
                         budget)
    torch.cuda.synchronize()
    assert canary_intact(ws, budget)
    assert mmsr.mm_last_device_status() == 0
    return dC.cpu().numpy()


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("m,k,n", [(256, 256, 256), (512, 384, 768), (2, 2, 2), (22, 14, 10), (130, 66, 262),
                                   (1000, 2050, 514)])
def test_integer_inputs_exact(variant, m, k, n):
    A, B = inputs.small_int(m, k, n, seed=m + 3 * k + 7 * n, bound=3, dtype=np.float32)
    np.testing.assert_array_equal(run_tar(variant, A, B), oracle.mm_f64(A, B).astype(np.float32))


@pytest.mark.parametrize("variant", VARIANTS)
def test_uniform_error_within_one_level_bound(variant):
    m, k, n = 1024, 2048, 768
    A, B = inputs.uniform_f64(m, k, n, seed=3)
    A32, B32 = A.astype(np.float32), B.astype(np.float32)
    err = rel_fro(run_tar(variant, A32, B32), oracle.mm_f64(A32, B32))
    print("tar-strassen variant %d rel_fro %.3e" % (variant, err))
    # the paper's formulas at one level meet the plain FP32-mode tolerance;
    # Winograd's are held to the derived one-level tolerance (9 x 1e-5)
    assert err <= (FP32_TOL if variant == mmsr.MM_STRASSEN_PAPER else fp32_strassen_tol(variant, 1)), err


def test_same_result_class_as_stored_products():
    # normal inputs: TAR and the stored-product level agree to FP32 rounding
    import torch

    m = k = n = 512
    A, B = inputs.normal_f32(m, k, n, seed=7)
    tar = run_tar(mmsr.MM_STRASSEN_WINOGRAD, A, B)
    p = mmsr.mm_plan_query(F32, 1, m, n, k, 0)
    ws = workspace(int(p.workspace_min))
    dC = empty((m, n), torch.float32)
    mmsr.mm_strassen(1, mmsr.MM_STRASSEN_WINOGRAD, F32, m, n, k, dev(A), dev(B), dC, ws, int(p.workspace_min))
    torch.cuda.synchronize()
    ref = oracle.mm_f64(A, B)
    tol = fp32_strassen_tol(mmsr.MM_STRASSEN_WINOGRAD, 1)
    assert rel_fro(dC.cpu().numpy(), ref) <= tol
    assert rel_fro(tar, ref) <= tol
    # same leaf products, different summation into C: the two differ by at
    # most the sum of their bounds
    assert rel_fro(tar, dC.cpu().numpy()) <= 2 * tol


def test_full_size_n16384_sampled_rows():
    import torch

    n = 16384
    A, B = inputs.uniform_f64(n, n, n, seed=3)
    A, B = A.astype(np.float32), B.astype(np.float32)
    C = run_tar(mmsr.MM_STRASSEN_WINOGRAD, A, B)
    rows = oracle.sample_rows(n, 128)
    err = rel_fro(C[rows], oracle.mm_f64(A, B, rows=rows))
    print("n16384 tar-strassen winograd rel_fro %.3e" % err)
    assert err <= fp32_strassen_tol(mmsr.MM_STRASSEN_WINOGRAD, 1), err
    torch.cuda.empty_cache()
