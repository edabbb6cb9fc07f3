"""One FP32-mode Strassen level with the operand sums formed in the leaf's
staging (MM_OPT_STRASSEN_FUSED): the converter warps add the source
quadrants in the level passes' order and split them as the passes do, so the
result must equal the materialised path bit for bit; integer inputs are exact
against the oracle; a STAR-Strassen-1 plan over it agrees too."""
import numpy as np
import pytest

import oracle
from paper_1911_05328_gb300 import inputs, mmsr

from error_bounds import fp32_strassen_tol
from gpu_util import canary_intact, dev, empty, rel_fro, workspace

pytestmark = pytest.mark.gpu
F32 = mmsr.MM_SR_PLUS_TIMES_F32
VARIANTS = [mmsr.MM_STRASSEN_PAPER, mmsr.MM_STRASSEN_WINOGRAD]


def run(variant, A, B, fused, star_classic=0):
    import torch

    m, k = A.shape
    n = B.shape[1]
    mmsr.mm_set_option(mmsr.MM_OPT_STRASSEN_FUSED, 1 if fused else 0)
    try:
        if star_classic:
            p = mmsr.mm_star_strassen_query(star_classic, 1, F32, m, n, k)
        else:
            p = mmsr.mm_plan_query(F32, 1, m, n, k, 0)
        budget = int(p.workspace_min)
        ws = workspace(budget)
        dC = empty((m, n), torch.float32)
        dC.fill_(float("nan"))
        if star_classic:
            mmsr.mm_star_strassen(star_classic, 1, variant, F32, m, n, k, dev(A), dev(B), dC, ws, budget)
        else:
            mmsr.mm_strassen(1, variant, F32, m, n, k, dev(A), dev(B), dC, ws, budget)
        torch.cuda.synchronize()
        assert canary_intact(ws, budget)
        assert mmsr.mm_last_device_status() == 0
        return dC.cpu().numpy(), budget
    finally:
        mmsr.mm_set_option(mmsr.MM_OPT_STRASSEN_FUSED, 0)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("m,k,n", [(256, 64, 256), (512, 512, 512), (1024, 2048, 768), (768, 320, 1280)])
def test_fused_equals_materialised(variant, m, k, n):
    A, B = inputs.normal_f32(m, k, n, seed=m + 2 * k + 3 * n)
    Cf, wf = run(variant, A, B, True)
    Cm, wm = run(variant, A, B, False)
    np.testing.assert_array_equal(Cf, Cm)
    assert wf < wm  # the product stack alone
    assert rel_fro(Cf, oracle.mm_f64(A, B)) <= fp32_strassen_tol(variant, 1)


@pytest.mark.parametrize("variant", VARIANTS)
def test_fused_integer_inputs_exact(variant):
    A, B = inputs.small_int(512, 384, 256, seed=77, bound=3, dtype=np.float32)
    np.testing.assert_array_equal(run(variant, A, B, True)[0], oracle.mm_f64(A, B).astype(np.float32))


def test_fused_under_star_plan():
    # one classic in-place level over the fused Strassen level (strided
    # block views, accumulation into C)
    A, B = inputs.normal_f32(1024, 1024, 1024, seed=78)
    Cf, _ = run(mmsr.MM_STRASSEN_WINOGRAD, A, B, True, star_classic=1)
    Cm, _ = run(mmsr.MM_STRASSEN_WINOGRAD, A, B, False, star_classic=1)
    np.testing.assert_array_equal(Cf, Cm)


def test_fused_falls_back_on_other_shapes():
    # 200 x 130 leaves do not tile by 128: the materialised path runs
    A, B = inputs.normal_f32(400, 128, 260, seed=79)
    Cf, wf = run(mmsr.MM_STRASSEN_WINOGRAD, A, B, True)
    Cm, wm = run(mmsr.MM_STRASSEN_WINOGRAD, A, B, False)
    assert wf == wm
    np.testing.assert_array_equal(Cf, Cm)
