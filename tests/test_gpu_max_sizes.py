"""Products at the largest dimension the C ABI accepts (2^22 per dimension),
one dimension at a time: tall (m = 2^22), wide (n = 2^22) and deep
(k = 2^22), for every semiring, on sampled rows against the oracle.  These
shapes push launch grids past the 65535 limit of their y extent (row tiles
of the FP64 leaf, column tiles of the transposing operand passes), which
the kernels cover by looping; the deep shape also runs the largest split-K
factor the planner uses (64)."""
import numpy as np
import pytest

import oracle
from paper_1911_05328_gb300 import inputs, mmsr

from gpu_util import dev, empty, rel_fro, workspace

pytestmark = pytest.mark.gpu
MAXD = 1 << 22
SHAPES = {"tall": (MAXD, 16, 16), "wide": (16, MAXD, 16), "deep": (16, 16, MAXD)}


def _inputs(sr, m, n, k, seed):
    if sr == mmsr.MM_SR_MIN_PLUS_I32:
        return inputs.tropical_i32(m, k, n, seed=seed)
    if sr == mmsr.MM_SR_OR_AND_U8:
        # density so that about half the outputs are true
        return inputs.boolean_u8(m, k, n, seed=seed, density=float(min(0.3, np.sqrt(0.7 / k))))
    if sr == mmsr.MM_SR_PLUS_TIMES_F32:
        return inputs.normal_f32(m, k, n, seed=seed)
    return inputs.uniform_f64(m, k, n, seed=seed)


def _check(sr, C, A, B, rows):
    if sr == mmsr.MM_SR_MIN_PLUS_I32:
        np.testing.assert_array_equal(C[rows], oracle.mm_minplus(A, B, rows=rows))
    elif sr == mmsr.MM_SR_OR_AND_U8:
        np.testing.assert_array_equal(C[rows], oracle.mm_orand(A, B, rows=rows))
    else:
        ref = oracle.mm_f64(A, B, rows=rows)
        tol = 1e-5 if sr == mmsr.MM_SR_PLUS_TIMES_F32 else 1e-12
        assert rel_fro(C[rows], ref) <= tol


DTYPES = {mmsr.MM_SR_PLUS_TIMES_F64: "float64", mmsr.MM_SR_PLUS_TIMES_F32: "float32",
          mmsr.MM_SR_PLUS_TIMES_F64ACC: "float64", mmsr.MM_SR_MIN_PLUS_I32: "int32",
          mmsr.MM_SR_OR_AND_U8: "uint8"}
ACC = {mmsr.MM_SR_PLUS_TIMES_F64: 8, mmsr.MM_SR_PLUS_TIMES_F32: 4, mmsr.MM_SR_PLUS_TIMES_F64ACC: 8,
       mmsr.MM_SR_MIN_PLUS_I32: 4, mmsr.MM_SR_OR_AND_U8: 1}


@pytest.mark.parametrize("shape", list(SHAPES))
@pytest.mark.parametrize("sr", list(DTYPES), ids=["f64", "f32", "f64acc", "minplus", "orand"])
def test_largest_dimension(sr, shape):
    import torch

    m, n, k = SHAPES[shape]
    A, B = _inputs(sr, m, n, k, seed=41)
    wmin = int(mmsr.mm_plan_query(sr, -1, m, n, k, 0).workspace_min)
    # the deep shape also takes the largest split-K factor (64 slices)
    budget = wmin + (63 * m * n * ACC[sr] if shape == "deep" else 0)
    if shape == "deep":
        assert mmsr.mm_plan_query(sr, -1, m, n, k, budget).split_k == 64
    ws = workspace(budget)
    dC = empty((m, n), getattr(torch, DTYPES[sr]))
    mmsr.mm_semiring(sr, m, n, k, dev(A), dev(B), dC, ws, budget)
    torch.cuda.synchronize()
    assert mmsr.mm_last_device_status() == 0
    C = dC.cpu().numpy()
    rows = oracle.sample_rows(m, 256) if m > 256 else np.arange(m)
    _check(sr, C, A, B, rows)


@pytest.mark.parametrize("levels", [1, 2])
def test_strassen_widest(levels):
    # FP32-mode Strassen-Winograd with n = 2^22: the transposing operand
    # passes of one and two levels cover 2^21 / 2^20 columns of B
    import torch

    m, n, k = 16, MAXD, 16
    A, B = inputs.small_int(m, k, n, seed=42, bound=4, dtype=np.float32)
    sr = mmsr.MM_SR_PLUS_TIMES_F32
    w = int(mmsr.mm_plan_query(sr, levels, m, n, k, 0).workspace_min)
    dC = empty((m, n), torch.float32)
    mmsr.mm_strassen(levels, mmsr.MM_STRASSEN_WINOGRAD, sr, m, n, k, dev(A), dev(B), dC, workspace(w), w)
    torch.cuda.synchronize()
    assert mmsr.mm_last_device_status() == 0
    # small integers: every product and sum is exact, so the result is too
    np.testing.assert_array_equal(dC.cpu().numpy(), oracle.mm_f64(A, B).astype(np.float32))
