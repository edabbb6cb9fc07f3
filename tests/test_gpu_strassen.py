"""Strassen / Strassen-Winograd levels on the GPU vs the oracle.

* Integer-valued inputs whose every intermediate is exact (bf16 split, FP32
  sums below 2^24) must reproduce the classic oracle product bit for bit,
  for L = 1..4 and both variants (the paper's pin: exact agreement of
  Strassen with the classic result on small-integer inputs).
* Plain FP64 mode must stay within 1e-12 relative Frobenius error.
* FP32 mode (bf16x3 leaves) has an error that grows with the number of
  levels (the operand sums are larger than the entries and the post-additions
  cancel).  It is printed per level and held to the tolerance derived from
  the standard worst-case analysis (tests/error_bounds.py): 1e-5 x 6^L for the
  paper's formulas, 1e-5 x 9^L for Winograd's; the paper's formulas at one
  level are also held to the plain FP32-mode 1e-5.
"""
import numpy as np
import pytest

import oracle
from paper_1911_05328_gb300 import inputs, mmsr

from error_bounds import FP32_TOL, fp32_strassen_tol
from gpu_util import canary_intact, dev, empty, rel_fro, workspace

pytestmark = pytest.mark.gpu
VARIANTS = [mmsr.MM_STRASSEN_PAPER, mmsr.MM_STRASSEN_WINOGRAD]


def run(L, variant, sr, A, B):
    import torch

    m, k = A.shape
    n = B.shape[1]
    p = mmsr.mm_plan_query(sr, L, m, n, k, 0)
    budget = int(p.workspace_min)
    ws = workspace(budget)
    dt = torch.float32 if sr == mmsr.MM_SR_PLUS_TIMES_F32 else torch.float64
    npdt = np.float32 if dt == torch.float32 else np.float64
    dC = empty((m, n), dt)
    mmsr.mm_strassen(L, variant, sr, m, n, k, dev(A.astype(npdt)), dev(B.astype(npdt)), dC, ws, budget)
    torch.cuda.synchronize()
    assert canary_intact(ws, budget)
    return dC.cpu().numpy()


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("L,m,k,n,bound", [(1, 256, 256, 256, 2), (2, 512, 256, 384, 2),
                                           (3, 512, 512, 256, 2), (4, 1024, 1024, 768, 1)])
def test_fp32_integer_inputs_exact(variant, L, m, k, n, bound):
    A, B = inputs.small_int(m, k, n, seed=70 + L, bound=bound, dtype=np.float32)
    C = run(L, variant, mmsr.MM_SR_PLUS_TIMES_F32, A, B)
    np.testing.assert_array_equal(C, oracle.mm_f64(A, B).astype(np.float32))


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_fp64_integer_inputs_exact(variant, L):
    m, k, n = 256, 512, 320
    A, B = inputs.small_int(m, k, n, seed=80 + L, bound=5)
    np.testing.assert_array_equal(run(L, variant, mmsr.MM_SR_PLUS_TIMES_F64, A, B), oracle.mm_f64(A, B))


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_fp64_uniform_tolerance(variant, L):
    m, k, n = 512, 768, 256
    A, B = inputs.uniform_f64(m, k, n, seed=3)
    err = rel_fro(run(L, variant, mmsr.MM_SR_PLUS_TIMES_F64, A, B), oracle.mm_f64(A, B))
    assert err <= 1e-12, err


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_fp32_uniform_error_per_level(variant, L):
    m, k, n = 1024, 2048, 768
    A, B = inputs.uniform_f64(m, k, n, seed=3)
    A32, B32 = A.astype(np.float32), B.astype(np.float32)
    err = rel_fro(run(L, variant, mmsr.MM_SR_PLUS_TIMES_F32, A32, B32), oracle.mm_f64(A32, B32))
    print("fp32 strassen variant %d L %d rel_fro %.3e" % (variant, L, err))
    assert err <= fp32_strassen_tol(variant, L), err
    if variant == mmsr.MM_STRASSEN_PAPER and L == 1:
        assert err <= FP32_TOL, err


def test_rectangular_shape_all_levels():
    # the 12288 x 16384 x 8192 shape scaled down by 16, FP64 mode
    m, k, n = 768, 1024, 512
    A, B = inputs.uniform_f64(m, k, n, seed=3)
    ref = oracle.mm_f64(A, B)
    for L in (1, 2, 3, 4):
        assert rel_fro(run(L, mmsr.MM_STRASSEN_WINOGRAD, mmsr.MM_SR_PLUS_TIMES_F64, A, B), ref) <= 1e-12


def test_workspace_below_minimum_rejected():
    import torch

    p = mmsr.mm_plan_query(mmsr.MM_SR_PLUS_TIMES_F32, 2, 256, 256, 256, 0)
    ws = empty((int(p.workspace_min),), torch.uint8)
    d = empty((256, 256), torch.float32)
    rc = mmsr.mm_strassen(2, 1, mmsr.MM_SR_PLUS_TIMES_F32, 256, 256, 256, d, d, d, ws,
                          int(p.workspace_min) - 1024, check=False)
    assert rc == mmsr.MM_ERR_WORKSPACE


def test_full_size_n16384_fp32_sampled_rows():
    # the Strassen-Winograd workload: n = 16384, uniform[-1,1] (seed 3) cast
    # to float32; error per level on the sampled rows (incl. quadrant edges)
    import torch

    n = 16384
    A, B = inputs.uniform_f64(n, n, n, seed=3)
    A32, B32 = A.astype(np.float32), B.astype(np.float32)
    del A, B
    rows = oracle.sample_rows(n)
    ref = oracle.mm_f64(A32, B32, rows=rows)
    dA, dB = dev(A32), dev(B32)
    dC = empty((n, n), torch.float32)
    for L in (1, 2, 3, 4):
        p = mmsr.mm_plan_query(mmsr.MM_SR_PLUS_TIMES_F32, L, n, n, n, 0)
        ws = empty((int(p.workspace_min),), torch.uint8)
        mmsr.mm_strassen(L, mmsr.MM_STRASSEN_WINOGRAD, mmsr.MM_SR_PLUS_TIMES_F32, n, n, n, dA, dB, dC, ws,
                         int(p.workspace_min))
        torch.cuda.synchronize()
        err = rel_fro(dC.cpu().numpy()[rows], ref)
        print("n16384 fp32 winograd L %d rel_fro %.3e workspace %.2f n^2*4B" % (L, err, p.workspace_min / (n * n * 4)))
        assert err <= fp32_strassen_tol(mmsr.MM_STRASSEN_WINOGRAD, L), err
        del ws
        torch.cuda.empty_cache()


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_f64acc_integer_inputs_exact(variant, L):
    m, k, n = 256, 512, 320
    A, B = inputs.small_int(m, k, n, seed=110 + L, bound=50)
    C = run(L, variant, mmsr.MM_SR_PLUS_TIMES_F64ACC, A, B)
    np.testing.assert_array_equal(C, oracle.mm_f64(A, B))


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_f64acc_uniform_tolerance_every_level(variant, L):
    # FP64-accuracy mode must meet 1e-12 at every level
    m, k, n = 512, 1024, 384
    A, B = inputs.uniform_f64(m, k, n, seed=3)
    err = rel_fro(run(L, variant, mmsr.MM_SR_PLUS_TIMES_F64ACC, A, B), oracle.mm_f64(A, B))
    print("f64acc strassen variant %d L %d rel_fro %.3e" % (variant, L, err))
    assert err <= 1e-12, err


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("L", [2, 3, 4])
def test_f64acc_zero_and_scaled_leaf_lines(variant, L):
    # The last operand pass also produces the digit split's row exponents and
    # column maxima.  Zero rows of A at one position in every row block of
    # the leaves' size (and zero columns of B likewise) make zero leaf lines
    # -- the pass's full re-scan -- and zero lines of C; rows and columns
    # scaled by 2^-900 and 2^600 move the exponents far from 0.
    m, k, n = 512, 1024, 384
    h, w = m >> L, n >> L
    A, B = inputs.uniform_f64(m, k, n, seed=7)
    zr, sr_ = [5 % h + a * h for a in range(1 << L)], [(17 % h) + a * h for a in range(1 << L)]
    zc, sc_ = [3 % w + b * w for b in range(1 << L)], [(11 % w) + b * w for b in range(1 << L)]
    A[zr] = 0.0
    A[sr_] *= 2.0 ** -900
    B[:, zc] = 0.0
    B[:, sc_] *= 2.0 ** 600
    C = run(L, variant, mmsr.MM_SR_PLUS_TIMES_F64ACC, A, B)
    ref = oracle.mm_f64(A, B)
    assert not np.any(C[zr]) and not np.any(C[:, zc])
    keep_r = np.setdiff1d(np.arange(m), zr)
    keep_c = np.setdiff1d(np.arange(n), zc)
    Ck, Rk = C[np.ix_(keep_r, keep_c)], ref[np.ix_(keep_r, keep_c)]
    rs = np.abs(Rk).max(axis=1, keepdims=True)
    cs = np.abs(Rk / rs).max(axis=0, keepdims=True)
    err = rel_fro(Ck / rs / cs, Rk / rs / cs)
    assert err <= 1e-12, err


def test_full_size_n16384_f64acc_sampled_rows():
    import torch

    n = 16384
    A, B = inputs.uniform_f64(n, n, n, seed=3)
    rows = oracle.sample_rows(n)
    ref = oracle.mm_f64(A, B, rows=rows)
    dA, dB = dev(A), dev(B)
    del A, B
    dC = empty((n, n), torch.float64)
    for L in (1, 2, 3, 4):
        p = mmsr.mm_plan_query(mmsr.MM_SR_PLUS_TIMES_F64ACC, L, n, n, n, 0)
        ws = empty((int(p.workspace_min),), torch.uint8)
        mmsr.mm_strassen(L, mmsr.MM_STRASSEN_WINOGRAD, mmsr.MM_SR_PLUS_TIMES_F64ACC, n, n, n, dA, dB, dC, ws,
                         int(p.workspace_min))
        torch.cuda.synchronize()
        err = rel_fro(dC.cpu().numpy()[rows], ref)
        print("n16384 f64acc winograd L %d rel_fro %.3e workspace %.2f n^2*8B" % (L, err, p.workspace_min / (n * n * 8)))
        assert err <= 1e-12, err
        del ws
        torch.cuda.empty_cache()


def test_full_size_rectangular_both_modes_sampled_rows():
    # the rectangular Strassen-Winograd workload at full size: m = 12288,
    # k = 16384, n = 8192, uniform[-1,1] (seed 3), L = 1..4, FP64-accuracy
    # mode (1e-12) and FP32 mode on the float32 cast (derived tolerance),
    # sampled rows incl. the quadrant edges of every level
    import torch

    m, k, n = 12288, 16384, 8192
    A, B = inputs.uniform_f64(m, k, n, seed=3)
    rows = oracle.sample_rows(m)
    for sr in (mmsr.MM_SR_PLUS_TIMES_F64ACC, mmsr.MM_SR_PLUS_TIMES_F32):
        f32 = sr == mmsr.MM_SR_PLUS_TIMES_F32
        Ax, Bx = (A.astype(np.float32), B.astype(np.float32)) if f32 else (A, B)
        ref = oracle.mm_f64(Ax, Bx, rows=rows)
        dA, dB = dev(Ax), dev(Bx)
        dC = empty((m, n), torch.float32 if f32 else torch.float64)
        for L in (1, 2, 3, 4):
            p = mmsr.mm_plan_query(sr, L, m, n, k, 0)
            ws = empty((int(p.workspace_min),), torch.uint8)
            mmsr.mm_strassen(L, mmsr.MM_STRASSEN_WINOGRAD, sr, m, n, k, dA, dB, dC, ws, int(p.workspace_min))
            torch.cuda.synchronize()
            idx = torch.from_numpy(rows).cuda()
            err = rel_fro(dC.index_select(0, idx).cpu().numpy(), ref)
            print("rect %s winograd L %d rel_fro %.3e" % ("fp32" if f32 else "f64acc", L, err))
            tol = fp32_strassen_tol(mmsr.MM_STRASSEN_WINOGRAD, L) if f32 else 1e-12
            assert err <= tol, (sr, L, err)
            assert mmsr.mm_last_device_status() == 0
            del ws
            torch.cuda.empty_cache()
        del dA, dB, dC
        torch.cuda.empty_cache()


@pytest.mark.parametrize("sr", [mmsr.MM_SR_PLUS_TIMES_F32, mmsr.MM_SR_PLUS_TIMES_F64ACC, mmsr.MM_SR_PLUS_TIMES_F64])
def test_auto_depth_runs_the_planned_depth(sr):
    # MM_LEVELS_AUTO under the full budget of the planned depth, and under a
    # budget one byte short of it (one level less)
    import torch

    m = n = k = 2048
    A, B = inputs.uniform_f64(m, k, n, seed=7)
    f32 = sr == mmsr.MM_SR_PLUS_TIMES_F32
    Ax, Bx = (A.astype(np.float32), B.astype(np.float32)) if f32 else (A, B)
    ref = oracle.mm_f64(Ax, Bx)
    big = 1 << 36
    p = mmsr.mm_plan_query(sr, mmsr.MM_LEVELS_AUTO, m, n, k, big)
    assert p.levels >= 1
    for budget in (int(p.workspace_min), int(p.workspace_min) - 1):
        q = mmsr.mm_plan_query(sr, mmsr.MM_LEVELS_AUTO, m, n, k, budget)
        assert q.levels == (p.levels if budget == p.workspace_min else p.levels - 1)
        ws = workspace(budget)
        dC = empty((m, n), torch.float32 if f32 else torch.float64)
        mmsr.mm_strassen(mmsr.MM_LEVELS_AUTO, mmsr.MM_STRASSEN_WINOGRAD, sr, m, n, k, dev(Ax), dev(Bx), dC, ws,
                         budget)
        torch.cuda.synchronize()
        assert canary_intact(ws, budget)
        tol = fp32_strassen_tol(mmsr.MM_STRASSEN_WINOGRAD, q.levels) if f32 else 1e-12
        assert rel_fro(dC.cpu().numpy(), ref) <= tol
