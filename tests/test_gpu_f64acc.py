"""FP64-accuracy mode (+,x) vs the FP64 oracle at 1e-12 relative Frobenius
error, under both digit schemes: six 8-bit slices (21 exact slice products,
the default for plain products) and seven 7-bit slices (28 products, the
scheme under three or four Strassen levels).  Integer inputs pin the
exactness of the chunked TMEM accumulation: their digits are exact integers
and so is the whole product."""
import numpy as np
import pytest

import oracle
from paper_1911_05328_gb300 import inputs, mmsr

from gpu_util import canary_intact, dev, empty, rel_fro, workspace

pytestmark = pytest.mark.gpu
SR = mmsr.MM_SR_PLUS_TIMES_F64ACC
TOL = 1e-12
INT_BITS = {6: 47, 7: 49}  # width of the one scaled rounding of each scheme


@pytest.fixture(autouse=True, params=[6, 7], ids=["six-8bit-slices", "seven-7bit-slices"])
def slices(request):
    mmsr.mm_set_option(mmsr.MM_OPT_F64ACC_SLICES, request.param)
    yield request.param
    mmsr.mm_set_option(mmsr.MM_OPT_F64ACC_SLICES, 0)


def run(A, B, extra_parts=0):
    import torch

    m, k = A.shape
    n = B.shape[1]
    p0 = mmsr.mm_plan_query(SR, -1, m, n, k, 0)
    budget = int(p0.workspace_min) + extra_parts * m * n * 8
    ws = workspace(budget)
    dC = empty((m, n), torch.float64)
    mmsr.mm_semiring(SR, m, n, k, dev(A), dev(B), dC, ws, budget)
    torch.cuda.synchronize()
    assert canary_intact(ws, budget)
    assert mmsr.mm_last_device_status() == 0
    return dC.cpu().numpy()


@pytest.mark.parametrize("m,n,k", [(128, 64, 32), (128, 64, 64), (200, 130, 300), (512, 384, 2048)])
def test_integer_inputs_exact(m, n, k):
    A, B = inputs.small_int(m, k, n, seed=90 + k, bound=100)
    np.testing.assert_array_equal(run(A, B), oracle.mm_f64(A, B))


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (7, 5, 3), (128, 64, 32), (129, 65, 33), (300, 200, 1000), (1024, 768, 4096)])
def test_uniform_tolerance(m, n, k):
    A, B = inputs.uniform_f64(m, k, n, seed=m + n + k)
    err = rel_fro(run(A, B), oracle.mm_f64(A, B))
    assert err <= TOL, err


def test_row_and_column_scaling():
    # rows of A and columns of B spanning 2^-300 .. 2^300: the per-line
    # power-of-two scales must carry the exponent range exactly
    rng = np.random.default_rng(91)
    m, n, k = 256, 192, 512
    A, B = inputs.uniform_f64(m, k, n, seed=92)
    A *= np.exp2(rng.integers(-300, 300, size=(m, 1)).astype(np.float64))
    B *= np.exp2(rng.integers(-300, 300, size=(1, n)).astype(np.float64))
    C = run(A, B)
    ref = oracle.mm_f64(A, B)
    # compare row/column-normalised products (the scales make a plain
    # Frobenius norm meaningless across 600 binades)
    rs = np.abs(ref).max(axis=1, keepdims=True)
    cs = np.abs(ref / rs).max(axis=0, keepdims=True)
    assert rel_fro(C / rs / cs, ref / rs / cs) <= TOL


def test_extreme_scales_both_epilogue_paths():
    # row and column scales of 2^-500, 1 and 2^500: their sums reach 2^+-1000,
    # beyond the range where the epilogue builds its fma operands from bits
    # (it then takes the plain FP64 path); every output stays a normal double
    rng = np.random.default_rng(93)
    m, n, k = 192, 160, 384
    A, B = inputs.uniform_f64(m, k, n, seed=94)
    A *= np.exp2(rng.choice([-500.0, 0.0, 500.0], size=(m, 1)))
    B *= np.exp2(rng.choice([-500.0, 0.0, 500.0], size=(1, n)))
    C = run(A, B)
    ref = oracle.mm_f64(A, B)
    rs = np.abs(ref).max(axis=1, keepdims=True)
    cs = np.abs(ref / rs).max(axis=0, keepdims=True)
    assert np.all(np.isfinite(C))
    assert rel_fro(C / rs / cs, ref / rs / cs) <= TOL


@pytest.mark.parametrize("parts", [2, 5])
def test_split_k(parts):
    m, n, k = 256, 192, 4096
    A, B = inputs.uniform_f64(m, k, n, seed=93)
    assert rel_fro(run(A, B, extra_parts=parts), oracle.mm_f64(A, B)) <= TOL


def test_digit_rounding_edges_exact(slices):
    # Rows that drive the split's one rounding (x 2^(W-E) to an integer, ties
    # to even, E = frexp exponent of the row maximum, W = 47 or 49) through
    # its edge cases; B holds small integers, so the product of what the split
    # represents is exact in FP64 and the result must equal it bit for bit.
    W = INT_BITS[slices]
    rng = np.random.default_rng(95)
    k, n = 64, 40
    B = rng.integers(-8, 9, size=(k, n)).astype(np.float64)
    A = np.zeros((4, k))
    # ties: max 1.5 (E = 1); the others are odd multiples of 2^-W, half a unit
    A[0] = (2 * rng.integers(0, 1000, size=k) + 1) * 2.0 ** -W * rng.choice([-1.0, 1.0], size=k)
    A[0, 0] = 1.5
    # the largest value below 2^-2: its scaled value rounds up to 2^W
    A[1] = (2 - 2.0 ** -52) * 2.0 ** -3
    # subnormal row (its exponent comes from the significand's leading bit)
    A[2] = rng.integers(-100, 101, size=k) * 2.0 ** -1074
    # one normal entry: the subnormal rest scales far below one unit (to 0)
    A[3] = rng.integers(-100, 101, size=k) * 2.0 ** -1074
    A[3, 5] = 0.75
    E = [np.frexp(np.abs(r).max())[1] for r in A]
    Aq = np.array([np.ldexp(np.rint(np.ldexp(r, W - e)), e - W) for r, e in zip(A, E)])
    assert Aq[1, 0] == 0.25 and np.all(Aq[3, np.arange(k) != 5] == 0.0)
    np.testing.assert_array_equal(run(A, B), Aq @ B)


def test_zero_rows_and_columns():
    A, B = inputs.uniform_f64(130, 70, 90, seed=94)
    A[5] = 0.0
    B[:, 7] = 0.0
    C = run(A, B)
    assert np.all(C[5] == 0.0) and np.all(C[:, 7] == 0.0)
    assert rel_fro(C, oracle.mm_f64(A, B)) <= TOL


def test_full_size_n16384_sampled_rows():
    import torch

    n = 16384
    A, B = inputs.uniform_f64(n, n, n, seed=3)
    rows = oracle.sample_rows(n)
    ref = oracle.mm_f64(A, B, rows=rows)
    C = run(A, B)
    err = rel_fro(C[rows], ref)
    print("f64acc n16384 rel_fro %.3e" % err)
    assert err <= TOL, err
    torch.cuda.empty_cache()


def test_k_zero_writes_zero():
    import torch

    p = mmsr.mm_plan_query(SR, -1, 4, 6, 0, 0)
    ws = empty((int(p.workspace_min),), torch.uint8)
    dC = empty((4, 6), torch.float64)
    dC.fill_(5.0)
    mmsr.mm_semiring(SR, 4, 6, 0, empty((4, 1), torch.float64), empty((1, 6), torch.float64), dC, ws,
                     int(p.workspace_min))
    torch.cuda.synchronize()
    assert np.all(dC.cpu().numpy() == 0.0)
