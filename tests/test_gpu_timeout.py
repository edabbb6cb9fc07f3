"""The bounded-wait timeout path of the tensor-core pipelines, exercised
without any fault: a one-shot test switch makes the first CTA of the next
launch skip the arrival (and loads) of its first pipeline stage, so that its
MMA wait runs out after 2 s.  The call must record MM_ERR_TIMEOUT, the CTA
must write zeros for its own output tile and leave every other tile correct,
and the next call (switch consumed) must run normally with a clean status."""
import numpy as np
import pytest

import oracle
from paper_1911_05328_gb300 import inputs, mmsr

from gpu_util import dev, empty, rel_fro, workspace

pytestmark = pytest.mark.gpu
MM_ERR_TIMEOUT = -6


@pytest.fixture(autouse=True)
def disarm():
    mmsr.mm_last_device_status()
    yield
    mmsr.mm_set_option(mmsr.MM_OPT_TEST_SKIP_SIGNAL, 0)
    mmsr.mm_last_device_status()


def _run(sr, A, B, dtype):
    import torch

    m, k = A.shape
    n = B.shape[1]
    budget = int(mmsr.mm_plan_query(sr, -1, m, n, k, 0).workspace_min)
    ws = workspace(budget)
    dC = empty((m, n), dtype)
    dC.fill_(7)
    mmsr.mm_semiring(sr, m, n, k, dev(A), dev(B), dC, ws, budget)
    torch.cuda.synchronize()
    return dC.cpu().numpy()


@pytest.mark.parametrize(
    "sr,arm,shape,tile",
    [
        # FP32 mode: 128 x 256 output tiles; 16 k-blocks of 32 in a 4-deep ring
        (mmsr.MM_SR_PLUS_TIMES_F32, 1, (128, 200, 512), (128, 256)),
        (mmsr.MM_SR_PLUS_TIMES_F32, 1, (256, 512, 512), (128, 256)),
        # FP64-accuracy mode: 128 x 64 output tiles, 2-deep ring
        (mmsr.MM_SR_PLUS_TIMES_F64ACC, 2, (128, 64, 512), (128, 64)),
        (mmsr.MM_SR_PLUS_TIMES_F64ACC, 2, (256, 192, 512), (128, 64)),
    ],
    ids=["f32-1cta", "f32-4cta", "f64acc-1cta", "f64acc-6cta"],
)
def test_skipped_signal_times_out_cleanly(sr, arm, shape, tile):
    import torch

    m, n, k = shape
    cast, dtype, tol = ((np.float32, torch.float32, 1e-5) if sr == mmsr.MM_SR_PLUS_TIMES_F32
                        else (np.float64, torch.float64, 1e-12))
    A, B = inputs.normal_f32(m, k, n, seed=31)
    A, B = A.astype(cast), B.astype(cast)
    ref = oracle.mm_f64(A, B)

    mmsr.mm_set_option(mmsr.MM_OPT_TEST_SKIP_SIGNAL, arm)
    C = _run(sr, A, B, dtype)
    assert mmsr.mm_last_device_status() == MM_ERR_TIMEOUT
    # the first CTA owns output tile (0, 0): zeros; every other tile is correct
    tm, tn = min(tile[0], m), min(tile[1], n)
    assert np.all(C[:tm, :tn] == 0)
    mask = np.ones((m, n), bool)
    mask[:tm, :tn] = False
    if mask.any():
        assert rel_fro(C[mask], ref[mask]) <= tol

    # the switch was one-shot: the next call is whole and clean
    C = _run(sr, A, B, dtype)
    assert mmsr.mm_last_device_status() == 0
    assert rel_fro(C, ref) <= tol


def test_batched_skipped_signal_times_out_cleanly():
    """The persistent batched kernel: the first CTA's first tile times out; the
    CTA quiesces and leaves the tile queue, the others finish their tiles, and
    the next call is correct."""
    import torch

    rng = np.random.default_rng(32)
    dims = rng.integers(128, 400, size=(12, 3))
    probs = inputs.batched_problems(count=12, seed=32, dims=dims)
    dA = [dev(p.A) for p in probs]
    dB = [dev(p.B) for p in probs]
    F32 = mmsr.MM_SR_PLUS_TIMES_F32
    assert any(p.semiring == F32 for p in probs)
    dC = [empty((p.m, p.n), torch.float32 if p.semiring == F32 else torch.int32) for p in probs]
    table = [(p.semiring, p.m, p.n, p.k, a, b, c) for p, a, b, c in zip(probs, dA, dB, dC)]
    need = mmsr.mm_batched_query(table)
    ws = empty((need,), torch.uint8)

    mmsr.mm_set_option(mmsr.MM_OPT_TEST_SKIP_SIGNAL, 3)
    mmsr.mm_batched(table, ws, need)
    torch.cuda.synchronize()
    assert mmsr.mm_last_device_status() == MM_ERR_TIMEOUT
    # (min,+) problems run in their own launch and are unaffected
    for p, c in zip(probs, dC):
        if p.semiring != F32:
            np.testing.assert_array_equal(c.cpu().numpy(), oracle.mm_minplus(p.A, p.B))

    mmsr.mm_batched(table, ws, need)
    torch.cuda.synchronize()
    assert mmsr.mm_last_device_status() == 0
    for p, c in zip(probs, dC):
        if p.semiring == F32:
            assert rel_fro(c.cpu().numpy(), oracle.mm_f64(p.A, p.B)) <= 1e-5
        else:
            np.testing.assert_array_equal(c.cpu().numpy(), oracle.mm_minplus(p.A, p.B))
