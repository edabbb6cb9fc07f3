"""The allocation-free (min,+) entry point, checked through the C ABI
against mm_semiring given a caller workspace with the same split factor:
bit-exact, on two calls in a row (the second with different inputs, so a
stale partial from the first call would show).  Collected last on purpose."""
import numpy as np
import pytest

from paper_1911_05328_gb300 import inputs, mmsr

pytestmark = pytest.mark.gpu
SR = mmsr.MM_SR_MIN_PLUS_I32
SCRATCH = 64 << 20


def _with_workspace(dA, dB, m, n, k, s):
    import torch

    budget = (s - 1) * m * n * 4
    ws = torch.empty((max(budget, 16),), dtype=torch.uint8, device="cuda")
    dC = torch.empty((m, n), dtype=torch.int32, device="cuda")
    mmsr.mm_semiring(SR, m, n, k, dA, dB, dC, ws, budget)
    plan = mmsr.mm_plan_query(SR, -1, m, n, k, budget)
    return dC, plan.split_k


@pytest.mark.parametrize("m,n,k,s", [(1000, 900, 2000, 3), (4096, 4096, 4096, 2), (257, 129, 77, 9)])
def test_noalloc_matches_workspace_path_twice(m, n, k, s):
    import torch

    for call, seed in enumerate((101, 202)):
        A, B = inputs.tropical_i32(m, k, n, seed=seed + m)
        dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        ref, s_used = _with_workspace(dA, dB, m, n, k, s)
        dC = torch.full((m, n), -7, dtype=torch.int32, device="cuda")
        mmsr.mm_minplus_noalloc(m, n, k, dA, dB, dC, s)
        torch.cuda.synchronize()
        assert s_used > 1 or s == 1
        np.testing.assert_array_equal(dC.cpu().numpy(), ref.cpu().numpy(), err_msg="call %d" % call)


def test_noalloc_rejects_scratch_overflow():
    import torch

    n = 4096
    dA = torch.zeros((n, n), dtype=torch.int32, device="cuda")
    dC = torch.zeros((n, n), dtype=torch.int32, device="cuda")
    # s = 3 needs 2 * 64 MiB of partials > the 64 MiB array
    rc = mmsr.mm_minplus_noalloc(n, n, n, dA, dA, dC, 3, check=False)
    assert rc == mmsr.MM_ERR_WORKSPACE
