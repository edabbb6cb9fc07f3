"""Boolean (or, and) semiring on the GPU vs the oracle: bit-exact, including
split-K (byte partials folded by OR), ragged shapes and transitive closure."""
import numpy as np
import pytest

import oracle
from paper_1911_05328_gb300 import inputs, mmsr

from gpu_util import canary_intact, dev, empty, workspace

pytestmark = pytest.mark.gpu
SR = mmsr.MM_SR_OR_AND_U8


def run(A, B, extra_parts=0):
    import torch

    m, k = A.shape
    n = B.shape[1]
    p0 = mmsr.mm_plan_query(SR, -1, m, n, k, 0)
    budget = int(p0.workspace_min) + extra_parts * m * n
    ws = workspace(budget)
    dC = empty((m, n), torch.uint8)
    mmsr.mm_semiring(SR, m, n, k, dev(A), dev(B), dC, ws, budget)
    torch.cuda.synchronize()
    assert canary_intact(ws, budget)
    return dC.cpu().numpy()


@pytest.mark.parametrize("m,n,k,density", [(1, 1, 1, 0.5), (7, 5, 3, 0.5), (128, 128, 1024, 0.002),
                                           (129, 131, 33, 0.05), (500, 300, 4000, 0.001), (1000, 1000, 1000, 0.003),
                                           # k % 16 == 0 (16-byte row loads), last word partial or whole
                                           (70, 90, 48, 0.1), (200, 130, 1008, 0.01), (256, 256, 4096, 0.5),
                                           # n % 16 == 0: 16-byte column loads, last column block partial
                                           (64, 1008, 100, 0.05), (33, 48, 300, 0.02)])
def test_matches_oracle(m, n, k, density):
    A, B = inputs.boolean_u8(m, k, n, seed=m + k, density=density)
    np.testing.assert_array_equal(run(A, B), oracle.mm_orand(A, B))


@pytest.mark.parametrize("k", [100, 96])
def test_nonzero_bytes_are_true(k):
    # every nonzero byte value counts as true, on both the byte-wise and the
    # 16-byte packing paths
    A, B = inputs.boolean_u8(64, k, 64, seed=3, density=0.05)
    rng = np.random.default_rng(k)
    A2 = A * rng.integers(1, 256, size=A.shape).astype(np.uint8)
    B2 = B * rng.integers(1, 256, size=B.shape).astype(np.uint8)
    np.testing.assert_array_equal(run(A2, B2), oracle.mm_orand(A, B))


@pytest.mark.parametrize("parts", [2, 3])
def test_split_k(parts):
    A, B = inputs.boolean_u8(300, 5000, 200, seed=9, density=0.0005)
    assert mmsr.mm_plan_query(SR, -1, 300, 200, 5000, 10 ** 9).split_k >= 2
    np.testing.assert_array_equal(run(A, B, extra_parts=parts), oracle.mm_orand(A, B))


def test_transitive_closure():
    from scipy.sparse.csgraph import shortest_path

    A, _ = inputs.boolean_u8(300, 300, 1, seed=21, density=0.004)
    R = (A | np.eye(300, dtype=np.uint8)).astype(np.uint8)
    for _ in range(9):
        R = run(R, R)
    reach = np.isfinite(shortest_path(A.astype(np.float64), unweighted=True, directed=True)).astype(np.uint8)
    np.testing.assert_array_equal(R, reach)
