"""The autotuner on the GPU: it times every split factor the budget allows,
caches the fastest, and the tuned call still reproduces the oracle."""
import numpy as np
import pytest

import oracle
from paper_1911_05328_gb300 import autotune, inputs, mmsr

from gpu_util import dev, empty

pytestmark = pytest.mark.gpu


def test_tuned_minplus_split(tmp_path, monkeypatch):
    import torch

    monkeypatch.setenv("MMSR_TUNE_CACHE", str(tmp_path / "tune.json"))
    m, n, k = 512, 384, 3000
    A, B = inputs.tropical_i32(m, k, n, seed=300)
    dA, dB = dev(A), dev(B)
    dC = empty((m, n), torch.int32)
    budget = 4 * m * n * 4
    ws = empty((budget,), torch.uint8)
    best = autotune.tune_semiring(mmsr.MM_SR_MIN_PLUS_I32, m, n, k, dA, dB, dC, ws, budget)
    assert 1 <= best["split_k"] <= 5 and best["budget"] <= budget and best["ms"] > 0
    dC.fill_(-1)
    autotune.mm_semiring_tuned(mmsr.MM_SR_MIN_PLUS_I32, m, n, k, dA, dB, dC, ws, budget)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(dC.cpu().numpy(), oracle.mm_minplus(A, B))


def test_tuned_strassen_depth(tmp_path, monkeypatch):
    import torch

    monkeypatch.setenv("MMSR_TUNE_CACHE", str(tmp_path / "tune.json"))
    n = 1024
    A, B = inputs.small_int(n, n, n, seed=301, bound=2, dtype=np.float32)
    dA, dB = dev(A), dev(B)
    dC = empty((n, n), torch.float32)
    budget = int(mmsr.mm_plan_query(mmsr.MM_SR_PLUS_TIMES_F32, 2, n, n, n, 0).workspace_min)
    ws = empty((budget,), torch.uint8)
    best = autotune.tune_strassen(mmsr.MM_SR_PLUS_TIMES_F32, n, n, n, dA, dB, dC, ws, budget)
    assert best["levels"] in (0, 1, 2)
    L = best["levels"]
    mmsr.mm_strassen(L, mmsr.MM_STRASSEN_WINOGRAD, mmsr.MM_SR_PLUS_TIMES_F32, n, n, n, dA, dB, dC, ws,
                     best["workspace"])
    torch.cuda.synchronize()
    np.testing.assert_array_equal(dC.cpu().numpy(), oracle.mm_f64(A, B).astype(np.float32))


def test_tuned_batched_k_slices(tmp_path, monkeypatch):
    # the batch tuner times k-slice hints per k bucket on the device and the
    # tuned call still reproduces the oracle (integer inputs: exact)
    import torch

    monkeypatch.setenv("MMSR_TUNE_CACHE", str(tmp_path / "tune.json"))
    rng = np.random.default_rng(302)
    shapes = [(256, 256, 8192), (128, 192, 8192), (100, 100, 2000), (64, 64, 64)]
    probs, dCs = [], []
    for m, n, k in shapes:
        A = rng.integers(-3, 4, size=(m, k)).astype(np.float32)
        B = rng.integers(-3, 4, size=(k, n)).astype(np.float32)
        dC = empty((m, n), torch.float32)
        probs.append((mmsr.MM_SR_PLUS_TIMES_F32, m, n, k, dev(A), dev(B), dC, A, B))
        dCs.append(dC)
    table = [p[:7] for p in probs]
    need = max(mmsr.mm_batched_query(autotune.apply_splits(table, [h] * len(table))) for h in (0, 16))
    ws = empty((need,), torch.uint8)
    rec = autotune.tune_batched(table, ws, need)
    assert set(rec["buckets"]) == {"8192", "2048"} and len(rec["splits"]) == 4 and rec["splits"][3] == 0
    for c in dCs:
        c.fill_(-1)
    autotune.mm_batched_tuned(table, ws, need)
    torch.cuda.synchronize()
    assert mmsr.mm_last_device_status() == 0
    for p, c in zip(probs, dCs):
        np.testing.assert_array_equal(c.cpu().numpy(), oracle.mm_f64(p[7], p[8]).astype(np.float32))
