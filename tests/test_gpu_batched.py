"""mm_batched: mixed FP32 (+,x) and (min,+) problems of uneven shapes in one
persistent launch, each checked against the oracle (bit-exact for (min,+)
and for integer-valued FP32 inputs, rel. Frobenius <= 1e-5 otherwise)."""
import numpy as np
import pytest

import oracle
from paper_1911_05328_gb300 import inputs, mmsr

from gpu_util import dev, empty, rel_fro

pytestmark = pytest.mark.gpu
F32, MP = mmsr.MM_SR_PLUS_TIMES_F32, mmsr.MM_SR_MIN_PLUS_I32


def _launch(probs, capture=False, splits=None, reps=1, levels=None):
    """probs: list of inputs.Problem; splits / levels: optional per-problem
    k-slice hints and Strassen levels (mm_problem_t.split_k / .levels);
    returns the list of output arrays (of the last of `reps` eager calls)."""
    import torch

    dA = [dev(p.A) for p in probs]
    dB = [dev(p.B) for p in probs]
    dC = [empty((p.m, p.n), torch.float32 if p.semiring == F32 else torch.int32) for p in probs]
    splits = splits or [0] * len(probs)
    levels = levels or [0] * len(probs)
    table = [(p.semiring, p.m, p.n, p.k, a, b, c, h, lv)
             for p, a, b, c, h, lv in zip(probs, dA, dB, dC, splits, levels)]
    need = mmsr.mm_batched_query(table)
    assert need > 0
    ws = empty((need,), torch.uint8)
    if capture:
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            mmsr.mm_batched(table, ws, need, stream=s)  # warm-up (sets kernel attributes)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        for c in dC:
            c.zero_()
        with torch.cuda.graph(g):
            mmsr.mm_batched(table, ws, need, stream=torch.cuda.current_stream())
        for c in dC:
            c.fill_(-1)
        g.replay()
    else:
        for _ in range(reps):
            for c in dC:
                c.fill_(-7)
            mmsr.mm_batched(table, ws, need)
    torch.cuda.synchronize()
    assert mmsr.mm_last_device_status() == 0
    return [c.cpu().numpy() for c in dC]


def _check(probs, outs, exact_fp32=False):
    for p, C in zip(probs, outs):
        if p.semiring == MP:
            np.testing.assert_array_equal(C, oracle.mm_minplus(p.A, p.B), err_msg=str((p.m, p.n, p.k)))
        elif exact_fp32:
            np.testing.assert_array_equal(C, oracle.mm_f64(p.A, p.B).astype(np.float32))
        else:
            ref = oracle.mm_f64(p.A, p.B)
            assert rel_fro(C, ref) <= 1e-5, (p.m, p.n, p.k, rel_fro(C, ref))


def _mixed(count, seed, lo=1, hi=300, integer=False):
    rng = np.random.default_rng(seed)
    dims = rng.integers(lo, hi + 1, size=(count, 3))
    probs = inputs.batched_problems(count=count, seed=seed, dims=dims)
    if integer:
        for p in probs:
            if p.semiring == F32:
                p.A = rng.integers(-4, 5, size=p.A.shape).astype(np.float32)
                p.B = rng.integers(-4, 5, size=p.B.shape).astype(np.float32)
    return probs


def test_small_mixed_batch_integer_exact():
    probs = _mixed(24, seed=200, integer=True)
    _check(probs, _launch(probs), exact_fp32=True)


def test_small_mixed_batch_normal():
    probs = _mixed(40, seed=201, lo=1, hi=700)
    _check(probs, _launch(probs))


def test_minplus_out_of_packed_range_in_batch():
    probs = _mixed(10, seed=202, lo=50, hi=400)
    for p in probs:
        if p.semiring == MP:
            p.A[0, 0] = 30000
            p.A[p.m // 2, p.k - 1] = inputs.INF
    _check(probs, _launch(probs))


def test_graph_capture_replay():
    probs = _mixed(16, seed=203, lo=30, hi=500)
    _check(probs, _launch(probs, capture=True))


def test_rejects_unsupported_semiring():
    import torch

    d = empty((8, 8), torch.float64)
    rc = mmsr.mm_batched([(mmsr.MM_SR_PLUS_TIMES_F64, 8, 8, 8, d, d, d)], d, 64, check=False)
    assert rc == mmsr.MM_ERR_UNSUPPORTED


def test_workload_512_problems():
    # 512 problems, m, n, k log-uniform in [64, 2048], 70% FP32 normal(0,1),
    # 30% (min,+) integers in [0, 1000], seed 4
    probs = inputs.batched_problems(count=512, seed=4)
    assert sum(p.semiring == F32 for p in probs) == 358
    _check(probs, _launch(probs))


@pytest.mark.parametrize("only", [F32, MP])
def test_single_semiring_batches(only):
    # a batch with no (min,+) (or no FP32) problem skips that launch entirely
    probs = [p for p in _mixed(30, seed=204, lo=20, hi=600) if p.semiring == only]
    assert probs
    _check(probs, _launch(probs))


def test_k_zero_and_tiny_problems():
    # k = 0 writes the semiring's 0; 1 x 1 x 1 problems of both kinds
    rng = np.random.default_rng(205)
    probs = []
    for sr, m, n, k in ((F32, 3, 5, 0), (MP, 4, 6, 0), (F32, 1, 1, 1), (MP, 1, 1, 1), (F32, 130, 129, 257)):
        if sr == F32:
            A = rng.standard_normal((m, k)).astype(np.float32)
            B = rng.standard_normal((k, n)).astype(np.float32)
        else:
            A = rng.integers(0, 1001, size=(m, k)).astype(np.int32)
            B = rng.integers(0, 1001, size=(k, n)).astype(np.int32)
        probs.append(inputs.Problem(sr, m, n, k, A, B))
    outs = _launch(probs)
    assert np.all(outs[0] == 0.0) and np.all(outs[1] == mmsr.INF)
    _check(probs, outs)


@pytest.mark.parametrize("capture", [False, True], ids=["eager", "graph-replay"])
def test_batch_beyond_one_table_chunk(capture):
    # 1500 problems: past the old by-value table limit of 512 and more than
    # one table upload launch (72 bytes per problem, 30 KB per launch); every
    # problem checked, eagerly and as a replayed graph
    probs = _mixed(1500, seed=206, lo=1, hi=96, integer=True)
    _check(probs, _launch(probs, capture=capture), exact_fp32=True)


def _fp32(rng, m, n, k, integer=False):
    if integer:
        A = rng.integers(-4, 5, size=(m, k)).astype(np.float32)
        B = rng.integers(-4, 5, size=(k, n)).astype(np.float32)
    else:
        A = rng.standard_normal((m, k)).astype(np.float32)
        B = rng.standard_normal((k, n)).astype(np.float32)
    return inputs.Problem(F32, m, n, k, A, B)


@pytest.mark.parametrize("integer", [True, False], ids=["integer-exact", "normal"])
def test_k_sliced_tiles_by_hint(integer):
    # FP32 tiles cut into 2, 3 and 7 k-slices (ragged last slices, ragged
    # tiles), beside unsplit FP32 and (min,+) problems: the last slice to
    # finish folds the partial tiles in slice order, so repeated calls agree
    # bit for bit
    rng = np.random.default_rng(207)
    probs = [_fp32(rng, 200, 300, 1000, integer), _fp32(rng, 129, 257, 3000, integer),
             _fp32(rng, 64, 64, 4500, integer), _fp32(rng, 300, 100, 200, integer)]
    probs += [p for p in _mixed(8, seed=208, lo=40, hi=300) if p.semiring == MP][:3]
    splits = [2, 3, 7, 1] + [0] * (len(probs) - 4)
    outs = _launch(probs, splits=splits)
    _check(probs, outs, exact_fp32=integer)
    again = _launch(probs, splits=splits, reps=2)
    for a, b in zip(outs, again):
        np.testing.assert_array_equal(a, b)


def test_k_sliced_tiles_library_rule():
    # a few long-k FP32 problems among many short ones: their tiles exceed an
    # eighth of an SM's share of the batch's work, so the library slices them
    # (the workspace grows by their partial tiles); results as unsliced
    rng = np.random.default_rng(209)
    probs = [_fp32(rng, 256, 256, 16384), _fp32(rng, 130, 200, 12000)]
    probs += [_fp32(rng, 128, 128, 64) for _ in range(6)]
    import torch

    d = empty((8,), torch.float32)
    auto = [(F32, p.m, p.n, p.k, d, d, d, 0) for p in probs]
    plain = [(F32, p.m, p.n, p.k, d, d, d, 1) for p in probs]
    assert mmsr.mm_batched_query(auto) > mmsr.mm_batched_query(plain)
    sliced = _launch(probs)
    _check(probs, sliced)
    unsliced = _launch(probs, splits=[1] * len(probs))
    for a, b in zip(sliced, unsliced):
        assert rel_fro(a, b.astype(np.float64)) <= 2e-6


def test_k_sliced_tiles_graph_replay():
    # the per-tile counters are zeroed by the call's own memset, so a captured
    # call replays correctly
    rng = np.random.default_rng(210)
    probs = [_fp32(rng, 190, 260, 2500, integer=True), _fp32(rng, 70, 90, 700, integer=True)]
    _check(probs, _launch(probs, capture=True, splits=[5, 2]), exact_fp32=True)


def test_strassen_level_in_batch_integer_exact():
    # FP32 problems with one Strassen-Winograd level beside plain FP32 and
    # (min,+) problems: leaf operand sums in the pre-pass, leaf products in the
    # tile queue, the post pass folds them into C -- exact on small integers
    rng = np.random.default_rng(211)
    probs = [_fp32(rng, 256, 384, 512, True), _fp32(rng, 130, 66, 258, True), _fp32(rng, 2, 2, 2, True),
             _fp32(rng, 300, 200, 100, True)]
    probs += [p for p in _mixed(10, seed=212, lo=40, hi=300) if p.semiring == MP][:3]
    levels = [1, 1, 1, 0] + [0] * (len(probs) - 4)
    _check(probs, _launch(probs, levels=levels), exact_fp32=True)


def test_strassen_level_in_batch_normal_and_sliced():
    # normal inputs within the derived one-level Winograd tolerance, also with
    # the leaves' tiles cut into k-slices, and as a replayed graph
    from error_bounds import fp32_strassen_tol

    rng = np.random.default_rng(213)
    probs = [_fp32(rng, 512, 512, 4096), _fp32(rng, 200, 300, 1000), _fp32(rng, 128, 128, 64)]
    tol = fp32_strassen_tol(mmsr.MM_STRASSEN_WINOGRAD, 1)
    for kw in ({}, {"splits": [4, 0, 0]}, {"capture": True}):
        outs = _launch(probs, levels=[1, 1, 0], **kw)
        for p, C in zip(probs, outs):
            assert rel_fro(C, oracle.mm_f64(p.A, p.B)) <= tol, (p.m, p.n, p.k, kw)
