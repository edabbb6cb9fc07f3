"""Multi-rank decompositions on CPU: world_size 2 over gloo, the local
products computed by the oracle.  k-sharding with the semiring's (+) as the
all-reduce, and row-sharding with an all-gather, must reproduce the
single-rank oracle product exactly (integer semirings) or within rounding."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1911_05328_gb300 import distributed, inputs, mmsr


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, case, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle

        if case == "minplus":
            A, B = inputs.tropical_i32(37, 101, 29, seed=5)
            sr = mmsr.MM_SR_MIN_PLUS_I32
            local = lambda a, b: torch.from_numpy(oracle.mm_minplus(a.numpy(), b.numpy()))
            C = distributed.kshard_mm(sr, torch.from_numpy(A), torch.from_numpy(B), local)
        elif case == "orand":
            A, B = inputs.boolean_u8(30, 90, 25, seed=6, density=0.05)
            sr = mmsr.MM_SR_OR_AND_U8
            local = lambda a, b: torch.from_numpy(oracle.mm_orand(a.numpy(), b.numpy()))
            C = distributed.kshard_mm(sr, torch.from_numpy(A), torch.from_numpy(B), local)
        elif case == "f64":
            A, B = inputs.uniform_f64(21, 77, 18, seed=7)
            sr = mmsr.MM_SR_PLUS_TIMES_F64
            local = lambda a, b: torch.from_numpy(oracle.mm_f64(a.numpy(), b.numpy()))
            C = distributed.kshard_mm(sr, torch.from_numpy(A), torch.from_numpy(B), local)
        else:  # row sharding, (min,+)
            A, B = inputs.tropical_i32(41, 50, 33, seed=8)
            local = lambda a, b: torch.from_numpy(oracle.mm_minplus(a.numpy(), b.numpy()))
            C = distributed.rowshard_mm(torch.from_numpy(A), torch.from_numpy(B), local)
        if rank == 0:
            q.put(C.numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", ["minplus", "orand", "f64", "rows"])
def test_two_rank_decomposition(case):
    import oracle

    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, case, q)) for r in range(2)]
    for p in procs:
        p.start()
    C = q.get()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    if case == "minplus":
        A, B = inputs.tropical_i32(37, 101, 29, seed=5)
        np.testing.assert_array_equal(C, oracle.mm_minplus(A, B))
    elif case == "orand":
        A, B = inputs.boolean_u8(30, 90, 25, seed=6, density=0.05)
        np.testing.assert_array_equal(C, oracle.mm_orand(A, B))
    elif case == "f64":
        A, B = inputs.uniform_f64(21, 77, 18, seed=7)
        ref = oracle.mm_f64(A, B)
        assert np.linalg.norm(C - ref) / np.linalg.norm(ref) < 1e-14
    else:
        A, B = inputs.tropical_i32(41, 50, 33, seed=8)
        np.testing.assert_array_equal(C, oracle.mm_minplus(A, B))


def test_split_range_covers_exactly():
    for total in (0, 1, 7, 100, 4097):
        for world in (1, 2, 3, 8):
            rs = [distributed.split_range(total, world, r) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == total
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            assert max(h - l for l, h in rs) - min(h - l for l, h in rs) <= 1
