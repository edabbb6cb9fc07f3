"""Multi-GPU decompositions of one semiring product (host logic, torch.distributed).

Two shardings of C = A (x) B over `world` ranks:

* k-sharding -- the paper's k-parallel split (the two (+)-terms of Eq. mm-dac,
  CO3's temporary D and its madd, Fig. mm-n3) carried across devices: rank r
  multiplies the k-slice [k_r, k_{r+1}) of A's columns and B's rows, and one
  all-reduce with the semiring's (+) folds the partials: MIN for (min,+),
  SUM for (+,x), MAX (= OR on 0/1) for boolean.  Each rank holds a full
  m x n partial: the multi-device counterpart of one workspace buffer per
  extra k-slice.
* row-sharding -- rank r owns rows [i_r, i_{r+1}) of C (A's row panel times
  all of B); an all-gather assembles C.  No (+) crosses devices.

Independent problems (the batched workload, replicas of one product) need no
collective at all.  The local product is a callable so the same host logic
runs on GPUs (mm_semiring) and in CPU tests.
"""
from __future__ import annotations

from . import mmsr


def split_range(total: int, world: int, rank: int):
    """Contiguous balanced [lo, hi) of `total` items for `rank` of `world`."""
    base, extra = divmod(total, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def reduce_op(semiring: int):
    import torch.distributed as dist

    if semiring == mmsr.MM_SR_MIN_PLUS_I32:
        return dist.ReduceOp.MIN
    if semiring == mmsr.MM_SR_OR_AND_U8:
        return dist.ReduceOp.MAX
    return dist.ReduceOp.SUM


def kshard_mm(semiring: int, A, B, local_mm, group=None):
    """C = A (x) B with k split across the ranks of `group`.

    A: m x k, B: k x n (torch tensors, same on every rank); local_mm(Ak, Bk)
    returns the m x n partial of one k-slice as a torch tensor on the
    communication device.  Returns C on every rank."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    lo, hi = split_range(A.shape[1], world, rank)
    part = local_mm(A[:, lo:hi].contiguous(), B[lo:hi, :].contiguous())
    dist.all_reduce(part, op=reduce_op(semiring), group=group)
    return part


def rowshard_mm(A, B, local_mm, group=None):
    """C = A (x) B with C's rows split across ranks; returns the full C on
    every rank (all-gather of equal-height panels, padded on the last rank)."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    m = A.shape[0]
    h = (m + world - 1) // world
    lo, hi = min(rank * h, m), min((rank + 1) * h, m)
    panel = local_mm(A[lo:hi].contiguous(), B)
    padded = torch.zeros((h, B.shape[1]), dtype=panel.dtype, device=panel.device)
    padded[: hi - lo] = panel
    gathered = [torch.empty_like(padded) for _ in range(world)]
    dist.all_gather(gathered, padded, group=group)
    return torch.cat(gathered, dim=0)[:m]
