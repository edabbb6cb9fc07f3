"""Shared helpers for the GPU parity tests (device buffers via torch)."""
import numpy as np

INF = 1 << 30


def dev(x):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def empty(shape, dtype):
    import torch

    return torch.empty(shape, dtype=dtype, device="cuda")


def workspace(nbytes, canary_bytes=4096, fill=0x5A):
    """Workspace of `nbytes` followed by a canary region the call must not touch."""
    import torch

    buf = torch.full((max(nbytes, 0) + canary_bytes,), fill, dtype=torch.uint8, device="cuda")
    return buf


def canary_intact(buf, nbytes, fill=0x5A):
    import torch

    tail = buf[nbytes:]
    return bool(torch.all(tail == fill).item())


def rel_fro(C, ref):
    C = np.asarray(C, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(C - ref) / (den if den > 0 else 1.0))
