"""Run one workload a few times on cuda:0, for profilers (ncu) and timing.

    python -m paper_1911_05328_gb300.profile_case --case minplus4096 --reps 3

Cases: minplus4096 (the (min,+) n=4096 product, budget 0 unless --budget),
f32_<n> (FP32 mode, bf16x3 on tensor cores), f64acc_<n> (FP64-accuracy mode),
f64_<n> (plain FP64 path), orand_<n> (boolean), batched512 (the 512-problem
mixed batch), batched_longk (8 long-k FP32 products among 56 short ones),
strassen<L>_<n> (FP32-mode Strassen-Winograd, L levels,
uniform[-1,1] inputs), fa_strassen<L>_<n> (the same in FP64-accuracy mode), tar_<n>
(one TAR-Strassen level, FP32 mode), probes (one
launch of each instruction-throughput probe, kinds 0..3).
Inputs come from the seeded generators; nothing is checked here.
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="minplus4096")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--budget", type=int, default=0, help="extra m x n accumulator buffers")
    ap.add_argument("--shape", default="", help="m,n,k of a rectangular product (f32 / f64acc / f64 cases)")
    ap.add_argument("--budget-bytes", type=int, default=-1, help="workspace budget in bytes (overrides --budget)")
    a = ap.parse_args()
    import torch

    import __graft_entry__
    from paper_1911_05328_gb300 import inputs, mmsr

    __graft_entry__.build()
    torch.cuda.set_device(0)
    if a.case == "probes":
        import ctypes

        lib = mmsr.load()
        lib.mm_probe_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        rate, ms = ctypes.c_double(), ctypes.c_double()
        for kind, iters in ((0, 20000), (1, 20000), (2, 2000), (3, 20000)):
            for _ in range(a.reps):
                lib.mm_probe_peak(kind, iters, None, ctypes.byref(rate), ctypes.byref(ms))
            print("probe kind %d: %.2f Tops/s" % (kind, rate.value / 1e12))
        return
    if a.case.startswith("minplus"):
        n = int(a.case[len("minplus"):] or 4096)
        A, B = inputs.tropical_i32(n, n, n, seed=1)
        sr, dt = mmsr.MM_SR_MIN_PLUS_I32, torch.int32
        acc = 4
    elif a.case.startswith("f32_"):
        n = int(a.case[4:])
        A, B = inputs.normal_f32(n, n, n, seed=2)
        sr, dt = mmsr.MM_SR_PLUS_TIMES_F32, torch.float32
        acc = 4
    elif a.case.startswith("f64acc_"):
        n = int(a.case[7:])
        A, B = inputs.uniform_f64(n, n, n, seed=3)
        sr, dt = mmsr.MM_SR_PLUS_TIMES_F64ACC, torch.float64
        acc = 8
    elif a.case.startswith("orand_"):
        n = int(a.case[6:])
        A, B = inputs.boolean_u8(n, n, n, seed=6, density=0.01)
        sr, dt = mmsr.MM_SR_OR_AND_U8, torch.uint8
        acc = 1
    elif a.case in ("batched512", "batched_longk"):
        if a.case == "batched512":
            probs = inputs.batched_problems(count=512, seed=4)
        else:
            probs = inputs.batched_long_k_problems(seed=11)
        dA = [torch.from_numpy(p.A).cuda() for p in probs]
        dB = [torch.from_numpy(p.B).cuda() for p in probs]
        dC = [torch.empty((p.m, p.n), dtype=torch.float32 if p.semiring == mmsr.MM_SR_PLUS_TIMES_F32
                          else torch.int32, device="cuda") for p in probs]
        table = [(p.semiring, p.m, p.n, p.k, x, y, z) for p, x, y, z in zip(probs, dA, dB, dC)]
        need = mmsr.mm_batched_query(table)
        ws = torch.empty((need,), dtype=torch.uint8, device="cuda")
        for _ in range(a.reps):
            mmsr.mm_batched(table, ws, need)
        torch.cuda.synchronize()
        print("done", a.case, "reps", a.reps)
        return
    elif a.case.startswith("fa_strassen"):
        # FP64-accuracy Strassen-Winograd: fa_strassen<L>_<n>
        L = int(a.case[len("fa_strassen"):a.case.index("_", 3)])
        n = int(a.case[a.case.index("_", 3) + 1:])
        A, B = inputs.uniform_f64(n, n, n, seed=3)
        dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        del A, B
        dC = torch.empty((n, n), dtype=torch.float64, device="cuda")
        sr = mmsr.MM_SR_PLUS_TIMES_F64ACC
        p = mmsr.mm_plan_query(sr, L, n, n, n, 0)
        ws = torch.empty((int(p.workspace_min),), dtype=torch.uint8, device="cuda")
        for _ in range(a.reps):
            mmsr.mm_strassen(L, mmsr.MM_STRASSEN_WINOGRAD, sr, n, n, n, dA, dB, dC, ws, int(p.workspace_min))
        torch.cuda.synchronize()
        print("done", a.case, "reps", a.reps)
        return
    elif a.case.startswith("strassen") or a.case.startswith("tar_"):
        tar = a.case.startswith("tar_")
        L = 1 if tar else int(a.case[len("strassen"):a.case.index("_")])
        n = int(a.case[a.case.index("_") + 1:])
        A, B = inputs.uniform_f64(n, n, n, seed=3)
        dA = torch.from_numpy(A.astype("float32")).cuda()
        dB = torch.from_numpy(B.astype("float32")).cuda()
        dC = torch.empty((n, n), dtype=torch.float32, device="cuda")
        sr = mmsr.MM_SR_PLUS_TIMES_F32
        p = mmsr.mm_strassen_tar_query(1, sr, n, n, n) if tar else mmsr.mm_plan_query(sr, L, n, n, n, 0)
        ws = torch.empty((int(p.workspace_min),), dtype=torch.uint8, device="cuda")
        for _ in range(a.reps):
            if tar:
                mmsr.mm_strassen_tar(1, mmsr.MM_STRASSEN_WINOGRAD, sr, n, n, n, dA, dB, dC, ws, int(p.workspace_min))
            else:
                mmsr.mm_strassen(L, mmsr.MM_STRASSEN_WINOGRAD, sr, n, n, n, dA, dB, dC, ws, int(p.workspace_min))
        torch.cuda.synchronize()
        print("done", a.case, "reps", a.reps)
        return
    elif a.case.startswith("f64_"):
        n = int(a.case[4:])
        A, B = inputs.uniform_f64(n, n, n, seed=0)
        sr, dt = mmsr.MM_SR_PLUS_TIMES_F64, torch.float64
        acc = 8
    else:
        raise SystemExit("unknown case " + a.case)
    m = k = n
    if a.shape:
        m, n, k = (int(x) for x in a.shape.split(","))
        gen = {torch.float32: lambda: inputs.normal_f32(m, k, n, seed=2),
               torch.float64: lambda: inputs.uniform_f64(m, k, n, seed=3)}
        A, B = gen[dt]() if dt in gen else (A, B)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.empty((m, n), dtype=dt, device="cuda")
    p0 = mmsr.mm_plan_query(sr, -1, m, n, k, 0)
    budget = int(p0.workspace_min) + a.budget * m * n * acc
    if a.budget_bytes >= 0:
        budget = a.budget_bytes
    ws = torch.empty((max(budget, 16),), dtype=torch.uint8, device="cuda")
    print("plan", mmsr.mm_plan_query(sr, -1, m, n, k, budget).kernel, "budget", budget)
    for _ in range(a.reps):
        mmsr.mm_semiring(sr, m, n, k, dA, dB, dC, ws, budget)
    torch.cuda.synchronize()
    print("done", a.case, "reps", a.reps)


if __name__ == "__main__":
    main()
