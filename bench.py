#!/usr/bin/env python
"""Benchmark of the semiring MM library on GB300.

Headline workload: (min,+) tropical MM, n = 4096, int32 entries uniform in
[0, 1000] with 10% set to the +inf sentinel 2^30 (seed 1), run under the
five workspace budgets 0, 1, 2, 4 and 8 extra n x n int32 buffers (split-K
factors s = 1, 2, 3, 5, 9).  One step = the five calls; ops per call =
2 n^3 (one (x) = add and one (+) = min per term).

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
instead on a bounded row sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GOp/s & % of dtype peak at stated error vs plain FP64 path; peak workspace bytes"
N = 4096
BUDGETS = (0, 1, 2, 4, 8)  # extra n x n int32 buffers
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="mmsr", choices=["mmsr", "reference"])
    p.add_argument("--no-extras", action="store_true", help="skip the secondary workloads")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_id=None):
        self.path = tempfile.mktemp(prefix="mmsr_clocks_", suffix=".csv")
        cmd = ["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits",
               "-lms", "100"]
        if gpu_id:
            cmd.insert(1, "--id=" + gpu_id)
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                tok = [t.strip() for t in line.split(",")]
                if len(tok) < 9:
                    continue
                try:
                    sm.append(float(tok[1]))
                    smax.append(float(tok[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, tok[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def gpu_uuid():
    try:
        import torch

        u = torch.cuda.get_device_properties(torch.cuda.current_device()).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        return None


def sm_max_mhz():
    """Maximum SM clock of this GPU (nvidia-smi), 2070 MHz when unavailable."""
    try:
        cmd = ["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"]
        u = gpu_uuid()
        if u:
            cmd += ["-i", u]
        return float(subprocess.run(cmd, capture_output=True, text=True, timeout=20).stdout.split()[0])
    except Exception:
        return 2070.0


# ------------------------------------------------------------ measured peaks
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def source_sha(files):
    """Hash of the sources that define a kernel (csrc/ file names, in order)."""
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1911_05328_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_files, key):
    """DRAM bytes per launch from the committed ncu summary, or None when the
    kernel's sources changed after the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(key)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("source_sha") != source_sha(kernel_files):
        return None
    return rec.get("dram_bytes_per_launch")


def bench_config(world):
    """The workload both arms report (the reference arm times a row sample of it)."""
    return {"workload": "minplus_n4096_int32_inf10pct_seed1_budgets_0_1_2_4_8", "n": N,
            "budgets_buffers": list(BUDGETS), "l2": "flushed between timed steps (256 MiB write)",
            "parallelism": "replicas" if world > 1 else "single"}


# --------------------------------------------------------------- reference
def run_reference(args, rank):
    if rank != 0:
        return 0
    import oracle
    from paper_1911_05328_gb300 import inputs

    A, B = inputs.tropical_i32(N, N, N, seed=1)
    rows_per_step = 256
    rng = np.random.default_rng(0)
    times = []
    for it in range(args.warmup + args.steps):
        rows = np.sort(rng.choice(N, rows_per_step, replace=False))
        t0 = time.perf_counter()
        oracle.mm_minplus(A, B, rows=rows)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    ops = 2.0 * rows_per_step * N * N
    tot = sum(times)
    value = ops * len(times) / tot / 1e9
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GOp/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i64",
        "data": "synthetic",
        "config": bench_config(args.gpus),
        "cpu_baseline": {"value": value, "unit": "GOp/s", "cores": cores, "kind": "oracle",
                         "sample": "%d random rows of C (x 4096 x 4096) per step; the oracle has no "
                                   "budget, so every step is one product's row sample" % rows_per_step},
        "e2e": {"value": value, "unit": "GOp/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------------- mmsr
def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank)

    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist  # noqa: F811

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__

    __graft_entry__.build()
    from paper_1911_05328_gb300 import inputs, mmsr

    lib = mmsr.load()
    SR = mmsr.MM_SR_MIN_PLUS_I32
    stream = torch.cuda.current_stream()
    sp = int(stream.cuda_stream)

    A_h, B_h = inputs.tropical_i32(N, N, N, seed=1)
    dA = torch.from_numpy(A_h).cuda()
    dB = torch.from_numpy(B_h).cuda()
    outs = [torch.empty((N, N), dtype=torch.int32, device="cuda") for _ in BUDGETS]
    max_budget = max(BUDGETS) * N * N * 4
    ws = torch.empty((max_budget,), dtype=torch.uint8, device="cuda")
    flush = torch.empty((L2_FLUSH_BYTES,), dtype=torch.uint8, device="cuda")
    plans = [mmsr.mm_plan_query(SR, -1, N, N, N, b * N * N * 4) for b in BUDGETS]

    def one_step():
        for b, C in zip(BUDGETS, outs):
            mmsr.mm_semiring(SR, N, N, N, dA, dB, C, ws, b * N * N * 4, sp)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    consistent = all(bool(torch.equal(outs[0], C)) for C in outs[1:])

    # roofline denominators: measured probe of the fused add-min instruction
    import ctypes

    rate, pms = ctypes.c_double(), ctypes.c_double()
    lib.mm_probe_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.mm_probe_peak(0, 2000, sp, ctypes.byref(rate), ctypes.byref(pms))
    lib.mm_probe_peak(0, 20000, sp, ctypes.byref(rate), ctypes.byref(pms))
    alu_peak_tops = rate.value / 1e12
    lib.mm_probe_peak(1, 20000, sp, ctypes.byref(rate), ctypes.byref(pms))
    alu_peak_u16x2_tops = rate.value / 1e12

    # ---------------------------------------------------------- timed region
    per_budget_ms = [0.0] * len(BUDGETS)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(BUDGETS) + 1)] for _ in range(args.steps)]
    sampler = ClockSampler(gpu_uuid())
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    lib.mm_trace_enable(1)
    for s in range(args.steps):
        flush.zero_()  # evict L2 between timed steps (not timed)
        e = ev[s]
        e[0].record(stream)
        for i, (b, C) in enumerate(zip(BUDGETS, outs)):
            mmsr.mm_semiring(SR, N, N, N, dA, dB, C, ws, b * N * N * 4, sp)
            e[i + 1].record(stream)
    torch.cuda.synchronize()
    lib.mm_trace_enable(0)
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    step_ms = []
    for s in range(args.steps):
        e = ev[s]
        step_ms.append(e[0].elapsed_time(e[-1]))
        for i in range(len(BUDGETS)):
            per_budget_ms[i] += e[i].elapsed_time(e[i + 1])
    total_ms = sum(step_ms)
    if dist:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())

    # per-kernel trace
    kernels = {}
    launches_total = 0
    for kid in range(lib.mm_trace_kernel_count()):
        cnt, tot = ctypes.c_int64(), ctypes.c_double()
        lib.mm_trace_summary.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]
        lib.mm_trace_summary(kid, ctypes.byref(cnt), ctypes.byref(tot))
        if cnt.value:
            lib.mm_trace_kernel_name.restype = ctypes.c_char_p
            kernels[lib.mm_trace_kernel_name(kid).decode()] = {"launches": cnt.value, "ms": tot.value}
            launches_total += cnt.value

    ops_per_call = 2.0 * N * N * N
    ops_per_step = ops_per_call * len(BUDGETS)
    value = world * ops_per_step * args.steps / (total_ms * 1e-3) / 1e9
    # dominant kernel: the leaf that did the work (the packed 2 x 16-bit leaf
    # when the device-side range scan allows it, else the 32-bit leaf)
    leaf_name = max(("minplus16_leaf", "minplus_leaf"), key=lambda k: kernels.get(k, {"ms": 0.0})["ms"])
    leaf = kernels[leaf_name]
    # every call launches both leaves; the one that is not chosen exits at once
    leaf_avg_ms = leaf["ms"] / (args.steps * len(BUDGETS))
    achieved_tops = ops_per_call / (leaf_avg_ms * 1e-3) / 1e12
    peak_tops = alu_peak_u16x2_tops if leaf_name == "minplus16_leaf" else alu_peak_tops
    traffic = ncu_traffic(["minplus.cu", "minplus_tile.cuh"], leaf_name + "_n4096")
    per_budget = []
    for i, b in enumerate(BUDGETS):
        ms = per_budget_ms[i] / args.steps
        per_budget.append({"budget_buffers": b, "budget_bytes": b * N * N * 4, "split_k": plans[i].split_k,
                           "workspace_used_bytes": int(plans[i].workspace_used), "ms": ms,
                           "gops": ops_per_call / (ms * 1e-3) / 1e9})

    # ----------------------------------------------------- end to end (host)
    # Every step uploads its inputs from pinned host memory and downloads
    # every result.  Uploads and downloads run on two copy streams (the two
    # directions use separate copy engines) with double-buffered device
    # inputs and outputs: a step's uploads overlap the previous step's
    # kernels and each result's download overlaps the next product.  On one
    # shared copy stream the next step's upload queued behind the last
    # download, serialising every step boundary.
    e2e = None
    if True:
        pA = torch.from_numpy(A_h).pin_memory()
        pB = torch.from_numpy(B_h).pin_memory()
        pC = [torch.empty((N, N), dtype=torch.int32).pin_memory() for _ in BUDGETS]
        dA2 = [dA, torch.empty_like(dA)]
        dB2 = [dB, torch.empty_like(dB)]
        outs2 = [outs, [torch.empty_like(c) for c in outs]]
        cs_up, cs_down = torch.cuda.Stream(), torch.cuda.Stream()
        e2e_steps = max(2, min(args.steps, 10))
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        in_ready = [torch.cuda.Event() for _ in range(2)]
        in_free = [torch.cuda.Event() for _ in range(2)]
        out_ready = [[torch.cuda.Event() for _ in BUDGETS] for _ in range(2)]
        out_free = [[torch.cuda.Event() for _ in BUDGETS] for _ in range(2)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        evs[0].record(stream)
        cs_up.wait_event(evs[0])
        cs_down.wait_event(evs[0])
        for t in range(e2e_steps):
            j = t & 1
            with torch.cuda.stream(cs_up):
                if t >= 2:
                    cs_up.wait_event(in_free[j])
                dA2[j].copy_(pA, non_blocking=True)
                dB2[j].copy_(pB, non_blocking=True)
                in_ready[j].record(cs_up)
            stream.wait_event(in_ready[j])
            for i, b in enumerate(BUDGETS):
                if t >= 2:
                    stream.wait_event(out_free[j][i])
                mmsr.mm_semiring(SR, N, N, N, dA2[j], dB2[j], outs2[j][i], ws, b * N * N * 4, sp)
                out_ready[j][i].record(stream)
                with torch.cuda.stream(cs_down):
                    cs_down.wait_event(out_ready[j][i])
                    pC[i].copy_(outs2[j][i], non_blocking=True)
                    out_free[j][i].record(cs_down)
            in_free[j].record(stream)
        stream.wait_stream(cs_up)
        stream.wait_stream(cs_down)
        evs[1].record(stream)
        torch.cuda.synchronize()
        e2e_ms = evs[0].elapsed_time(evs[1])
        if dist:
            t = torch.tensor([e2e_ms], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_ms = float(t.item())
        e2e = {"value": world * ops_per_step * e2e_steps / (e2e_ms * 1e-3) / 1e9, "unit": "GOp/s",
               "h2d_bytes_per_step": int(A_h.nbytes + B_h.nbytes),
               "d2h_bytes_per_step": int(sum(c.numel() * 4 for c in pC)), "steps": e2e_steps,
               "overlap": "uploads and downloads on two copy streams, double-buffered device buffers"}
        consistent = consistent and all(bool(torch.equal(pC[0], c)) for c in pC[1:])

    # ----------------------------------------------------------- extras
    extras = {}
    if not args.no_extras and rank == 0:
        extras = run_extras(mmsr, lib, torch, sp)

    # ------------------------------------------------------ CPU baseline
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle

        rows = np.arange(0, N, 4, dtype=np.int64)  # 1024 rows, every 4th
        t0 = time.perf_counter()
        oracle.mm_minplus(A_h, B_h, rows=rows)
        dt = time.perf_counter() - t0
        cpu = {"value": 2.0 * len(rows) * N * N / dt / 1e9, "unit": "GOp/s", "cores": oracle.num_threads(),
               "kind": "oracle", "sample": "%d of 4096 rows (every 4th) of one n=4096 product, %.1f s"
                                           % (len(rows), dt)}

    peaks, peak_src = measured_peaks()
    line = {
        "metric": METRIC, "value": value, "unit": "GOp/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i32", "data": "synthetic",
        "config": bench_config(world),
        "error": "bit-exact vs int64 oracle (tests); budgets agree: %s" % consistent,
        "pct_of_dtype_peak": 100.0 * (value / world) / (peak_tops * 1e3),
        "peak_workspace_bytes": int(max(p.workspace_used for p in plans)),
        "per_budget": per_budget,
        "roofline": {"bound": "alu", "kernel": leaf_name, "achieved": achieved_tops,
                     "peak": peak_tops, "unit": "TOp/s", "frac": achieved_tops / peak_tops,
                     "traffic": traffic,
                     "peak_source": ("measured: mm_probe_peak fused add-min on packed 2 x u16 "
                                     "(4 ops/lane-instr), all SMs" if leaf_name == "minplus16_leaf" else
                                     "measured: mm_probe_peak fused add-min u32 (2 ops/lane-instr), all SMs"),
                     "alu_peak_u32_tops": alu_peak_tops, "alu_peak_u16x2_tops": alu_peak_u16x2_tops},
        "kernels": kernels,
        "gpu_launches": launches_total,
        "clocks": clocks,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "peaks_file": peak_src,
        "extras": extras,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def _probe(lib, sp, kind, iters):
    """Measured rate (ops/s) of one instruction kind on every SM: a short
    warm-up launch, then the timed one (mm_probe_peak, include/mmsr_probe.h)."""
    import ctypes

    rate, pms = ctypes.c_double(), ctypes.c_double()
    lib.mm_probe_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.mm_probe_peak(kind, max(iters // 10, 1), sp, ctypes.byref(rate), ctypes.byref(pms))
    lib.mm_probe_peak(kind, iters, sp, ctypes.byref(rate), ctypes.byref(pms))
    return rate.value


def _roof(bound, achieved, peak, unit, peak_source):
    """Roofline record of one kernel or call: achieved vs peak in `unit`."""
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": (achieved / peak) if peak else None, "peak_source": peak_source}


def _time_call(torch, fn, reps):
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def run_extras(mmsr, lib, torch, sp):
    """Secondary workloads (not the headline): reported for context."""
    import ctypes

    from paper_1911_05328_gb300 import inputs

    lib.mm_trace_summary.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]

    out = {}
    # roofline denominators of the CUDA-core rows: measured probes (bf16
    # tensor peaks come from the measured-peaks file)
    peaks, src = measured_peaks()
    u16_peak = _probe(lib, sp, 1, 20000) / 1e12
    # boolean leaf: one three-input logic op covers 32 terms (32 ANDs + 32
    # ORs) and issues on the same ALU pipe as the packed add-min, whose probe
    # issues exactly one ALU instruction per step: ALU rate x 64 ops
    lop_peak = u16_peak / 4 * 64
    # FP64: 2 FMA lanes per SM per clock (the nominal 1.25 TFLOP/s at the
    # maximum clock); the FMA-chain probe reaches ~89% of it
    mhz = sm_max_mhz()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    fp64_peak = sms * 2 * 2 * mhz * 1e6 / 1e12
    fp64_src = "derived: %d SMs x 2 FP64 FMA/clk x 2 FLOP x %.0f MHz" % (sms, mhz)
    bf16_src = "%s: bf16 dense burst (cuBLAS)" % src
    # FP64 classic n=256, uniform[-1,1], seed 0, budget 0 (plain FP64 path)
    A, B = inputs.uniform_f64(256, 256, 256, seed=0)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.empty((256, 256), dtype=torch.float64, device="cuda")
    ms = _time_call(torch, lambda: mmsr.mm_semiring(mmsr.MM_SR_PLUS_TIMES_F64, 256, 256, 256, dA, dB, dC, None, 0, sp), 50)
    out["fp64_n256_budget0"] = {"ms": ms, "gops": 2 * 256 ** 3 / (ms * 1e-3) / 1e9,
                                "roofline": _roof("fp64", 2 * 256 ** 3 / (ms * 1e-3) / 1e12, fp64_peak,
                                                  "TFLOP/s", fp64_src)}
    # FP64 DFMA path at n=8192 (comparator of the FP32 split-precision path)
    n = 8192
    A, B = inputs.uniform_f64(n, n, n, seed=2)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.empty((n, n), dtype=torch.float64, device="cuda")
    ms = _time_call(torch, lambda: mmsr.mm_semiring(mmsr.MM_SR_PLUS_TIMES_F64, n, n, n, dA, dB, dC, None, 0, sp), 2)
    out["fp64_dfma_n8192"] = {"ms": ms, "gops": 2 * n ** 3 / (ms * 1e-3) / 1e9,
                              "roofline": _roof("fp64", 2 * n ** 3 / (ms * 1e-3) / 1e12, fp64_peak,
                                                "TFLOP/s", fp64_src)}
    del dA, dB, dC
    # FP32 mode n=8192, normal(0,1), seed 2: bf16x3 split products on tcgen05
    A, B = inputs.normal_f32(n, n, n, seed=2)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.empty((n, n), dtype=torch.float32, device="cuda")
    sr = mmsr.MM_SR_PLUS_TIMES_F32
    wmin = int(mmsr.mm_plan_query(sr, -1, n, n, n, 0).workspace_min)
    ws = torch.empty((wmin,), dtype=torch.uint8, device="cuda")
    lib.mm_trace_enable(1)
    ms = _time_call(torch, lambda: mmsr.mm_semiring(sr, n, n, n, dA, dB, dC, ws, wmin, sp), 10)
    lib.mm_trace_enable(0)
    cnt, tot = ctypes.c_int64(), ctypes.c_double()
    lib.mm_trace_summary(5, ctypes.byref(cnt), ctypes.byref(tot))  # tc_bf16x3
    gemm_ms = tot.value / max(cnt.value, 1)
    issued = 3 * 2.0 * n ** 3 / (gemm_ms * 1e-3) / 1e12
    out["fp32_bf16x3_n8192"] = {
        "ms": ms, "gops_useful": 2 * n ** 3 / (ms * 1e-3) / 1e9, "gemm_ms": gemm_ms,
        "tensor_tflops_issued": issued, "frac_of_bf16_peak": issued / peaks["bf16_tflops"],
        "roofline": _roof("tensor", issued, peaks["bf16_tflops"], "TFLOP/s", bf16_src),
        "peak_source": src, "workspace_bytes": wmin,
        "speedup_vs_fp64_dfma": out["fp64_dfma_n8192"]["ms"] / ms,
        "error": "rel. Frobenius vs FP64 oracle on 512 sampled rows <= 1e-5 (tests)"}
    import ctypes

    rate, pms = ctypes.c_double(), ctypes.c_double()
    del dA, dB, dC, ws
    torch.cuda.empty_cache()
    # FP64-accuracy mode at n = 8192 (uniform[-1,1]) beside the plain FP64
    # path at the same size and the same stated accuracy (1e-12)
    A, B = inputs.uniform_f64(n, n, n, seed=3)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    del A, B
    dC = torch.empty((n, n), dtype=torch.float64, device="cuda")
    sr = mmsr.MM_SR_PLUS_TIMES_F64ACC
    wmin = int(mmsr.mm_plan_query(sr, -1, n, n, n, 0).workspace_min)
    ws = torch.empty((wmin,), dtype=torch.uint8, device="cuda")
    lib.mm_trace_enable(1)
    ms = _time_call(torch, lambda: mmsr.mm_semiring(sr, n, n, n, dA, dB, dC, ws, wmin, sp), 3)
    lib.mm_trace_enable(0)
    lib.mm_trace_summary(8, ctypes.byref(cnt), ctypes.byref(tot))  # tc_f64acc
    gemm_ms = tot.value / max(cnt.value, 1)
    issued = 28 * 2.0 * n ** 3 / (gemm_ms * 1e-3) / 1e12
    out["fp64acc_n8192"] = {
        "ms": ms, "gflops_useful": 2 * n ** 3 / (ms * 1e-3) / 1e9, "gemm_ms": gemm_ms,
        "tensor_tflops_issued_28_slice_products": issued, "frac_of_bf16_peak": issued / peaks["bf16_tflops"],
        "roofline": _roof("tensor", issued, peaks["bf16_tflops"], "TFLOP/s", bf16_src),
        "workspace_bytes": wmin, "speedup_vs_fp64_dfma": out["fp64_dfma_n8192"]["ms"] / ms,
        "error": "rel. Frobenius vs FP64 oracle <= 1e-12 (tests; 4.6e-15 at n=16384)"}
    del dA, dB, dC, ws
    torch.cuda.empty_cache()
    out["batched_512"] = run_batched_extras(mmsr, lib, torch, sp, ctypes, peaks["bf16_tflops"], u16_peak, bf16_src)
    out["strassen_fp32_n16384"] = run_strassen_extras(mmsr, lib, torch, sp, ctypes, peaks["bf16_tflops"], bf16_src)
    out["closure_minplus_n4096"] = run_closure_extras(mmsr, torch, sp, u16_peak)
    out["orand_n4096"] = run_orand_extras(mmsr, lib, torch, sp, ctypes, lop_peak)
    out["fp64_fma_probe_tflops"] = _probe(lib, sp, 2, 2000) / 1e12
    out["fp64_peak_derived_tflops"] = fp64_peak
    out["addmin_u16x2_probe_tops"] = u16_peak
    out["orand_peak_derived_tops"] = lop_peak
    out["fp32_fma_probe_tflops"] = _probe(lib, sp, 3, 20000) / 1e12
    torch.cuda.empty_cache()
    return out


def run_batched_extras(mmsr, lib, torch, sp, ctypes, bf16_peak, u16_peak, bf16_src):
    """512 problems (m, n, k log-uniform in [64, 2048], 70% FP32 (+,x) with
    normal(0,1) entries, 30% (min,+) with integers in [0, 1000], seed 4) in
    one persistent launch, captured once in a CUDA graph and replayed."""
    from paper_1911_05328_gb300 import inputs

    probs = inputs.batched_problems(count=512, seed=4)
    dA = [torch.from_numpy(p.A).cuda() for p in probs]
    dB = [torch.from_numpy(p.B).cuda() for p in probs]
    dC = [torch.empty((p.m, p.n), dtype=torch.float32 if p.semiring == mmsr.MM_SR_PLUS_TIMES_F32 else torch.int32,
                      device="cuda") for p in probs]
    table = [(p.semiring, p.m, p.n, p.k, a, b, c) for p, a, b, c in zip(probs, dA, dB, dC)]
    need = mmsr.mm_batched_query(table)
    ws = torch.empty((need,), dtype=torch.uint8, device="cuda")
    ops = sum(2.0 * p.m * p.n * p.k for p in probs)
    ops_fp32 = sum(2.0 * p.m * p.n * p.k for p in probs if p.semiring == mmsr.MM_SR_PLUS_TIMES_F32)
    mmsr.mm_batched(table, ws, need, stream=sp)  # sets kernel attributes before capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        mmsr.mm_batched(table, ws, need, stream=torch.cuda.current_stream())
    ms = _time_call(torch, g.replay, 10)
    # per-kernel split from three traced eager calls (graph replays carry no
    # trace events)
    lib.mm_trace_enable(1)
    for _ in range(3):
        mmsr.mm_batched(table, ws, need, stream=sp)
    torch.cuda.synchronize()
    lib.mm_trace_enable(0)
    lib.mm_trace_kernel_name.restype = ctypes.c_char_p
    split = {}
    for kid in range(lib.mm_trace_kernel_count()):
        cnt, tot = ctypes.c_int64(), ctypes.c_double()
        lib.mm_trace_summary(kid, ctypes.byref(cnt), ctypes.byref(tot))
        if cnt.value:
            split[lib.mm_trace_kernel_name(kid).decode()] = tot.value / 3
    # ideal time: every FP32 product's three bf16 split products at the tensor
    # peak plus every (min,+) product at the packed add-min peak
    ideal_ms = (3 * ops_fp32 / (bf16_peak * 1e12) + (ops - ops_fp32) / (u16_peak * 1e12)) * 1e3
    res = {"ms": ms, "gops": ops / (ms * 1e-3) / 1e9, "ops": ops, "fp32_share_of_ops": ops_fp32 / ops,
           "roofline": _roof("tensor (FP32 tiles) + alu ((min,+) tiles)", ops / (ms * 1e-3) / 1e12,
                             ops / (ideal_ms * 1e-3) / 1e12, "TOp/s",
                             bf16_src + "; measured packed add-min probe"),
           "kernel_ms_eager": split,
           "workspace_bytes": int(need), "launch": "one CUDA graph: memset + 2 pre-passes + persistent tcgen05 kernel (FP32 tiles) + "
                     "packed (min,+) tile launch + 32-bit (min,+) launch (exits at once when unused)",
           "error": "bit-exact (min,+), <= 1e-5 FP32, per problem (tests)"}
    del dA, dB, dC, ws
    torch.cuda.empty_cache()
    return res


def run_orand_extras(mmsr, lib, torch, sp, ctypes, lop_peak):
    """(or, and) semiring, n = 4096, 0/1 entries with density 1% (seed 6):
    the bit-packed leaf, budget = the plan's minimum (packing buffers)."""
    from paper_1911_05328_gb300 import inputs

    n = 4096
    A, B = inputs.boolean_u8(n, n, n, seed=6, density=0.01)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.empty((n, n), dtype=torch.uint8, device="cuda")
    sr = mmsr.MM_SR_OR_AND_U8
    w = int(mmsr.mm_plan_query(sr, -1, n, n, n, 0).workspace_min)
    ws = torch.empty((max(w, 16),), dtype=torch.uint8, device="cuda")
    fn = lambda: mmsr.mm_semiring(sr, n, n, n, dA, dB, dC, ws, w, sp)
    ms = _time_call(torch, fn, 20)
    lib.mm_trace_enable(1)
    for _ in range(5):
        fn()
    torch.cuda.synchronize()
    lib.mm_trace_enable(0)
    lib.mm_trace_kernel_name.restype = ctypes.c_char_p
    split = {}
    for kid in range(lib.mm_trace_kernel_count()):
        cnt, tot = ctypes.c_int64(), ctypes.c_double()
        lib.mm_trace_summary(kid, ctypes.byref(cnt), ctypes.byref(tot))
        if cnt.value:
            split[lib.mm_trace_kernel_name(kid).decode()] = tot.value / 5
    res = {"ms": ms, "gops": 2.0 * n ** 3 / (ms * 1e-3) / 1e9, "workspace_bytes": w, "kernel_ms": split,
           "roofline": _roof("alu", 2.0 * n ** 3 / (ms * 1e-3) / 1e12, lop_peak, "TOp/s",
                             "derived: measured ALU-pipe rate (packed add-min probe / 4) x 64 ops per "
                             "32-bit and-or"),
           "error": "bit-exact vs oracle (tests)"}
    del dA, dB, dC, ws
    torch.cuda.empty_cache()
    return res


def run_closure_extras(mmsr, torch, sp, u16_peak):
    """(min,+) closure (all-pairs shortest paths) of a 4096-vertex graph with
    10% arcs of length in [0, 1000] (seed 1) by repeated squaring, one extra
    n x n buffer of budget per squaring: all 12 squarings, and stopping at
    the fixed point."""
    n = 4096
    rng = np.random.default_rng(1)
    D = rng.integers(0, 1001, size=(n, n)).astype(np.int32)
    D[rng.random((n, n)) >= 0.1] = mmsr.INF
    dA = torch.from_numpy(D).cuda()
    dC = torch.empty_like(dA)
    sr = mmsr.MM_SR_MIN_PLUS_I32
    p = mmsr.mm_closure_query(sr, n, 0)
    budget = int(p.workspace_min) + n * n * 4
    ws = torch.empty((budget,), dtype=torch.uint8, device="cuda")
    res = {}
    for name, flags in (("all_squarings", 0), ("early_exit", mmsr.MM_CLOSURE_EARLY_EXIT)):
        sq = []

        def fn():
            sq.append(mmsr.mm_closure(sr, n, dA, dC, ws, budget, flags=flags, stream=sp)[1])

        ms = _time_call(torch, fn, 3)
        res[name] = {"ms": ms, "squarings": sq[-1],
                     "gops": sq[-1] * 2.0 * n ** 3 / (ms * 1e-3) / 1e9,
                     "workspace_bytes": budget,
                     "roofline": _roof("alu", sq[-1] * 2.0 * n ** 3 / (ms * 1e-3) / 1e12, u16_peak, "TOp/s",
                                       "measured: mm_probe_peak packed add-min, all SMs")}
    del dA, dC, ws
    torch.cuda.empty_cache()
    return res


def run_strassen_extras(mmsr, lib, torch, sp, ctypes, bf16_peak, bf16_src):
    """Strassen-Winograd, FP32 mode, n = 16384 (uniform[-1,1], seed 3, cast
    to float32): classic (L = 0) and L = 1..4, per-level time, classic-
    equivalent GOp/s, workspace as a multiple of n^2 * 4 bytes and the time
    split between operand sums, leaf products and post-additions."""
    from paper_1911_05328_gb300 import inputs

    n = 16384
    A, B = inputs.uniform_f64(n, n, n, seed=3)
    dA64, dB64 = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dA = dA64.float()
    dB = dB64.float()
    del A, B
    dC = torch.empty((n, n), dtype=torch.float32, device="cuda")
    sr = mmsr.MM_SR_PLUS_TIMES_F32
    res = {}
    names = {}
    lib.mm_trace_kernel_name.restype = ctypes.c_char_p
    for kid in range(lib.mm_trace_kernel_count()):
        names[kid] = lib.mm_trace_kernel_name(kid).decode()
    for L in range(0, 5):
        p = mmsr.mm_plan_query(sr, L, n, n, n, 0)
        ws = torch.empty((max(int(p.workspace_min), 16),), dtype=torch.uint8, device="cuda")
        fn = lambda: mmsr.mm_strassen(L, mmsr.MM_STRASSEN_WINOGRAD, sr, n, n, n, dA, dB, dC, ws,
                                      int(p.workspace_min), sp)
        fn()
        torch.cuda.synchronize()
        lib.mm_trace_enable(1)
        ms = _time_call(torch, fn, 3)
        lib.mm_trace_enable(0)
        split = {}
        for kid, nm in names.items():
            cnt, tot = ctypes.c_int64(), ctypes.c_double()
            lib.mm_trace_summary(kid, ctypes.byref(cnt), ctypes.byref(tot))
            if cnt.value:
                split[nm] = tot.value / 4  # 1 untimed-warm call + 3 timed calls traced
        res["L%d" % L] = {"ms": ms, "gops_classic_equiv": 2.0 * n ** 3 / (ms * 1e-3) / 1e9,
                          "workspace_bytes": int(p.workspace_min),
                          "workspace_n2x4B": p.workspace_min / (n * n * 4.0), "kernel_ms": split}
        leaf_ms = split.get("tc_bf16x3", 0.0)
        if leaf_ms > 0:
            # 7^L leaf products of size n / 2^L, three bf16 split products each
            leaf_tf = 3 * 2.0 * (n >> L) ** 3 * 7 ** L / (leaf_ms * 1e-3) / 1e12
            res["L%d" % L]["leaf_roofline"] = _roof("tensor", leaf_tf, bf16_peak, "TFLOP/s", bf16_src)
            res["L%d" % L]["leaf_share_of_time"] = leaf_ms / ms
        del ws
        torch.cuda.empty_cache()
    # TAR-Strassen: one level, products added into C's quadrants by the leaf
    # epilogue in conflict-free waves (no product temporaries)
    p = mmsr.mm_strassen_tar_query(sr, n, n, n)
    ws = torch.empty((int(p.workspace_min),), dtype=torch.uint8, device="cuda")
    fn = lambda: mmsr.mm_strassen_tar(mmsr.MM_STRASSEN_WINOGRAD, sr, n, n, n, dA, dB, dC, ws,
                                      int(p.workspace_min), sp)
    ms = _time_call(torch, fn, 3)
    res["tar_L1"] = {"ms": ms, "gops_classic_equiv": 2.0 * n ** 3 / (ms * 1e-3) / 1e9,
                     "workspace_bytes": int(p.workspace_min), "workspace_n2x4B": p.workspace_min / (n * n * 4.0)}
    del ws
    torch.cuda.empty_cache()
    # STAR-Strassen-1 mixed plans: c classic in-place levels over L Strassen
    # levels; the workspace of one block product only
    for c, L in ((1, 1), (1, 2), (2, 1), (2, 2)):
        p = mmsr.mm_star_strassen_query(c, L, sr, n, n, n)
        ws = torch.empty((int(p.workspace_min),), dtype=torch.uint8, device="cuda")
        fn = lambda: mmsr.mm_star_strassen(c, L, mmsr.MM_STRASSEN_WINOGRAD, sr, n, n, n, dA, dB, dC, ws,
                                           int(p.workspace_min), sp)
        ms = _time_call(torch, fn, 3)
        res["star_c%d_L%d" % (c, L)] = {"ms": ms, "gops_classic_equiv": 2.0 * n ** 3 / (ms * 1e-3) / 1e9,
                                        "workspace_bytes": int(p.workspace_min),
                                        "workspace_n2x4B": p.workspace_min / (n * n * 4.0)}
        del ws
        torch.cuda.empty_cache()
    del dC
    # FP64-accuracy mode (28 digit-slice products per leaf) at the same size
    dC64 = torch.empty((n, n), dtype=torch.float64, device="cuda")
    sr64 = mmsr.MM_SR_PLUS_TIMES_F64ACC
    for L in range(0, 3):
        p = mmsr.mm_plan_query(sr64, L, n, n, n, 0)
        ws = torch.empty((int(p.workspace_min),), dtype=torch.uint8, device="cuda")
        fn = lambda: mmsr.mm_strassen(L, mmsr.MM_STRASSEN_WINOGRAD, sr64, n, n, n, dA64, dB64, dC64, ws,
                                      int(p.workspace_min), sp)
        ms = _time_call(torch, fn, 2)
        res["fp64acc_L%d" % L] = {"ms": ms, "gflops_classic_equiv": 2.0 * n ** 3 / (ms * 1e-3) / 1e9,
                                  "workspace_bytes": int(p.workspace_min),
                                  "workspace_n2x8B": p.workspace_min / (n * n * 8.0)}
        del ws
        torch.cuda.empty_cache()
    del dA, dB, dA64, dB64, dC64
    torch.cuda.empty_cache()
    # the rectangular product m = 12288, k = 16384, n = 8192, FP32 mode
    m, k, n2 = 12288, 16384, 8192
    A, B = inputs.uniform_f64(m, k, n2, seed=3)
    dA = torch.from_numpy(A.astype(np.float32)).cuda()
    dB = torch.from_numpy(B.astype(np.float32)).cuda()
    del A, B
    dC = torch.empty((m, n2), dtype=torch.float32, device="cuda")
    for L in range(0, 4):
        p = mmsr.mm_plan_query(sr, L, m, n2, k, 0)
        ws = torch.empty((max(int(p.workspace_min), 16),), dtype=torch.uint8, device="cuda")
        fn = lambda: mmsr.mm_strassen(L, mmsr.MM_STRASSEN_WINOGRAD, sr, m, n2, k, dA, dB, dC, ws,
                                      int(p.workspace_min), sp)
        ms = _time_call(torch, fn, 3)
        res["rect_12288x16384x8192_L%d" % L] = {"ms": ms, "gops_classic_equiv": 2.0 * m * n2 * k / (ms * 1e-3) / 1e9,
                                               "workspace_bytes": int(p.workspace_min)}
        del ws
        torch.cuda.empty_cache()
    del dA, dB, dC
    torch.cuda.empty_cache()
    return res


if __name__ == "__main__":
    sys.exit(main())
