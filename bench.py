#!/usr/bin/env python
"""Benchmark of the semiring MM library on GB300.

Headline workload: FP64-accuracy (+,x) matrix multiplication by
Strassen-Winograd, square n = 16384, entries i.i.d. uniform[-1, 1] (seed 3;
A drawn before B), HEADLINE_LEVELS recursion levels over the tensor-core leaf
that sums integer digit slices of each operand (six 8-bit slices and 21 bf16
slice products up to two levels, seven 7-bit slices and 28 products beyond;
exact integer accumulation, one FP64 combination per output).  One step = one
product through ``mm_strassen``; ``value`` = classic-equivalent 2 n^3 / step
time (GOp/s).  The stated accuracy is a relative Frobenius error <= 1e-12 against
the FP64 oracle, measured on 512 sampled rows.  Beside it, on the same inputs
and at the same stated accuracy, the plain FP64 CUDA-core path (DFMA leaf).

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
instead, on a bounded row sample of the same product per step.
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
N = 16384
SEED = 3
HEADLINE_LEVELS = 2
TOL_F64 = 1e-12
SAMPLE_ROWS = 512


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="mmsr", choices=["mmsr", "reference"])
    p.add_argument("--levels", type=int, default=HEADLINE_LEVELS, help="Strassen levels of the headline")
    p.add_argument("--no-extras", action="store_true", help="skip the secondary workloads")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle (baseline and errors)")
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


F64ACC_SOURCES = ["tc_f64acc.cu", "tcgen05.cuh"]


def f64acc_products(levels):
    """bf16 slice products per leaf k-step of the FP64-accuracy scheme the
    library picks at this Strassen depth (6 slices up to two levels, else 7)."""
    return 21 if levels <= 2 else 28


def bench_config(world, levels=HEADLINE_LEVELS):
    """The workload both arms report (the reference arm times a row sample of it)."""
    sl = 6 if levels <= 2 else 7
    return {"workload": "fp64acc_strassen_winograd_L%d_n%d_uniform_seed%d" % (levels, N, SEED),
            "semiring": "(+,x) FP64-accuracy (%d digit slices, %d bf16 tensor-core products, exact sums)"
                        % (sl, f64acc_products(levels)),
            "n": N, "levels": levels, "variant": "Strassen-Winograd",
            "l2": "inputs larger than L2 (2 x 2 GiB FP64)",
            "parallelism": "replicas" if world > 1 else "single"}


def sample_rows(m, count=SAMPLE_ROWS):
    """Rows of C whose error is measured: an even spread plus the quadrant
    edges of up to four halvings (where a Strassen level puts a block edge)."""
    base = set(np.linspace(0, m - 1, max(count - 40, 1)).round().astype(np.int64).tolist())
    for lvl in range(1, 5):
        q = m >> lvl
        if q <= 0:
            break
        for b in range(0, m, q):
            base.update(x for x in (b - 1, b) if 0 <= x < m)
    return np.array(sorted(base), dtype=np.int64)


def rel_fro(C, R):
    C = np.asarray(C, np.float64)
    R = np.asarray(R, np.float64)
    return float(np.linalg.norm(C - R) / np.linalg.norm(R))


# --------------------------------------------------------------- reference
def run_reference(args, rank):
    """The oracle (plain C triple loop, FP64, OpenMP over rows) on a bounded
    row sample of the headline product per step."""
    if rank != 0:
        return 0
    import oracle
    from paper_1911_05328_gb300 import inputs

    A, B = inputs.uniform_f64(N, N, N, seed=SEED)
    rows_per_step = 64
    rng = np.random.default_rng(0)
    times = []
    for it in range(args.warmup + args.steps):
        rows = np.sort(rng.choice(N, rows_per_step, replace=False))
        t0 = time.perf_counter()
        oracle.mm_f64(A, B, rows=rows)
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
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": bench_config(args.gpus, args.levels),
        "cpu_baseline": {"value": value, "unit": "GOp/s", "cores": cores, "kind": "oracle",
                         "sample": "%d random rows of C (x %d x %d) per step, FP64 triple loop; "
                                   "the oracle computes the classic definition, so its GOp/s counts "
                                   "the same 2 n^3 per product" % (rows_per_step, N, N)},
        "e2e": {"value": value, "unit": "GOp/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ helpers
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


def _time_call(torch, fn, reps, stream=None):
    """Mean milliseconds per call over `reps` calls after one untimed call,
    CUDA events on the launching stream."""
    fn()
    torch.cuda.synchronize()
    s = stream if stream is not None else torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(reps):
        fn()
    b.record(s)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _trace(lib, ctypes):
    """Per-kernel launches and total milliseconds recorded by the library's
    event trace since it was last enabled."""
    lib.mm_trace_summary.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]
    lib.mm_trace_kernel_name.restype = ctypes.c_char_p
    out = {}
    for kid in range(lib.mm_trace_kernel_count()):
        cnt, tot = ctypes.c_int64(), ctypes.c_double()
        lib.mm_trace_summary(kid, ctypes.byref(cnt), ctypes.byref(tot))
        if cnt.value:
            out[lib.mm_trace_kernel_name(kid).decode()] = {"launches": cnt.value, "ms": tot.value}
    return out


class ErrBook:
    """Sampled GPU rows waiting for the oracle's rows of the same product.
    The oracle runs after every GPU measurement, once per input set, so no
    CPU work overlaps a timed region.  FP sets record the relative Frobenius
    error; (min,+) sets record whether the rows are bit-identical."""

    def __init__(self):
        self.sets = {}   # key -> (make() -> (A, B), rows, kind)
        self.items = []  # (key, record dict, field, gpu rows)
        self.cache = {}

    def add_set(self, key, make, rows, kind="f64"):
        self.sets.setdefault(key, (make, rows, kind))

    def add(self, key, record, field, gpu_rows):
        self.items.append((key, record, field, gpu_rows))

    def rows_of(self, key):
        return self.sets[key][1]

    def oracle_rows(self, key, oracle):
        if key not in self.cache:
            make, rows, kind = self.sets[key]
            A, B = make()
            fn = oracle.mm_minplus if kind == "minplus" else oracle.mm_f64
            t0 = time.perf_counter()
            R = fn(A, B, rows=rows)
            self.cache[key] = (R, time.perf_counter() - t0, A.shape, B.shape)
        return self.cache[key]

    def resolve(self, oracle):
        for key, rec, field, G in self.items:
            R = self.oracle_rows(key, oracle)[0]
            if self.sets[key][2] == "minplus":
                rec[field] = bool(np.array_equal(G, R))
            else:
                rec[field] = rel_fro(G, R)
        # input sets are large: release them once every error is known
        self.sets = {k: (None, v[1], v[2]) for k, v in self.sets.items()}
        self.cache.clear()


def kernels_per_call(torch, call):
    """Kernel launches of one call, counted from a CUDA graph that captures
    it on a side stream (nothing is launched).  call(stream_handle) issues
    the work; None when this runtime or the call cannot be captured."""
    import ctypes
    try:
        rt = ctypes.CDLL("libcudart.so.13")
    except OSError:
        return None
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    h = ctypes.c_void_p(side.cuda_stream)
    if rt.cudaStreamBeginCapture(h, ctypes.c_int(2)) != 0:  # relaxed capture mode
        return None
    graph = ctypes.c_void_p()
    try:
        call(int(side.cuda_stream))
    finally:
        rc = rt.cudaStreamEndCapture(h, ctypes.byref(graph))
    if rc != 0 or not graph.value:
        rt.cudaGetLastError()
        return None
    count = ctypes.c_size_t(0)
    rt.cudaGraphGetNodes(graph, None, ctypes.byref(count))
    nodes = (ctypes.c_void_p * max(1, count.value))()
    rt.cudaGraphGetNodes(graph, nodes, ctypes.byref(count))
    kernels = 0
    for i in range(count.value):
        t = ctypes.c_int(-1)
        rt.cudaGraphNodeGetType(ctypes.c_void_p(nodes[i]), ctypes.byref(t))
        kernels += 1 if t.value == 0 else 0  # cudaGraphNodeTypeKernel
    rt.cudaGraphDestroy(graph)
    return kernels


def _rows_of(torch, dC, rows):
    idx = torch.from_numpy(np.asarray(rows, np.int64)).to(dC.device)
    return dC.index_select(0, idx).cpu().numpy()


# -------------------------------------------------------------------- mmsr
def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank)

    import ctypes

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
    L = args.levels
    SR = mmsr.MM_SR_PLUS_TIMES_F64ACC
    VAR = mmsr.MM_STRASSEN_WINOGRAD
    stream = torch.cuda.current_stream()
    sp = int(stream.cuda_stream)
    book = ErrBook()

    A_h, B_h = inputs.uniform_f64(N, N, N, seed=SEED)
    rows = sample_rows(N, SAMPLE_ROWS)
    book.add_set("sq64", lambda A=A_h, B=B_h: (A, B), rows)
    dA = torch.from_numpy(A_h).cuda()
    dB = torch.from_numpy(B_h).cuda()
    dC = torch.empty((N, N), dtype=torch.float64, device="cuda")
    plan = mmsr.mm_plan_query(SR, L, N, N, N, 0)
    wbytes = int(plan.workspace_min)
    ws = torch.empty((wbytes,), dtype=torch.uint8, device="cuda")

    def call(a, b, c, s=sp):
        mmsr.mm_strassen(L, VAR, SR, N, N, N, a, b, c, ws, wbytes, s)

    for _ in range(args.warmup):
        call(dA, dB, dC)
    torch.cuda.synchronize()

    # ---------------------------------------------------------- timed region
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    sampler = ClockSampler(gpu_uuid())
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    lib.mm_trace_enable(1)
    ev[0].record(stream)
    for s in range(args.steps):
        call(dA, dB, dC)
        ev[s + 1].record(stream)
    torch.cuda.synchronize()
    lib.mm_trace_enable(0)
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    step_ms = [ev[s].elapsed_time(ev[s + 1]) for s in range(args.steps)]
    total_ms = sum(step_ms)
    if dist:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    kernels = _trace(lib, ctypes)
    per_call = kernels_per_call(torch, lambda h: call(dA, dB, dC, s=h))
    if per_call is not None:
        launches_total = per_call * args.steps
        launches_how = "%d kernels per step (counted from a CUDA graph capturing one step) x %d steps" % (
            per_call, args.steps)
    else:
        launches_total = sum(v["launches"] for v in kernels.values())
        launches_how = "trace scopes in the timed region (each covers one or more kernels)"
    head = {}
    book.add("sq64", head, "error", _rows_of(torch, dC, rows))

    ops_per_step = 2.0 * N ** 3  # classic-equivalent
    value = world * ops_per_step * args.steps / (total_ms * 1e-3) / 1e9
    # dominant kernel: the leaf GEMM over all 7^L products (one batched launch
    # per step); issued work = the 21 or 28 bf16 slice products of every leaf
    leaf = kernels.get("tc_f64acc", {"launches": 0, "ms": 0.0})
    products = 21 if plan.kernel == 7 else 28  # six- or seven-slice scheme (plan kernel id)
    leaf_issued = products * 2.0 * (N >> L) ** 3 * 7 ** L * args.steps
    peaks, peak_src = measured_peaks()
    leaf_tflops = leaf_issued / (leaf["ms"] * 1e-3) / 1e12 if leaf["ms"] else 0.0
    sustained = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
    traffic = ncu_traffic(F64ACC_SOURCES, "f64acc_gemm_strassen_L%d_n%d" % (L, N))

    # ----------------------------------------------------- end to end (host)
    # Every step uploads A and B from pinned host memory and downloads C.
    # Uploads and downloads run on two copy streams (separate copy engines)
    # with double-buffered device operands and results, so a step's uploads
    # overlap the previous step's product and its download the next one.
    pA = torch.from_numpy(A_h).pin_memory()
    pB = torch.from_numpy(B_h).pin_memory()
    pC = torch.empty((N, N), dtype=torch.float64).pin_memory()
    # three device buffer sets: an upload may run up to two products ahead,
    # which absorbs slow host-link periods (the host is shared)
    NB = 3
    dA2 = [dA] + [torch.empty_like(dA) for _ in range(NB - 1)]
    dB2 = [dB] + [torch.empty_like(dB) for _ in range(NB - 1)]
    dC2 = [dC] + [torch.empty_like(dC) for _ in range(NB - 1)]
    cs_up, cs_down = torch.cuda.Stream(), torch.cuda.Stream()
    e2e_steps = max(2, min(args.steps, 20))
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    in_ready = [torch.cuda.Event() for _ in range(NB)]
    in_free = [torch.cuda.Event() for _ in range(NB)]
    out_ready = [torch.cuda.Event() for _ in range(NB)]
    out_free = [torch.cuda.Event() for _ in range(NB)]
    # per step: the product on the compute stream, the uploads on theirs
    cev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(e2e_steps)]
    uev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(e2e_steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    evs[0].record(stream)
    cs_up.wait_event(evs[0])
    cs_down.wait_event(evs[0])
    for t in range(e2e_steps):
        j = t % NB
        with torch.cuda.stream(cs_up):
            if t >= NB:
                cs_up.wait_event(in_free[j])
            uev[t][0].record(cs_up)
            dA2[j].copy_(pA, non_blocking=True)
            dB2[j].copy_(pB, non_blocking=True)
            uev[t][1].record(cs_up)
            in_ready[j].record(cs_up)
        stream.wait_event(in_ready[j])
        if t >= NB:
            stream.wait_event(out_free[j])
        cev[t][0].record(stream)
        call(dA2[j], dB2[j], dC2[j])
        cev[t][1].record(stream)
        out_ready[j].record(stream)
        in_free[j].record(stream)
        with torch.cuda.stream(cs_down):
            cs_down.wait_event(out_ready[j])
            pC.copy_(dC2[j], non_blocking=True)
            out_free[j].record(cs_down)
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
           "h2d_bytes_per_step": int(A_h.nbytes + B_h.nbytes), "d2h_bytes_per_step": int(pC.numel() * 8),
           "steps": e2e_steps,
           "product_ms_median": float(np.median([a.elapsed_time(b) for a, b in cev])),
           "upload_ms_median": float(np.median([a.elapsed_time(b) for a, b in uev])),
           "upload_ms_max": float(max(a.elapsed_time(b) for a, b in uev)),
           "wait_between_products_ms": float(sum(cev[i][1].elapsed_time(cev[i + 1][0]) for i in range(e2e_steps - 1))),
           "overlap": "uploads and downloads on two copy streams, three device buffer sets"}
    e2e_same = bool(torch.equal(pC, dC2[(e2e_steps - 1) % NB].cpu()))
    del pA, pB, pC, dA2, dB2, dC2, ws
    torch.cuda.empty_cache()

    # ------------------------------------- the plain FP64 path beside it
    # same inputs, same stated accuracy; the DFMA leaf is bound by this
    # GPU's FP64 pipe, so one product is timed (after a small warm call)
    mmsr.mm_semiring(mmsr.MM_SR_PLUS_TIMES_F64, 256, 256, 256, dA, dB, dC, None, 0, sp)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    mmsr.mm_semiring(mmsr.MM_SR_PLUS_TIMES_F64, N, N, N, dA, dB, dC, None, 0, sp)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1)
    mhz = sm_max_mhz()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    fp64_peak = sms * 2 * 2 * mhz * 1e6 / 1e12
    plain = {"ms": plain_ms, "gops": 2.0 * N ** 3 / (plain_ms * 1e-3) / 1e9, "calls_timed": 1,
             "kernel": "dfma_leaf (64 x 64 tiles, FP64 FMA)",
             "roofline": _roof("fp64", 2.0 * N ** 3 / (plain_ms * 1e-3) / 1e12, fp64_peak, "TFLOP/s",
                               "derived: %d SMs x 2 FP64 FMA/clk x 2 FLOP x %.0f MHz" % (sms, mhz))}
    book.add("sq64", plain, "error", _rows_of(torch, dC, rows))
    del dA, dB, dC
    torch.cuda.empty_cache()

    # ----------------------------------------------------------- extras
    extras = {}
    if not args.no_extras and rank == 0:
        extras = run_extras(mmsr, lib, torch, sp, book, A_h, B_h, rows)

    # ------------------------------------- CPU phase: oracle, baseline, errors
    cpu = None
    if rank == 0 and not args.no_cpu:
        import oracle

        R, dt, _, _ = book.oracle_rows("sq64", oracle)
        if world == 1:
            cpu = {"value": 2.0 * len(rows) * N * N / dt / 1e9, "unit": "GOp/s", "cores": oracle.num_threads(),
                   "kind": "oracle",
                   "sample": "%d of %d rows (an even spread plus quadrant edges) of the n=%d product, FP64 "
                             "triple loop, %.1f s; the full product extrapolates to %.0f s"
                             % (len(rows), N, N, dt, dt * N / len(rows))}
        book.resolve(oracle)
    err = head.get("error")
    line = {
        "metric": METRIC, "value": value, "unit": "GOp/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)},
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "dtype_detail": "FP64 in/out; bf16 digit-slice products on tensor cores, exact FP32 chunks, "
                        "int64 group sums, FP64 combination and FP64 Strassen additions",
        "data": "synthetic",
        "config": bench_config(world, L),
        "error": err, "error_measure": "relative Frobenius vs FP64 oracle on %d sampled rows" % len(rows),
        "tolerance": TOL_F64, "within_tolerance": (err is not None and err <= TOL_F64),
        "vs_plain_fp64": dict(plain, speedup=plain["ms"] / (total_ms / args.steps)),
        "pct_of_dtype_peak": {
            "leaf_bf16_tensor_issued_vs_sustained": 100.0 * leaf_tflops / sustained,
            "useful_fp64_vs_fp64_peak": 100.0 * (value / world) / (fp64_peak * 1e3)},
        "peak_workspace_bytes": wbytes,
        "workspace_n2x8B": wbytes / (N * N * 8.0),
        "roofline": {"bound": "tensor", "kernel": "f64acc_gemm_kernel (all 7^L leaves in one launch)",
                     "achieved": leaf_tflops, "peak": sustained, "unit": "TFLOP/s",
                     "frac": leaf_tflops / sustained, "traffic": traffic,
                     "frac_of_burst": leaf_tflops / peaks["bf16_tflops"],
                     "peak_source": "%s: bf16 dense, sustained (the leaf runs back to back inside "
                                    "seconds-long steps); burst %.1f" % (peak_src, peaks["bf16_tflops"]),
                     "work": "%d bf16 products x 2 (n/2^L)^3 x 7^L issued FLOP per launch" % products,
                     "leaf_share_of_step": leaf["ms"] / total_ms if total_ms else None},
        "kernels": kernels,
        "gpu_launches": launches_total,
        "gpu_launches_how": launches_how,
        "clocks": clocks,
        "e2e": dict(e2e, result_matches_device_run=e2e_same),
        "cpu_baseline": cpu,
        "peaks_file": peak_src,
        "extras": extras,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# ----------------------------------------------------------------- extras
def run_extras(mmsr, lib, torch, sp, book, A_sq, B_sq, rows_sq):
    """Secondary workloads (not the headline), each with its own roofline
    record and, where the oracle can check it, its error."""
    import ctypes

    out = {}
    peaks, src = measured_peaks()
    u32_peak = _probe(lib, sp, 0, 20000) / 1e12
    u16_peak = _probe(lib, sp, 1, 20000) / 1e12
    # boolean leaf: one three-input logic op covers 32 terms (32 ANDs + 32
    # ORs) and issues on the same ALU pipe as the packed add-min, whose probe
    # issues exactly one ALU instruction per step: ALU rate x 64 ops
    lop_peak = u16_peak / 4 * 64
    mhz = sm_max_mhz()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    fp64_peak = sms * 2 * 2 * mhz * 1e6 / 1e12
    fp64_src = "derived: %d SMs x 2 FP64 FMA/clk x 2 FLOP x %.0f MHz" % (sms, mhz)
    bf16 = {"burst": peaks["bf16_tflops"], "sustained": peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])}
    bf16_src = "%s: bf16 dense burst (cuBLAS)" % src
    out["minplus_n4096_budgets"] = extras_minplus(mmsr, lib, torch, sp, ctypes, book, u32_peak, u16_peak)
    out.update(extras_fp(mmsr, lib, torch, sp, ctypes, book, fp64_peak, fp64_src, bf16, bf16_src))
    out["strassen_n16384"] = extras_strassen(mmsr, lib, torch, sp, ctypes, book, A_sq, B_sq, rows_sq, bf16,
                                             bf16_src)
    out["strassen_rect_12288x16384x8192"] = extras_strassen_rect(mmsr, lib, torch, sp, ctypes, book, bf16,
                                                                  bf16_src)
    out["batched_512"] = extras_batched(mmsr, lib, torch, sp, ctypes, bf16["burst"], u16_peak, bf16_src)
    out["batched_long_k_fp32"] = extras_batched_long_k(mmsr, torch, sp, book, bf16["burst"], bf16_src)
    out["batched_strassen_fp32"] = extras_batched_strassen(mmsr, torch, sp, book, bf16["burst"], bf16_src)
    out["closure_minplus_n4096"] = extras_closure(mmsr, torch, sp, u16_peak)
    out["orand_n4096"] = extras_orand(mmsr, lib, torch, sp, ctypes, lop_peak)
    out["probes"] = {"addmin_u32_tops": u32_peak, "addmin_u16x2_tops": u16_peak,
                     "fp64_fma_probe_tflops": _probe(lib, sp, 2, 2000) / 1e12, "fp64_peak_derived_tflops": fp64_peak,
                     "orand_peak_derived_tops": lop_peak, "fp32_fma_probe_tflops": _probe(lib, sp, 3, 20000) / 1e12,
                     # tensor-core products fed from shared memory alone (no TMA):
                     # the ceiling of the FP64-accuracy leaf's 128 x 64 x 16 shape
                     "tc_128x64x16_smem_tflops": _probe(lib, sp, 4, 4000) / 1e12,
                     "tc_128x128x16_smem_tflops": _probe(lib, sp, 5, 4000) / 1e12}
    torch.cuda.empty_cache()
    return out


def extras_minplus(mmsr, lib, torch, sp, ctypes, book, u32_peak, u16_peak):
    """(min,+) n = 4096, int32 in [0, 1000] with 10% +inf (seed 1), under the
    five budgets 0, 1, 2, 4, 8 extra n x n int32 buffers (s = 1, 2, 3, 5, 9),
    first with the packed 2 x 16-bit leaf (the inputs fit it), then with the
    exact 32-bit leaf that every other input takes."""
    from paper_1911_05328_gb300 import inputs

    n, budgets = 4096, (0, 1, 2, 4, 8)
    SR = mmsr.MM_SR_MIN_PLUS_I32
    A_h, B_h = inputs.tropical_i32(n, n, n, seed=1)
    rows = sample_rows(n)
    book.add_set("mp4096", lambda A=A_h, B=B_h: (A, B), rows, kind="minplus")
    dA, dB = torch.from_numpy(A_h).cuda(), torch.from_numpy(B_h).cuda()
    outs = [torch.empty((n, n), dtype=torch.int32, device="cuda") for _ in budgets]
    ws = torch.empty((max(budgets) * n * n * 4,), dtype=torch.uint8, device="cuda")
    flush = torch.empty((256 << 20,), dtype=torch.uint8, device="cuda")
    res = {}
    for leaf_name, packed, peak in (("minplus16_leaf", 1, u16_peak), ("minplus_leaf", 0, u32_peak)):
        mmsr.mm_set_option(mmsr.MM_OPT_MINPLUS_PACKED, packed)
        steps = 10 if packed else 4
        per = [0.0] * len(budgets)
        for b, C in zip(budgets, outs):  # warm
            mmsr.mm_semiring(SR, n, n, n, dA, dB, C, ws, b * n * n * 4, sp)
        torch.cuda.synchronize()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(budgets) + 1)] for _ in range(steps)]
        lib.mm_trace_enable(1)
        for s in range(steps):
            flush.zero_()  # evict L2 between steps (not timed)
            evs[s][0].record()
            for i, (b, C) in enumerate(zip(budgets, outs)):
                mmsr.mm_semiring(SR, n, n, n, dA, dB, C, ws, b * n * n * 4, sp)
                evs[s][i + 1].record()
        torch.cuda.synchronize()
        lib.mm_trace_enable(0)
        kern = _trace(lib, ctypes)
        for s in range(steps):
            for i in range(len(budgets)):
                per[i] += evs[s][i].elapsed_time(evs[s][i + 1]) / steps
        k = kern.get(leaf_name, {"launches": 1, "ms": 0.0})
        leaf_ms = k["ms"] / (steps * len(budgets))
        ach = 2.0 * n ** 3 / (leaf_ms * 1e-3) / 1e12 if leaf_ms else 0.0
        step_ms = sum(per)
        rec = {"ms_per_step_5_calls": step_ms, "gops": 5 * 2.0 * n ** 3 / (step_ms * 1e-3) / 1e9,
               "per_budget": [{"budget_buffers": b, "split_k": mmsr.mm_plan_query(SR, -1, n, n, n, b * n * n * 4).split_k,
                               "workspace_used_bytes": int(mmsr.mm_plan_query(SR, -1, n, n, n, b * n * n * 4).workspace_used),
                               "ms": per[i], "gops": 2.0 * n ** 3 / (per[i] * 1e-3) / 1e9}
                              for i, b in enumerate(budgets)],
               "budgets_agree": all(bool(torch.equal(outs[0], C)) for C in outs[1:]),
               "kernels": kern,
               "roofline": dict(_roof("alu", ach, peak, "TOp/s",
                                      "measured: mm_probe_peak fused add-min %s, all SMs"
                                      % ("packed 2 x u16 (4 ops/lane-instr)" if packed else "u32 (2 ops/lane-instr)")),
                                kernel=leaf_name,
                                traffic=ncu_traffic(["minplus.cu", "minplus_tile.cuh"], leaf_name + "_n4096"))}
        book.add("mp4096", rec, "bit_exact_sampled_rows", _rows_of(torch, outs[-1], rows))
        res["packed_u16x2" if packed else "u32"] = rec
    mmsr.mm_set_option(mmsr.MM_OPT_MINPLUS_PACKED, 1)
    del dA, dB, outs, ws, flush
    torch.cuda.empty_cache()
    return res


def extras_fp(mmsr, lib, torch, sp, ctypes, book, fp64_peak, fp64_src, bf16, bf16_src):
    """FP64 classic n = 256 (budget 0); FP32 mode (bf16x3) and FP64-accuracy
    mode at n = 8192 beside the plain FP64 path at the same size."""
    from paper_1911_05328_gb300 import inputs

    out = {}
    A, B = inputs.uniform_f64(256, 256, 256, seed=0)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.empty((256, 256), dtype=torch.float64, device="cuda")
    ms = _time_call(torch, lambda: mmsr.mm_semiring(mmsr.MM_SR_PLUS_TIMES_F64, 256, 256, 256, dA, dB, dC, None, 0,
                                                    sp), 50)
    book.add_set("n256", lambda A=A, B=B: (A, B), np.arange(256))
    out["fp64_n256_budget0"] = {"ms": ms, "gops": 2 * 256 ** 3 / (ms * 1e-3) / 1e9,
                                "roofline": _roof("fp64", 2 * 256 ** 3 / (ms * 1e-3) / 1e12, fp64_peak,
                                                  "TFLOP/s", fp64_src)}
    book.add("n256", out["fp64_n256_budget0"], "error", dC.cpu().numpy())
    # the same product in the stream-K form (Fig. tar-mm) with the budget of
    # its per-CTA partial tiles (forced: the planner keeps the 8 x 8 tiles
    # here, which balance without slots)
    mmsr.mm_set_option(mmsr.MM_OPT_F64_STREAMK, 2)
    for b in (1 << 20, 1 << 22, 1 << 24):
        p = mmsr.mm_plan_query(mmsr.MM_SR_PLUS_TIMES_F64, -1, 256, 256, 256, b)
        if p.kernel == 6:
            w = int(p.workspace_used)
            ws = torch.empty((w,), dtype=torch.uint8, device="cuda")
            ms = _time_call(torch, lambda: mmsr.mm_semiring(mmsr.MM_SR_PLUS_TIMES_F64, 256, 256, 256, dA, dB, dC,
                                                            ws, w, sp), 50)
            out["fp64_n256_streamk"] = {"ms": ms, "gops": 2 * 256 ** 3 / (ms * 1e-3) / 1e9, "workspace_bytes": w,
                                        "roofline": _roof("fp64", 2 * 256 ** 3 / (ms * 1e-3) / 1e12, fp64_peak,
                                                          "TFLOP/s", fp64_src)}
            book.add("n256", out["fp64_n256_streamk"], "error", dC.cpu().numpy())
            mmsr.mm_set_option(mmsr.MM_OPT_F64_STREAMK, 1)
            out["fp64_n256_streamk"]["planner_kernel_at_this_budget"] = int(
                mmsr.mm_plan_query(mmsr.MM_SR_PLUS_TIMES_F64, -1, 256, 256, 256, w).kernel)
            del ws
            break
    mmsr.mm_set_option(mmsr.MM_OPT_F64_STREAMK, 1)
    n = 8192
    rows = sample_rows(n)
    A, B = inputs.uniform_f64(n, n, n, seed=2)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    del A, B
    dC = torch.empty((n, n), dtype=torch.float64, device="cuda")
    ms = _time_call(torch, lambda: mmsr.mm_semiring(mmsr.MM_SR_PLUS_TIMES_F64, n, n, n, dA, dB, dC, None, 0, sp), 1)
    out["fp64_dfma_n8192"] = {"ms": ms, "gops": 2 * n ** 3 / (ms * 1e-3) / 1e9,
                              "roofline": _roof("fp64", 2 * n ** 3 / (ms * 1e-3) / 1e12, fp64_peak,
                                                "TFLOP/s", fp64_src)}
    del dA, dB, dC
    # FP32 mode n=8192, normal(0,1), seed 2: bf16x3 split products on tcgen05
    A, B = inputs.normal_f32(n, n, n, seed=2)
    book.add_set("n8192_f32", lambda A=A, B=B: (A, B), rows)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.empty((n, n), dtype=torch.float32, device="cuda")
    sr = mmsr.MM_SR_PLUS_TIMES_F32
    wmin = int(mmsr.mm_plan_query(sr, -1, n, n, n, 0).workspace_min)
    ws = torch.empty((wmin,), dtype=torch.uint8, device="cuda")
    lib.mm_trace_enable(1)
    ms = _time_call(torch, lambda: mmsr.mm_semiring(sr, n, n, n, dA, dB, dC, ws, wmin, sp), 10)
    lib.mm_trace_enable(0)
    kern = _trace(lib, ctypes)
    g = kern.get("tc_bf16x3", {"launches": 1, "ms": 0.0})
    gemm_ms = g["ms"] / max(g["launches"], 1)
    issued = 3 * 2.0 * n ** 3 / (gemm_ms * 1e-3) / 1e12 if gemm_ms else 0.0
    out["fp32_bf16x3_n8192"] = {
        "ms": ms, "gops_useful": 2 * n ** 3 / (ms * 1e-3) / 1e9, "gemm_ms": gemm_ms, "kernels": kern,
        "tensor_tflops_issued": issued,
        "roofline": _roof("tensor", issued, bf16["burst"], "TFLOP/s", bf16_src),
        "workspace_bytes": wmin, "speedup_vs_fp64_dfma": out["fp64_dfma_n8192"]["ms"] / ms, "tolerance": 1e-5}
    book.add("n8192_f32", out["fp32_bf16x3_n8192"], "error", _rows_of(torch, dC, rows))
    del dA, dB, dC, ws
    torch.cuda.empty_cache()
    # k-parallel forms where the classic grid quantises: 2048 x n x 8192
    # (normal inputs, seed 2) in 128 x 256 tiles, n = 2560 (160 tiles, 1.05
    # waves on 152 SMs: the planner takes stream-K) and n = 4096 (256 tiles,
    # 1.68 waves: the classic grid).  Each shape: the classic grid (stream-K
    # off, no budget), the budgeted split-K at the stream-K budget (stream-K
    # off), stream-K over every tile's units (option 2), whole waves first
    # and stream-K over the rest (option 3), and the planner's own choice.
    m, kk = 2048, 8192
    sr = mmsr.MM_SR_PLUS_TIMES_F32
    for nn in (2560, 4096):
        A, B = inputs.normal_f32(m, kk, nn, seed=2)
        key = "f32_kpar_%d" % nn
        book.add_set(key, lambda A=A, B=B: (A, B), sample_rows(m))
        dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        dC = torch.empty((m, nn), dtype=torch.float32, device="cuda")
        base = int(mmsr.mm_plan_query(sr, -1, m, nn, kk, 0).workspace_min)
        mmsr.mm_set_option(mmsr.MM_OPT_F32_STREAMK, 2)
        skb = None
        for extra in (1 << 26, 1 << 28):
            p = mmsr.mm_plan_query(sr, -1, m, nn, kk, base + extra)
            if p.kernel == 5:
                skb = int(p.workspace_used)
                break
        rec = {"tiles": (m // 128) * (nn // 256)}
        for name, opt, budget in (("classic", 0, base), ("split_k", 0, skb), ("streamk", 2, skb),
                                  ("whole_waves_then_streamk", 3, skb), ("planner", 1, skb)):
            if budget is None:
                continue
            mmsr.mm_set_option(mmsr.MM_OPT_F32_STREAMK, opt)
            p = mmsr.mm_plan_query(sr, -1, m, nn, kk, budget)
            ws = torch.empty((budget,), dtype=torch.uint8, device="cuda")
            ms = _time_call(torch, lambda: mmsr.mm_semiring(sr, m, nn, kk, dA, dB, dC, ws, budget, sp), 10)
            rec[name] = {"ms": ms, "gops": 2.0 * m * nn * kk / (ms * 1e-3) / 1e9, "kernel": int(p.kernel),
                         "split_k": int(p.split_k), "workspace_bytes": budget}
            book.add(key, rec[name], "error", _rows_of(torch, dC, sample_rows(m)))
            del ws
        mmsr.mm_set_option(mmsr.MM_OPT_F32_STREAMK, 1)
        out["fp32_2048x%dx8192_k_parallel" % nn] = rec
        del dA, dB, dC
        torch.cuda.empty_cache()
    # FP64-accuracy mode at n = 8192 (uniform[-1,1], seed 3)
    A, B = inputs.uniform_f64(n, n, n, seed=3)
    book.add_set("n8192_f64", lambda A=A, B=B: (A, B), rows)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.empty((n, n), dtype=torch.float64, device="cuda")
    sr = mmsr.MM_SR_PLUS_TIMES_F64ACC
    pl = mmsr.mm_plan_query(sr, -1, n, n, n, 0)
    wmin = int(pl.workspace_min)
    products = 21 if pl.kernel == 7 else 28
    ws = torch.empty((wmin,), dtype=torch.uint8, device="cuda")
    lib.mm_trace_enable(1)
    ms = _time_call(torch, lambda: mmsr.mm_semiring(sr, n, n, n, dA, dB, dC, ws, wmin, sp), 4)
    lib.mm_trace_enable(0)
    kern = _trace(lib, ctypes)
    g = kern.get("tc_f64acc", {"launches": 1, "ms": 0.0})
    gemm_ms = g["ms"] / max(g["launches"], 1)
    issued = products * 2.0 * n ** 3 / (gemm_ms * 1e-3) / 1e12 if gemm_ms else 0.0
    out["fp64acc_n8192"] = {
        "ms": ms, "gflops_useful": 2 * n ** 3 / (ms * 1e-3) / 1e9, "gemm_ms": gemm_ms, "kernels": kern,
        "tensor_tflops_issued": issued, "slice_products": products,
        "roofline": dict(_roof("tensor", issued, bf16["burst"], "TFLOP/s", bf16_src),
                         frac_of_sustained=issued / bf16["sustained"]),
        "workspace_bytes": wmin, "speedup_vs_fp64_dfma": out["fp64_dfma_n8192"]["ms"] / ms, "tolerance": 1e-12}
    book.add("n8192_f64", out["fp64acc_n8192"], "error", _rows_of(torch, dC, rows))
    del dA, dB, dC, ws
    torch.cuda.empty_cache()
    return out


def _strassen_levels(mmsr, lib, torch, sp, ctypes, book, key, sr, m, n, k, dA, dB, dC, rows, bf16, bf16_src,
                     levels=range(0, 5), reps=3):
    """Time mm_strassen (Winograd) at each level on one product; record time,
    classic-equivalent GOp/s, workspace, the leaf launch's tensor roofline,
    the kernel split and the sampled-row error."""
    leaf_name = "tc_bf16x3" if sr == mmsr.MM_SR_PLUS_TIMES_F32 else "tc_f64acc"
    eb = 4 if sr == mmsr.MM_SR_PLUS_TIMES_F32 else 8
    res = {}
    for L in levels:
        p = mmsr.mm_plan_query(sr, L, m, n, k, 0)
        products = 3 if sr == mmsr.MM_SR_PLUS_TIMES_F32 else (21 if p.kernel == 7 else 28)
        ws = torch.empty((max(int(p.workspace_min), 16),), dtype=torch.uint8, device="cuda")
        fn = lambda: mmsr.mm_strassen(L, mmsr.MM_STRASSEN_WINOGRAD, sr, m, n, k, dA, dB, dC, ws,
                                      int(p.workspace_min), sp)
        fn()
        torch.cuda.synchronize()
        lib.mm_trace_enable(1)
        ms = _time_call(torch, fn, reps)
        lib.mm_trace_enable(0)
        kern = _trace(lib, ctypes)
        calls = reps + 1  # _time_call's untimed call is traced too
        split = {nm: v["ms"] / calls for nm, v in kern.items()}
        rec = {"ms": ms, "gops_classic_equiv": 2.0 * m * n * k / (ms * 1e-3) / 1e9,
               "workspace_bytes": int(p.workspace_min),
               "workspace_over_mn_x_elem": p.workspace_min / (float(max(m, n)) * max(m, n) * eb),
               "kernel_ms": split, "launches_per_call": {nm: v["launches"] / calls for nm, v in kern.items()}}
        leaf_ms = split.get(leaf_name, 0.0)
        if leaf_ms > 0:
            issued = products * 2.0 * (m >> L) * (n >> L) * (k >> L) * 7 ** L / (leaf_ms * 1e-3) / 1e12
            rec["leaf_roofline"] = dict(_roof("tensor", issued, bf16["burst"], "TFLOP/s", bf16_src),
                                        frac_of_sustained=issued / bf16["sustained"], kernel=leaf_name,
                                        products_per_kstep=products)
            rec["leaf_share_of_time"] = leaf_ms / ms
        book.add(key, rec, "error", _rows_of(torch, dC, rows))
        res["L%d" % L] = rec
        del ws
        torch.cuda.empty_cache()
    return res


def extras_strassen(mmsr, lib, torch, sp, ctypes, book, A_sq, B_sq, rows, bf16, bf16_src):
    """Strassen-Winograd at n = 16384 (uniform[-1,1], seed 3): FP64-accuracy
    mode and FP32 mode (the float32 cast of the same inputs), L = 0..4, with
    the error of every level; then the zero-temporary TAR-Strassen level and
    the STAR-Strassen-1 mixed plans in FP32 mode."""
    n = N
    res = {}
    dA64, dB64 = torch.from_numpy(A_sq).cuda(), torch.from_numpy(B_sq).cuda()
    dC64 = torch.empty((n, n), dtype=torch.float64, device="cuda")
    res["fp64acc"] = _strassen_levels(mmsr, lib, torch, sp, ctypes, book, "sq64", mmsr.MM_SR_PLUS_TIMES_F64ACC,
                                      n, n, n, dA64, dB64, dC64, rows, bf16, bf16_src, reps=2)
    # TAR-Strassen in FP64-accuracy mode: one Winograd level whose seven
    # digit-slice products add straight into C's quadrants (no post pass)
    fa = mmsr.MM_SR_PLUS_TIMES_F64ACC
    p = mmsr.mm_strassen_tar_query(1, fa, n, n, n)
    ws = torch.empty((int(p.workspace_min),), dtype=torch.uint8, device="cuda")
    fn = lambda: mmsr.mm_strassen_tar(1, mmsr.MM_STRASSEN_WINOGRAD, fa, n, n, n, dA64, dB64, dC64, ws,
                                      int(p.workspace_min), sp)
    ms = _time_call(torch, fn, 2)
    res["fp64acc_tar_L1"] = {"ms": ms, "gops_classic_equiv": 2.0 * n ** 3 / (ms * 1e-3) / 1e9,
                             "workspace_bytes": int(p.workspace_min),
                             "workspace_over_mn_x_elem": p.workspace_min / (n * n * 8.0)}
    book.add("sq64", res["fp64acc_tar_L1"], "error", _rows_of(torch, dC64, rows))
    del ws, dC64
    torch.cuda.empty_cache()
    book.add_set("sq32", lambda A=A_sq, B=B_sq: (A.astype(np.float32), B.astype(np.float32)), rows)
    dA, dB = dA64.float(), dB64.float()
    del dA64, dB64
    dC = torch.empty((n, n), dtype=torch.float32, device="cuda")
    sr = mmsr.MM_SR_PLUS_TIMES_F32
    res["fp32"] = _strassen_levels(mmsr, lib, torch, sp, ctypes, book, "sq32", sr, n, n, n, dA, dB, dC, rows,
                                   bf16, bf16_src)
    # TAR-Strassen: leaf products added into C's blocks by the leaf epilogue
    # in conflict-free waves (no product temporaries): one Winograd level,
    # two levels of the paper's formulas
    for key, L, var in (("fp32_tar_L1", 1, mmsr.MM_STRASSEN_WINOGRAD), ("fp32_tar_L2_paper", 2, mmsr.MM_STRASSEN_PAPER)):
        p = mmsr.mm_strassen_tar_query(L, sr, n, n, n)
        ws = torch.empty((int(p.workspace_min),), dtype=torch.uint8, device="cuda")
        fn = lambda: mmsr.mm_strassen_tar(L, var, sr, n, n, n, dA, dB, dC, ws, int(p.workspace_min), sp)
        ms = _time_call(torch, fn, 3)
        res[key] = {"ms": ms, "gops_classic_equiv": 2.0 * n ** 3 / (ms * 1e-3) / 1e9,
                    "workspace_bytes": int(p.workspace_min), "workspace_n2x4B": p.workspace_min / (n * n * 4.0),
                    "waves": mmsr.mm_strassen_tar_waves(L, var)[0]}
        book.add("sq32", res[key], "error", _rows_of(torch, dC, rows))
        del ws
        torch.cuda.empty_cache()
    # one level with the operand sums formed in the leaf's staging against the
    # materialised operand passes, for the paper's formulas and Winograd's
    for vname, var in (("paper", mmsr.MM_STRASSEN_PAPER), ("winograd", mmsr.MM_STRASSEN_WINOGRAD)):
        for fused in (0, 1):
            mmsr.mm_set_option(mmsr.MM_OPT_STRASSEN_FUSED, fused)
            p = mmsr.mm_plan_query(sr, 1, n, n, n, 0)
            ws = torch.empty((int(p.workspace_min),), dtype=torch.uint8, device="cuda")
            fn = lambda: mmsr.mm_strassen(1, var, sr, n, n, n, dA, dB, dC, ws, int(p.workspace_min), sp)
            lib.mm_trace_enable(1)
            ms = _time_call(torch, fn, 3)
            lib.mm_trace_enable(0)
            kern = {nm: v["ms"] / 4 for nm, v in _trace(lib, ctypes).items()}
            rec = {"ms": ms, "gops_classic_equiv": 2.0 * n ** 3 / (ms * 1e-3) / 1e9,
                   "workspace_bytes": int(p.workspace_min), "workspace_n2x4B": p.workspace_min / (n * n * 4.0),
                   "kernel_ms": kern}
            book.add("sq32", rec, "error", _rows_of(torch, dC, rows))
            res["fp32_L1_%s_%s" % (vname, "fused_staging" if fused else "materialised")] = rec
            del ws
            torch.cuda.empty_cache()
    mmsr.mm_set_option(mmsr.MM_OPT_STRASSEN_FUSED, 0)
    # STAR-Strassen-1 mixed plans: c classic in-place levels over L Strassen
    # levels; the workspace of one block product only
    for c, L in ((1, 1), (1, 2), (2, 1), (2, 2)):
        p = mmsr.mm_star_strassen_query(c, L, sr, n, n, n)
        ws = torch.empty((int(p.workspace_min),), dtype=torch.uint8, device="cuda")
        fn = lambda: mmsr.mm_star_strassen(c, L, mmsr.MM_STRASSEN_WINOGRAD, sr, n, n, n, dA, dB, dC, ws,
                                           int(p.workspace_min), sp)
        ms = _time_call(torch, fn, 3)
        rec = {"ms": ms, "gops_classic_equiv": 2.0 * n ** 3 / (ms * 1e-3) / 1e9,
               "workspace_bytes": int(p.workspace_min), "workspace_n2x4B": p.workspace_min / (n * n * 4.0)}
        book.add("sq32", rec, "error", _rows_of(torch, dC, rows))
        res["fp32_star_c%d_L%d" % (c, L)] = rec
        del ws
        torch.cuda.empty_cache()
    del dA, dB, dC
    torch.cuda.empty_cache()
    return res


def extras_strassen_rect(mmsr, lib, torch, sp, ctypes, book, bf16, bf16_src):
    """The rectangular product m = 12288, k = 16384, n = 8192 (uniform[-1,1],
    seed 3), Strassen-Winograd L = 0..4 in FP64-accuracy and FP32 modes."""
    from paper_1911_05328_gb300 import inputs

    m, k, n = 12288, 16384, 8192
    A, B = inputs.uniform_f64(m, k, n, seed=3)
    rows = sample_rows(m)
    book.add_set("rect64", lambda A=A, B=B: (A, B), rows)
    book.add_set("rect32", lambda A=A, B=B: (A.astype(np.float32), B.astype(np.float32)), rows)
    res = {}
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.empty((m, n), dtype=torch.float64, device="cuda")
    res["fp64acc"] = _strassen_levels(mmsr, lib, torch, sp, ctypes, book, "rect64", mmsr.MM_SR_PLUS_TIMES_F64ACC,
                                      m, n, k, dA, dB, dC, rows, bf16, bf16_src, reps=2)
    dA, dB = dA.float(), dB.float()
    dC = torch.empty((m, n), dtype=torch.float32, device="cuda")
    res["fp32"] = _strassen_levels(mmsr, lib, torch, sp, ctypes, book, "rect32", mmsr.MM_SR_PLUS_TIMES_F32,
                                   m, n, k, dA, dB, dC, rows, bf16, bf16_src)
    del dA, dB, dC
    torch.cuda.empty_cache()
    return res


def extras_batched(mmsr, lib, torch, sp, ctypes, bf16_peak, u16_peak, bf16_src):
    """512 problems (m, n, k log-uniform in [64, 2048], 70% FP32 (+,x) with
    normal(0,1) entries, 30% (min,+) with integers in [0, 1000], seed 4) in
    one capturable call, captured once in a CUDA graph and replayed."""
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
    split = {nm: v["ms"] / 3 for nm, v in _trace(lib, ctypes).items()}
    # ideal time: every FP32 product's three bf16 split products at the tensor
    # peak plus every (min,+) product at the packed add-min peak
    ideal_ms = (3 * ops_fp32 / (bf16_peak * 1e12) + (ops - ops_fp32) / (u16_peak * 1e12)) * 1e3
    res = {"ms": ms, "gops": ops / (ms * 1e-3) / 1e9, "ops": ops, "fp32_share_of_ops": ops_fp32 / ops,
           "roofline": _roof("tensor (FP32 tiles) + alu ((min,+) tiles)", ops / (ms * 1e-3) / 1e12,
                             ops / (ideal_ms * 1e-3) / 1e12, "TOp/s",
                             bf16_src + "; measured packed add-min probe"),
           "kernel_ms_eager": split, "workspace_bytes": int(need),
           "error": "bit-exact (min,+), <= 1e-5 FP32, per problem (tests)"}
    del dA, dB, dC, ws, g
    torch.cuda.empty_cache()
    return res


def extras_batched_long_k(mmsr, torch, sp, book, bf16_peak, bf16_src):
    """A batch whose few long-k FP32 products would end it alone: 8 products
    of 256 x 384 x 32768 among 56 with m, n, k log-uniform in [64, 1024]
    (normal(0,1), seed 11), FP32 mode.  Tiles unsliced (split_k = 1), the
    library's slicing rule (split_k = 0) and the autotuner's per-k-bucket
    choice, each captured in a graph and replayed."""
    from paper_1911_05328_gb300 import autotune, inputs

    probs = inputs.batched_long_k_problems(seed=11)
    dA = [torch.from_numpy(p.A).cuda() for p in probs]
    dB = [torch.from_numpy(p.B).cuda() for p in probs]
    dC = [torch.empty((p.m, p.n), dtype=torch.float32, device="cuda") for p in probs]
    base = [(p.semiring, p.m, p.n, p.k, a, b, c) for p, a, b, c in zip(probs, dA, dB, dC)]
    ops = sum(2.0 * p.m * p.n * p.k for p in probs)
    rows0 = sample_rows(probs[0].m, 32)
    book.add_set("batched_long_k_0", lambda p=probs[0]: (p.A, p.B), rows0)
    need = max(mmsr.mm_batched_query(autotune.apply_splits(base, [h] * len(base))) for h in (0, 1, 16))
    ws = torch.empty((need,), dtype=torch.uint8, device="cuda")
    tuned = autotune.tune_batched(base, ws, need, cache={}, persist=False)
    out = {"problems": len(probs), "ops": ops}
    for name, splits in (("unsliced", [1] * len(base)), ("library_rule", [0] * len(base)),
                         ("autotuned", tuned["splits"])):
        table = autotune.apply_splits(base, splits)
        mmsr.mm_batched(table, ws, need, stream=sp)
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            mmsr.mm_batched(table, ws, need, stream=torch.cuda.current_stream())
        ms = _time_call(torch, g.replay, 10)
        out[name] = {"ms": ms, "gops": ops / (ms * 1e-3) / 1e9,
                     "roofline": _roof("tensor", 3 * ops / (ms * 1e-3) / 1e12, bf16_peak, "TFLOP/s", bf16_src),
                     "workspace_bytes": int(mmsr.mm_batched_query(table))}
        # sampled rows of the first long-k product against the oracle
        book.add("batched_long_k_0", out[name], "error_long_k_product", _rows_of(torch, dC[0], rows0))
        del g
    out["autotuned"]["buckets"] = tuned["buckets"]
    del dA, dB, dC, ws
    torch.cuda.empty_cache()
    return out


def extras_batched_strassen(mmsr, torch, sp, book, bf16_peak, bf16_src):
    """FP32 batch with large products: 16 of 2048^3 among 48 with m, n, k
    log-uniform in [64, 512] (normal(0,1), seed 12).  The large products
    classic (levels = 0), with one Strassen-Winograd level inside the batch
    (levels = 1), and the autotuner's choice; each captured in a graph."""
    from paper_1911_05328_gb300 import autotune, inputs

    probs = inputs.batched_long_k_problems(seed=12, long_count=16, long_shape=(2048, 2048, 2048), short_count=48,
                                           lo=64, hi=512)
    dA = [torch.from_numpy(p.A).cuda() for p in probs]
    dB = [torch.from_numpy(p.B).cuda() for p in probs]
    dC = [torch.empty((p.m, p.n), dtype=torch.float32, device="cuda") for p in probs]
    base = [(p.semiring, p.m, p.n, p.k, a, b, c) for p, a, b, c in zip(probs, dA, dB, dC)]
    ops = sum(2.0 * p.m * p.n * p.k for p in probs)
    rows0 = sample_rows(probs[0].m, 32)
    book.add_set("batched_strassen_0", lambda p=probs[0]: (p.A, p.B), rows0)
    big = autotune.strassen_candidates_in_batch(base)
    lv1 = [1 if i in big else 0 for i in range(len(base))]
    need = max(mmsr.mm_batched_query(autotune.apply_splits(base, [h] * len(base), lv))
               for h in (0, 16) for lv in ([0] * len(base), lv1))
    ws = torch.empty((need,), dtype=torch.uint8, device="cuda")
    tuned = autotune.tune_batched(base, ws, need, cache={}, persist=False)
    out = {"problems": len(probs), "ops": ops, "large_products": len(big)}
    for name, splits, levels in (("classic", [0] * len(base), [0] * len(base)), ("strassen_L1", [0] * len(base), lv1),
                                 ("autotuned", tuned["splits"], tuned["levels"])):
        table = autotune.apply_splits(base, splits, levels)
        mmsr.mm_batched(table, ws, need, stream=sp)
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            mmsr.mm_batched(table, ws, need, stream=torch.cuda.current_stream())
        ms = _time_call(torch, g.replay, 10)
        out[name] = {"ms": ms, "gops_classic_equiv": ops / (ms * 1e-3) / 1e9,
                     "workspace_bytes": int(mmsr.mm_batched_query(table))}
        book.add("batched_strassen_0", out[name], "error_first_large_product", _rows_of(torch, dC[0], rows0))
        del g
    out["autotuned"]["levels_of_large"] = sorted({tuned["levels"][i] for i in big})
    del dA, dB, dC, ws
    torch.cuda.empty_cache()
    return out


def extras_orand(mmsr, lib, torch, sp, ctypes, lop_peak):
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
    split = {nm: v["ms"] / 5 for nm, v in _trace(lib, ctypes).items()}
    res = {"ms": ms, "gops": 2.0 * n ** 3 / (ms * 1e-3) / 1e9, "workspace_bytes": w, "kernel_ms": split,
           "roofline": _roof("alu", 2.0 * n ** 3 / (ms * 1e-3) / 1e12, lop_peak, "TOp/s",
                             "derived: measured ALU-pipe rate (packed add-min probe / 4) x 64 ops per "
                             "32-bit and-or"),
           "error": "bit-exact vs oracle (tests)"}
    del dA, dB, dC, ws
    torch.cuda.empty_cache()
    return res


def extras_closure(mmsr, torch, sp, u16_peak):
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


if __name__ == "__main__":
    sys.exit(main())
