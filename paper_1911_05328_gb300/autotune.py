"""Per-shape autotuner for the budget / split-K / Strassen-depth choices.

The C ABI takes a workspace *budget*; the paper's point (Sections 3-4) is that
more temporary space buys a shorter critical path, but on a GPU a larger
split factor is not always faster (extra partial traffic, smaller tiles per
CTA).  The tuner times the candidate plans a budget allows and remembers the
fastest per shape bucket:

* ``mm_semiring``: split factors s = 1 .. s_max, requested by handing the
  library a smaller budget (``budget_for_split``);
* ``mm_strassen``: Strassen depths L = 0 .. 4 whose workspace fits the budget
  and whose shape divides by 2^L;
* ``mm_star_strassen``: mixed plans (Theorem star-strassen-1) of c classic
  in-place levels over L Strassen levels, c + L <= 4 -- at a small budget a
  deep Strassen plan fits only below a few classic levels;
* ``mm_batched``: the k-slices of FP32 tiles (``split_k`` of each problem),
  one choice per power-of-two k bucket, found by coordinate descent over the
  buckets (longest k first) with the whole batch timed for each candidate;
  then one Strassen-Winograd level (``levels``) for the large FP32 problems
  (every dimension >= 1024 and even), kept if the batch gets faster.

Choices are cached in JSON (``MMSR_TUNE_CACHE``, default
``~/.cache/mmsr_tune.json``) keyed by semiring, power-of-two shape bucket and
budget bucket.  Timing uses CUDA events by default; any callable
``timer(fn) -> ms`` can be injected (the CPU tests do).
"""
from __future__ import annotations

import json
import math
import os
import threading

from . import mmsr

_ACC_BYTES = {mmsr.MM_SR_PLUS_TIMES_F64: 8, mmsr.MM_SR_PLUS_TIMES_F32: 4, mmsr.MM_SR_PLUS_TIMES_F64ACC: 8,
              mmsr.MM_SR_MIN_PLUS_I32: 4, mmsr.MM_SR_OR_AND_U8: 1}
_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("MMSR_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "mmsr_tune.json"))


def _bucket(x: int) -> int:
    return 0 if x <= 0 else 1 << int(math.ceil(math.log2(x)))


def key(op: str, semiring: int, m: int, n: int, k: int, budget: int) -> str:
    return "%s/%d/%dx%dx%d/%d" % (op, semiring, _bucket(m), _bucket(n), _bucket(k), _bucket(budget))


def load_cache(path=None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path=None) -> None:
    path = path or cache_path()
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = path + ".%d.tmp" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def budget_for_split(semiring: int, m: int, n: int, k: int, s: int) -> int:
    """Smallest budget whose plan uses split factor s (for s the planner can reach)."""
    base = int(mmsr.mm_plan_query(semiring, -1, m, n, k, 0).workspace_min)
    return base + (s - 1) * m * n * _ACC_BYTES[semiring]


def split_candidates(semiring: int, m: int, n: int, k: int, budget: int):
    """Distinct split factors the budget allows, as (s, budget_to_pass)."""
    smax = mmsr.mm_plan_query(semiring, -1, m, n, k, budget).split_k
    seen, out = set(), []
    for s in sorted({1, 2, 3, 4, 5, 8, 9, 16, smax}):
        if s > smax:
            continue
        b = budget_for_split(semiring, m, n, k, s)
        got = mmsr.mm_plan_query(semiring, -1, m, n, k, b).split_k
        if got not in seen and b <= budget:
            seen.add(got)
            out.append((got, b))
    return out


def strassen_candidates(semiring: int, m: int, n: int, k: int, budget: int):
    """Strassen depths whose workspace fits the budget, as (L, workspace)."""
    out = []
    for L in range(0, 5):
        mask = (1 << L) - 1
        if (m & mask) or (n & mask) or (k & mask):
            break
        p = mmsr.mm_plan_query(semiring, L if L else -1, m, n, k, budget, check=False)
        if p.status != mmsr.MM_OK:
            continue
        if int(p.workspace_min) <= budget:
            out.append((L, int(p.workspace_min)))
    return out


def star_candidates(semiring: int, m: int, n: int, k: int, budget: int, max_depth: int = 4):
    """Mixed plans (c classic levels, L Strassen levels) whose workspace fits
    the budget, as (c, L, workspace); c = L = 0 is the classic product.  Of
    plans with the same total depth c + L only the one with the fewest classic
    levels that fits is kept (it does the least arithmetic)."""
    out = []
    for depth in range(0, max_depth + 1):
        mask = (1 << depth) - 1
        if (m & mask) or (n & mask) or (k & mask):
            break
        for c in range(0, depth + 1):
            L = depth - c
            if L == 0 and c > 0:
                continue  # classic levels alone are the classic product
            p = mmsr.mm_star_strassen_query(c, L, semiring, m, n, k, budget, check=False)
            if p.status == mmsr.MM_OK and int(p.workspace_min) <= budget:
                out.append((c, L, int(p.workspace_min)))
                break
    return out


def tune_star_strassen(semiring, m, n, k, A, B, C, workspace, budget, variant=mmsr.MM_STRASSEN_WINOGRAD,
                       timer=None, cache=None, persist=True):
    """Time every mixed plan the budget allows; returns {"classic", "levels",
    "workspace", "ms"}."""
    timer = timer or cuda_timer
    kk = key("star%d" % variant, semiring, m, n, k, budget)
    with _lock:
        c = load_cache() if cache is None else cache
        if kk in c:
            return c[kk]
    best = None
    for cl, L, w in star_candidates(semiring, m, n, k, budget):
        ms = timer(lambda: mmsr.mm_star_strassen(cl, L, variant, semiring, m, n, k, A, B, C, workspace, w))
        if best is None or ms < best["ms"]:
            best = {"classic": cl, "levels": L, "workspace": w, "ms": ms}
    with _lock:
        c[kk] = best
        if persist and cache is None:
            save_cache(c)
    return best


def cuda_timer(fn, reps=3):
    import torch

    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def tune_semiring(semiring, m, n, k, A, B, C, workspace, budget, timer=cuda_timer, cache=None, persist=True):
    """Time every split factor the budget allows; returns {"split_k", "budget", "ms"}."""
    kk = key("semiring", semiring, m, n, k, budget)
    with _lock:
        c = load_cache() if cache is None else cache
        if kk in c:
            return c[kk]
    best = None
    for s, b in split_candidates(semiring, m, n, k, budget):
        ms = timer(lambda: mmsr.mm_semiring(semiring, m, n, k, A, B, C, workspace, b))
        if best is None or ms < best["ms"]:
            best = {"split_k": s, "budget": b, "ms": ms}
    with _lock:
        c[kk] = best
        if persist and cache is None:
            save_cache(c)
    return best


def tune_strassen(semiring, m, n, k, A, B, C, workspace, budget, variant=mmsr.MM_STRASSEN_WINOGRAD,
                  timer=cuda_timer, cache=None, persist=True):
    """Time every Strassen depth the budget allows; returns {"levels", "workspace", "ms"}."""
    kk = key("strassen%d" % variant, semiring, m, n, k, budget)
    with _lock:
        c = load_cache() if cache is None else cache
        if kk in c:
            return c[kk]
    best = None
    for L, w in strassen_candidates(semiring, m, n, k, budget):
        ms = timer(lambda: mmsr.mm_strassen(L, variant, semiring, m, n, k, A, B, C, workspace, w))
        if best is None or ms < best["ms"]:
            best = {"levels": L, "workspace": w, "ms": ms}
    with _lock:
        c[kk] = best
        if persist and cache is None:
            save_cache(c)
    return best


def mm_semiring_tuned(semiring, m, n, k, A, B, C, workspace, budget, stream=None):
    """mm_semiring with the cached best split factor for this shape and budget
    (falls back to the planner's own choice when the shape was never tuned)."""
    c = load_cache()
    rec = c.get(key("semiring", semiring, m, n, k, budget))
    b = rec["budget"] if rec and rec["budget"] <= budget else budget
    return mmsr.mm_semiring(semiring, m, n, k, A, B, C, workspace, b, stream)


BATCH_SPLITS = (0, 1, 2, 4, 8, 16)  # 0: the library's own rule


def batch_signature(problems) -> str:
    """Cache key of a batch: the multiset of (semiring, shape buckets)."""
    items = sorted("%d:%dx%dx%d" % (int(p[0]), _bucket(int(p[1])), _bucket(int(p[2])), _bucket(int(p[3])))
                   for p in problems)
    import hashlib

    return "batched/%d/%s" % (len(items), hashlib.sha1(",".join(items).encode()).hexdigest()[:16])


def batch_buckets(problems, min_k: int = 1024):
    """k buckets of the FP32 problems worth slicing (k >= min_k), longest
    first, each with the indices of its problems."""
    groups = {}
    for i, p in enumerate(problems):
        if int(p[0]) == mmsr.MM_SR_PLUS_TIMES_F32 and int(p[3]) >= min_k:
            groups.setdefault(_bucket(int(p[3])), []).append(i)
    return [(b, groups[b]) for b in sorted(groups, reverse=True)]


def apply_splits(problems, splits, levels=None):
    """The problem tuples with their split_k hints (and Strassen levels) set."""
    levels = levels or [int(p[8]) if len(p) > 8 else 0 for p in problems]
    return [tuple(p[:7]) + (int(h), int(lv)) for p, h, lv in zip(problems, splits, levels)]


def strassen_candidates_in_batch(problems, min_dim: int = 1024):
    """Indices of the FP32 problems one Strassen level may serve: every
    dimension at least min_dim and even."""
    return [i for i, p in enumerate(problems)
            if int(p[0]) == mmsr.MM_SR_PLUS_TIMES_F32 and min(int(p[1]), int(p[2]), int(p[3])) >= min_dim
            and not (int(p[1]) | int(p[2]) | int(p[3])) & 1]


def tune_batched(problems, workspace, workspace_bytes, timer=None, cache=None, persist=True,
                 candidates=BATCH_SPLITS):
    """Choose the k-slices of the batch's long-k FP32 problems.  problems:
    (semiring, m, n, k, A, B, C[, split_k]) tuples as ``mmsr.mm_batched``
    takes them.  Candidates whose workspace exceeds ``workspace_bytes`` are
    skipped.  Returns {"splits": [hint per problem], "levels": [Strassen
    levels per problem], "buckets": {k bucket: hint}, "ms": time of the chosen
    batch}."""
    timer = timer or cuda_timer
    kk = batch_signature(problems)
    buckets = batch_buckets(problems)
    with _lock:
        c = load_cache() if cache is None else cache
        if kk in c and len(c[kk].get("splits", [])) == len(problems):
            return c[kk]
    splits = [0] * len(problems)
    levels = [0] * len(problems)

    def run(sp, lv=None):
        table = apply_splits(problems, sp, lv or levels)
        if mmsr.mm_batched_query(table) > workspace_bytes:
            return None
        return timer(lambda: mmsr.mm_batched(table, workspace, workspace_bytes))

    best_ms = run(splits)
    chosen = {}
    for b, idx in buckets:
        best_h = 0
        for h in candidates:
            if h == 0:
                continue
            trial = list(splits)
            for i in idx:
                trial[i] = h
            ms = run(trial)
            if ms is not None and (best_ms is None or ms < best_ms):
                best_ms, best_h = ms, h
        for i in idx:
            splits[i] = best_h
        chosen[str(b)] = best_h
    big = strassen_candidates_in_batch(problems)
    if big:
        trial = list(levels)
        for i in big:
            trial[i] = 1
        ms = run(splits, trial)
        if ms is not None and (best_ms is None or ms < best_ms):
            best_ms, levels = ms, trial
    rec = {"splits": splits, "levels": levels, "buckets": chosen, "ms": best_ms}
    with _lock:
        c[kk] = rec
        if persist and cache is None:
            save_cache(c)
    return rec


def mm_batched_tuned(problems, workspace, workspace_bytes, stream=None):
    """mm_batched with the cached k-slice choices for this batch's signature
    (the library's own rule when the batch was never tuned)."""
    rec = load_cache().get(batch_signature(problems))
    table = problems
    if rec and len(rec.get("splits", [])) == len(problems):
        table = apply_splits(problems, rec["splits"], rec.get("levels"))
    return mmsr.mm_batched(table, workspace, workspace_bytes, stream)
