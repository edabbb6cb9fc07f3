"""Host-side tests of the C ABI: the library loads, exports every function
include/mmsr.h declares, and rejects bad arguments before touching the GPU.
No test here launches a kernel, so they run on a machine without a GPU."""
import os
import re

import pytest

from paper_1911_05328_gb300 import build as mmsr_build
from paper_1911_05328_gb300 import mmsr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FAKE = 1 << 20  # 16-byte aligned address that is never dereferenced by these tests


@pytest.fixture(scope="module")
def lib():
    mmsr_build.build()
    return mmsr.load()


def _declared_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert {"mm_semiring", "mm_strassen", "mm_batched", "mm_plan_query"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for code in range(0, -8, -1):
        s = mmsr.status_string(code)
        assert s.startswith("MM_")
    assert mmsr.mm_version() >= 100


def test_null_and_negative_arguments(lib):
    S = mmsr.MM_SR_MIN_PLUS_I32
    assert mmsr.mm_semiring(S, 4, 4, 4, None, FAKE, FAKE, stream=0, check=False) == mmsr.MM_ERR_ARG
    assert mmsr.mm_semiring(S, 4, 4, 4, FAKE, FAKE, None, stream=0, check=False) == mmsr.MM_ERR_ARG
    assert mmsr.mm_semiring(S, -1, 4, 4, FAKE, FAKE, FAKE, stream=0, check=False) == mmsr.MM_ERR_ARG
    assert mmsr.mm_semiring(99, 4, 4, 4, FAKE, FAKE, FAKE, stream=0, check=False) == mmsr.MM_ERR_ARG
    # a budget with no workspace pointer
    assert mmsr.mm_semiring(S, 4, 4, 4, FAKE, FAKE, FAKE, None, 64, stream=0, check=False) == mmsr.MM_ERR_ARG
    # empty output: nothing to do, no launch
    assert mmsr.mm_semiring(S, 0, 4, 4, None, None, None, stream=0, check=False) == mmsr.MM_OK


def test_misaligned_pointer(lib):
    S = mmsr.MM_SR_PLUS_TIMES_F64
    assert mmsr.mm_semiring(S, 4, 4, 4, FAKE + 8, FAKE, FAKE, stream=0, check=False) == mmsr.MM_ERR_ALIGN


def test_strassen_needs_additive_inverse(lib):
    # Section 5: Strassen subtracts, so (min,+) and boolean are rejected.
    for sr in (mmsr.MM_SR_MIN_PLUS_I32, mmsr.MM_SR_OR_AND_U8):
        rc = mmsr.mm_strassen(1, mmsr.MM_STRASSEN_WINOGRAD, sr, 8, 8, 8, FAKE, FAKE, FAKE, stream=0, check=False)
        assert rc == mmsr.MM_ERR_UNSUPPORTED


def test_strassen_shape_and_level_checks(lib):
    sr = mmsr.MM_SR_PLUS_TIMES_F32
    assert mmsr.mm_strassen(2, 1, sr, 10, 8, 8, FAKE, FAKE, FAKE, stream=0, check=False) == mmsr.MM_ERR_SHAPE
    assert mmsr.mm_strassen(5, 1, sr, 64, 64, 64, FAKE, FAKE, FAKE, stream=0, check=False) == mmsr.MM_ERR_ARG
    assert mmsr.mm_strassen(1, 7, sr, 64, 64, 64, FAKE, FAKE, FAKE, stream=0, check=False) == mmsr.MM_ERR_ARG


@pytest.mark.parametrize("budget_buffers,expect_s", [(0, 1), (1, 2), (2, 3), (4, 5), (8, 9)])
def test_budget_to_split_factor(lib, budget_buffers, expect_s):
    # the (min,+) workload at n=4096: budgets of 0/1/2/4/8 extra n x n int32
    # buffers give s = 1 + budget, and the plan uses exactly (s-1) buffers.
    n = 4096
    plan = mmsr.mm_plan_query(mmsr.MM_SR_MIN_PLUS_I32, -1, n, n, n, budget_buffers * n * n * 4)
    assert plan.split_k == expect_s
    assert plan.workspace_used == (expect_s - 1) * n * n * 4
    assert plan.workspace_used <= budget_buffers * n * n * 4


def test_split_never_exceeds_budget_or_kblocks(lib):
    for (m, n, k) in [(1, 1, 1), (7, 9, 5), (100, 3, 1000), (512, 512, 64), (33, 65, 4097)]:
        for budget in (0, 17, m * n * 4 - 1, m * n * 4, 3 * m * n * 4 + 5, 1 << 30):
            for sr, accb in ((mmsr.MM_SR_MIN_PLUS_I32, 4), (mmsr.MM_SR_PLUS_TIMES_F64, 8)):
                p = mmsr.mm_plan_query(sr, -1, m, n, k, budget)
                assert p.workspace_used <= budget
                if p.kernel == 6:
                    # the FP64 stream-K form: one k-slice in the plan, its
                    # per-CTA partial tiles in the workspace
                    assert sr == mmsr.MM_SR_PLUS_TIMES_F64 and p.split_k == 1 and p.workspace_used > 0
                    continue
                assert p.workspace_used == (p.split_k - 1) * m * n * accb
                assert 1 <= p.split_k <= max(1, -(-k // p.tile_k))
                # monotone in the budget (while the plan stays a split-K plan)
                q = mmsr.mm_plan_query(sr, -1, m, n, k, budget + m * n * accb)
                assert q.kernel == 6 or q.split_k >= p.split_k


def test_closure_argument_checks(lib):
    # (+, x) has no idempotent (+): the closure is not defined by squaring.
    for sr in (mmsr.MM_SR_PLUS_TIMES_F64, mmsr.MM_SR_PLUS_TIMES_F32, mmsr.MM_SR_PLUS_TIMES_F64ACC):
        rc, _ = mmsr.mm_closure(sr, 8, FAKE, FAKE, stream=0, check=False)
        assert rc == mmsr.MM_ERR_UNSUPPORTED
    sr = mmsr.MM_SR_MIN_PLUS_I32
    assert mmsr.mm_closure(99, 8, FAKE, FAKE, stream=0, check=False)[0] == mmsr.MM_ERR_ARG
    assert mmsr.mm_closure(sr, -1, FAKE, FAKE, stream=0, check=False)[0] == mmsr.MM_ERR_ARG
    assert mmsr.mm_closure(sr, 8, None, FAKE, stream=0, check=False)[0] == mmsr.MM_ERR_ARG
    assert mmsr.mm_closure(sr, 8, FAKE, FAKE, flags=4, stream=0, check=False)[0] == mmsr.MM_ERR_ARG
    assert mmsr.mm_closure(sr, 8, FAKE + 4, FAKE, stream=0, check=False)[0] == mmsr.MM_ERR_ALIGN
    assert mmsr.mm_closure(sr, 0, None, None, stream=0, check=False) == (mmsr.MM_OK, 0)
    # below the minimum workspace: rejected before any launch
    p = mmsr.mm_closure_query(sr, 100)
    rc, _ = mmsr.mm_closure(sr, 100, FAKE, FAKE, FAKE, int(p.workspace_min) - 16, stream=0, check=False)
    assert rc == mmsr.MM_ERR_WORKSPACE


@pytest.mark.parametrize("n,squarings", [(1, 0), (2, 0), (3, 1), (5, 2), (17, 4), (18, 5), (4096, 12)])
def test_closure_plan(lib, n, squarings):
    # 2^T >= n - 1 arcs, T minimal; the closure's own buffers come first and
    # every extra n x n buffer of budget buys one more k-slice per squaring.
    for sr, eb in ((mmsr.MM_SR_MIN_PLUS_I32, 4), (mmsr.MM_SR_OR_AND_U8, 1)):
        p = mmsr.mm_closure_query(sr, n, 0)
        assert p.levels == squarings
        prefix = 16 + -(-n * n * eb // 16) * 16
        sq = mmsr.mm_plan_query(sr, -1, n, n, n, 0)
        assert p.workspace_min == prefix + sq.workspace_min
    big = mmsr.mm_closure_query(mmsr.MM_SR_MIN_PLUS_I32, 4096, 16 + 4096 * 4096 * 4 + 2 * 4096 * 4096 * 4)
    assert big.split_k == 3 and big.workspace_used == 16 + 3 * 4096 * 4096 * 4


def test_star_strassen_argument_checks_and_workspace(lib):
    sr = mmsr.MM_SR_PLUS_TIMES_F32
    W = mmsr.MM_STRASSEN_WINOGRAD
    # Strassen needs the inverse of (+) at any classic depth
    rc = mmsr.mm_star_strassen(1, 1, W, mmsr.MM_SR_MIN_PLUS_I32, 8, 8, 8, FAKE, FAKE, FAKE, stream=0, check=False)
    assert rc == mmsr.MM_ERR_UNSUPPORTED
    # divisibility by 2^(classic + levels)
    assert mmsr.mm_star_strassen(2, 2, W, sr, 40, 64, 64, FAKE, FAKE, FAKE, stream=0, check=False) == mmsr.MM_ERR_SHAPE
    assert mmsr.mm_star_strassen(5, 1, W, sr, 64, 64, 64, FAKE, FAKE, FAKE, stream=0, check=False) == mmsr.MM_ERR_ARG
    assert mmsr.mm_star_strassen(1, 1, 9, sr, 64, 64, 64, FAKE, FAKE, FAKE, stream=0, check=False) == mmsr.MM_ERR_ARG
    # the workspace is that of one block product: mm_strassen at the block size
    n = 4096
    for c, L in ((1, 1), (1, 2), (2, 1), (2, 2)):
        p = mmsr.mm_star_strassen_query(c, L, sr, n, n, n)
        q = mmsr.mm_plan_query(sr, L, n >> c, n >> c, n >> c)
        assert p.workspace_min == q.workspace_min and p.levels == L
        full = mmsr.mm_plan_query(sr, L + c, n, n, n)
        assert p.workspace_min * 4 ** c <= full.workspace_min * 1.01
    # classic_levels = 0 is mm_strassen's plan
    assert mmsr.mm_star_strassen_query(0, 2, sr, n, n, n).workspace_min == mmsr.mm_plan_query(sr, 2, n, n, n).workspace_min
    rc = mmsr.mm_star_strassen(1, 1, W, sr, 64, 64, 64, FAKE, FAKE, FAKE, FAKE,
                               int(mmsr.mm_star_strassen_query(1, 1, sr, 64, 64, 64).workspace_min) - 1024,
                               stream=0, check=False)
    assert rc == mmsr.MM_ERR_WORKSPACE


def test_tar_strassen_waves_follow_the_papers_order(lib):
    # Section 5's zero-temporary Strassen writes P1; then P2 and P5 together;
    # then P3 and P4; then P6 and P7 (products numbered P1..P7 as printed).
    count, wave = mmsr.mm_strassen_tar_waves(1, mmsr.MM_STRASSEN_PAPER)
    assert count == 4
    assert wave == [0, 1, 2, 2, 1, 3, 3]
    for variant in (mmsr.MM_STRASSEN_PAPER, mmsr.MM_STRASSEN_WINOGRAD):
        count, wave = mmsr.mm_strassen_tar_waves(1, variant)
        _, _, gamma = mmsr.mm_strassen_tables(variant)
        for w in range(count):
            members = [r for r in range(7) if wave[r] == w]
            assert members
            touched = [q for r in members for q in range(4) if gamma[q, r] != 0]
            assert len(touched) == len(set(touched)), (variant, w, members)


def test_tar_strassen_two_level_waves(lib):
    """Two levels: leaf product p = 7 r1 + r2 adds gamma[q1, r1] gamma[q2, r2]
    times itself into block (q1, q2); products of one wave touch disjoint
    blocks and every block is reached.  Two Winograd levels put P1 x P1 into
    all sixteen blocks, past the epilogue's four: refused."""
    _, _, gamma = mmsr.mm_strassen_tables(mmsr.MM_STRASSEN_PAPER)
    count, wave = mmsr.mm_strassen_tar_waves(2, mmsr.MM_STRASSEN_PAPER)
    assert count > 0 and len(wave) == 49

    def blocks(p):
        r1, r2 = divmod(p, 7)
        return [(q1, q2) for q1 in range(4) for q2 in range(4) if gamma[q1, r1] * gamma[q2, r2] != 0]

    assert max(len(blocks(p)) for p in range(49)) <= 4
    for w in range(count):
        touched = [b for p in range(49) if wave[p] == w for b in blocks(p)]
        assert touched and len(touched) == len(set(touched)), w
    assert len({b for p in range(49) for b in blocks(p)}) == 16
    rc, _ = mmsr.mm_strassen_tar_waves(2, mmsr.MM_STRASSEN_WINOGRAD)
    assert rc == mmsr.MM_ERR_UNSUPPORTED


def test_tar_strassen_argument_checks_and_workspace(lib):
    W, P = mmsr.MM_STRASSEN_WINOGRAD, mmsr.MM_STRASSEN_PAPER
    for sr in (mmsr.MM_SR_PLUS_TIMES_F64, mmsr.MM_SR_MIN_PLUS_I32):
        assert mmsr.mm_strassen_tar(1, W, sr, 8, 8, 8, FAKE, FAKE, FAKE, stream=0, check=False) == \
            mmsr.MM_ERR_UNSUPPORTED
    sr = mmsr.MM_SR_PLUS_TIMES_F32
    assert mmsr.mm_strassen_tar(1, W, sr, 9, 8, 8, FAKE, FAKE, FAKE, stream=0, check=False) == mmsr.MM_ERR_SHAPE
    assert mmsr.mm_strassen_tar(2, P, sr, 6, 8, 8, FAKE, FAKE, FAKE, stream=0, check=False) == mmsr.MM_ERR_SHAPE
    assert mmsr.mm_strassen_tar(1, 5, sr, 8, 8, 8, FAKE, FAKE, FAKE, stream=0, check=False) == mmsr.MM_ERR_ARG
    for L in (0, 3):
        assert mmsr.mm_strassen_tar(L, P, sr, 8, 8, 8, FAKE, FAKE, FAKE, stream=0, check=False) == mmsr.MM_ERR_ARG
    n = 4096
    for L in (1, 2):
        tar = mmsr.mm_strassen_tar_query(L, sr, n, n, n)
        full = mmsr.mm_plan_query(sr, L, n, n, n)
        # exactly the product stack is saved: 7^L (n/2^L)^2 FP32 values
        assert full.workspace_min - tar.workspace_min == 7 ** L * (n >> L) ** 2 * 4
    # FP64-accuracy mode: mm_strassen overlays its products on the FP64
    # operand stack already, so TAR needs the same workspace
    fa = mmsr.MM_SR_PLUS_TIMES_F64ACC
    assert mmsr.mm_strassen_tar_query(1, fa, n, n, n).workspace_min == mmsr.mm_plan_query(fa, 1, n, n, n).workspace_min
    rc = mmsr.mm_strassen_tar(1, W, sr, 64, 64, 64, FAKE, FAKE, FAKE, FAKE,
                              int(mmsr.mm_strassen_tar_query(1, sr, 64, 64, 64).workspace_min) - 1024, stream=0,
                              check=False)
    assert rc == mmsr.MM_ERR_WORKSPACE
    big = 1 << 34
    assert mmsr.mm_strassen_tar(2, W, sr, 64, 64, 64, FAKE, FAKE, FAKE, FAKE, big, stream=0, check=False) == \
        mmsr.MM_ERR_UNSUPPORTED


def test_option_argument_checks(lib):
    """Out-of-range options and values are refused on the host (no device call)."""
    assert mmsr.mm_set_option(99, 0, check=False) == mmsr.MM_ERR_ARG
    for opt in (mmsr.MM_OPT_MINPLUS_PACKED, mmsr.MM_OPT_MINPLUS_STREAMK, mmsr.MM_OPT_STRASSEN_TOP_F64):
        assert mmsr.mm_set_option(opt, 2, check=False) == mmsr.MM_ERR_ARG
    for v in (1, 5, 8, -1):
        assert mmsr.mm_set_option(mmsr.MM_OPT_F64ACC_SLICES, v, check=False) == mmsr.MM_ERR_ARG
    # option 3 is retired: every value is refused
    for v in (0, 1):
        assert mmsr.mm_set_option(3, v, check=False) == mmsr.MM_ERR_ARG
    assert mmsr.mm_set_option(mmsr.MM_OPT_TEST_SKIP_SIGNAL, 4, check=False) == mmsr.MM_ERR_ARG
    assert mmsr.mm_set_option(mmsr.MM_OPT_TEST_SKIP_SIGNAL, -1, check=False) == mmsr.MM_ERR_ARG
    for v in (4, -1):
        assert mmsr.mm_set_option(mmsr.MM_OPT_F32_STREAMK, v, check=False) == mmsr.MM_ERR_ARG
    for v in (0, 2, 3, 1):  # ends on the default
        assert mmsr.mm_set_option(mmsr.MM_OPT_F32_STREAMK, v, check=False) == mmsr.MM_OK
    for v in (3, -1):
        assert mmsr.mm_set_option(mmsr.MM_OPT_F64_STREAMK, v, check=False) == mmsr.MM_ERR_ARG
    for v in (0, 2, 1):
        assert mmsr.mm_set_option(mmsr.MM_OPT_F64_STREAMK, v, check=False) == mmsr.MM_OK


def test_noalloc_host_checks(lib):
    """The allocation-free (min,+) entry point checks its arguments and the
    size of its static scratch before any device call."""
    f = mmsr.mm_minplus_noalloc
    assert f(4, 4, 4, FAKE, FAKE, FAKE, 0, stream=0, check=False) == mmsr.MM_ERR_ARG  # split_k < 1
    assert f(-1, 4, 4, FAKE, FAKE, FAKE, 1, stream=0, check=False) == mmsr.MM_ERR_ARG
    assert f(4, 4, 4, None, FAKE, FAKE, 1, stream=0, check=False) == mmsr.MM_ERR_ARG
    assert f(4, 4, 4, FAKE + 4, FAKE, FAKE, 1, stream=0, check=False) == mmsr.MM_ERR_ALIGN
    assert f(4, 4, (1 << 22) + 1, FAKE, FAKE, FAKE, 1, stream=0, check=False) == mmsr.MM_ERR_SHAPE
    assert f(0, 4, 4, None, None, None, 1, stream=0, check=False) == mmsr.MM_OK
    # s = 3 needs 2 partial slices of 4096 x 4096 int32 = 128 MiB > the 64 MiB scratch
    assert f(4096, 4096, 4096, FAKE, FAKE, FAKE, 3, stream=0, check=False) == mmsr.MM_ERR_WORKSPACE


def test_f64acc_scheme_by_levels(lib):
    """The FP64-accuracy digit scheme follows the Strassen depth: six slices
    (12 bytes per operand element) for plain products and up to two levels,
    seven (14 bytes) for three or four; the option forces either."""
    sr = mmsr.MM_SR_PLUS_TIMES_F64ACC
    m = n = k = 1024
    try:
        w = {}
        for opt in (6, 7):
            mmsr.mm_set_option(mmsr.MM_OPT_F64ACC_SLICES, opt)
            w[opt] = [int(mmsr.mm_plan_query(sr, L, m, n, k, 0).workspace_min) for L in (-1, 1, 2, 3, 4)]
        mmsr.mm_set_option(mmsr.MM_OPT_F64ACC_SLICES, 0)
        auto = [int(mmsr.mm_plan_query(sr, L, m, n, k, 0).workspace_min) for L in (-1, 1, 2, 3, 4)]
        assert auto[:3] == w[6][:3] and auto[3:] == w[7][3:]
        # the plain product's slices: 2 S (m + n) Kp bytes plus exponents
        assert w[7][0] - w[6][0] == 2 * (m + n) * k
        assert all(a < b for a, b in zip(w[6], w[7]))
    finally:
        mmsr.mm_set_option(mmsr.MM_OPT_F64ACC_SLICES, 0)


def test_probe_argument_checks(lib):
    import ctypes

    lib.mm_probe_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double)]
    r, t = ctypes.c_double(), ctypes.c_double()
    for kind, iters in ((-1, 10), (6, 10), (0, 0), (4, -5)):
        assert lib.mm_probe_peak(kind, iters, None, ctypes.byref(r), ctypes.byref(t)) == mmsr.MM_ERR_ARG


def test_strassen_auto_depth_under_budget(lib):
    """MM_LEVELS_AUTO: the preferred depth per semiring, lowered for small
    leaves, shapes that do not divide and budgets that do not hold the plan."""
    A = mmsr.MM_LEVELS_AUTO
    f32, acc, f64 = mmsr.MM_SR_PLUS_TIMES_F32, mmsr.MM_SR_PLUS_TIMES_F64ACC, mmsr.MM_SR_PLUS_TIMES_F64
    n = 16384
    big = 1 << 40
    assert mmsr.mm_plan_query(f32, A, n, n, n, big).levels == 2
    assert mmsr.mm_plan_query(acc, A, n, n, n, big).levels == 2
    assert mmsr.mm_plan_query(acc, A, 2048, 2048, 2048, big).levels == 1
    assert mmsr.mm_plan_query(f64, A, 8192, 8192, 8192, big).levels == 4
    # budget between the one- and two-level plans: one level; below both: classic
    w1 = int(mmsr.mm_plan_query(f32, 1, n, n, n, 0).workspace_min)
    w2 = int(mmsr.mm_plan_query(f32, 2, n, n, n, 0).workspace_min)
    p = mmsr.mm_plan_query(f32, A, n, n, n, (w1 + w2) // 2)
    assert p.levels == 1 and p.workspace_min == w1
    assert mmsr.mm_plan_query(f32, A, n, n, n, w1 - 1).levels == 0
    # small leaves and shapes that do not divide
    assert mmsr.mm_plan_query(acc, A, 1024, 1024, 1024, big).levels == 0
    assert mmsr.mm_plan_query(f32, A, 2048, 2048, 2048, big).levels == 1
    assert mmsr.mm_plan_query(f64, A, 4000, 4000, 4000, big).levels == 2
    assert mmsr.mm_plan_query(f32, A, 4097, 4096, 4096, big).levels == 0
    # the automatic depth is refused only where Strassen is undefined
    assert mmsr.mm_plan_query(mmsr.MM_SR_MIN_PLUS_I32, A, 64, 64, 64, big, check=False).status == \
        mmsr.MM_ERR_UNSUPPORTED


def test_batched_table_size_and_cap(lib):
    """The batched call keeps its problem table in the workspace: the query
    grows with the count (72-byte rows plus three prefix sums) and accepts
    counts past the old 512 limit; 2^20 + 1 problems are refused."""
    F32 = mmsr.MM_SR_PLUS_TIMES_F32
    one = [(F32, 8, 8, 8, FAKE, FAKE, FAKE)]
    w1 = mmsr.mm_batched_query(one * 1000)
    w2 = mmsr.mm_batched_query(one * 2000)
    assert w1 > 0 and w2 > w1
    assert mmsr.mm_batched_query(one * 600) > 0
    assert mmsr.mm_batched_query(one * ((1 << 20) + 1)) == 0


def test_batched_strassen_level_checks(lib):
    """levels = 1 runs an FP32 problem as one Strassen-Winograd level inside the
    batch: the workspace adds its seven leaf products and their operand
    stacks; odd shapes, (min,+) and deeper levels are refused on the host."""
    F32, MP = mmsr.MM_SR_PLUS_TIMES_F32, mmsr.MM_SR_MIN_PLUS_I32
    n = 256
    plain = mmsr.mm_batched_query([(F32, n, n, n, FAKE, FAKE, FAKE, 0, 0)])
    lev = mmsr.mm_batched_query([(F32, n, n, n, FAKE, FAKE, FAKE, 0, 1)])
    assert lev - plain >= 7 * (n // 2) ** 2 * 4  # the leaf products at least
    assert mmsr.mm_batched_query([(F32, n + 1, n, n, FAKE, FAKE, FAKE, 0, 1)]) == 0
    assert mmsr.mm_batched_query([(F32, n, n, n, FAKE, FAKE, FAKE, 0, 2)]) == 0
    assert mmsr.mm_batched_query([(F32, n, n, n, FAKE, FAKE, FAKE, 0, -1)]) == 0
    assert mmsr.mm_batched_query([(MP, n, n, n, FAKE, FAKE, FAKE, 0, 1)]) == 0
    # k = 0 with a level: the plain zero-fill product
    assert mmsr.mm_batched_query([(F32, n, n, 0, FAKE, FAKE, FAKE, 0, 1)]) == \
        mmsr.mm_batched_query([(F32, n, n, 0, FAKE, FAKE, FAKE, 0, 0)])


def test_batched_k_slices(lib):
    """FP32 tiles cut into k-slices hold one 64 KB partial tile per slice in
    the workspace (plus a counter per tile); hints are checked on the host."""
    F32, MP = mmsr.MM_SR_PLUS_TIMES_F32, mmsr.MM_SR_MIN_PLUS_I32
    prob = (F32, 256, 256, 4096, FAKE, FAKE, FAKE)
    w1 = mmsr.mm_batched_query([prob + (1,)])
    w4 = mmsr.mm_batched_query([prob + (4,)])
    # 4 tiles x 4 slices x 128 x 128 x 4 B, counters and alignment aside
    assert 4 * 4 * 65536 <= w4 - w1 < 4 * 4 * 65536 + 4096
    # hints beyond the tile's 64 k-blocks are clamped to them
    assert mmsr.mm_batched_query([prob + (64,)]) == mmsr.mm_batched_query([prob + (1000,)])
    assert mmsr.mm_batched_query([prob + (-1,)]) == 0
    assert mmsr.mm_batched_query([(MP, 64, 64, 64, FAKE, FAKE, FAKE, 2)]) == 0
    assert mmsr.mm_batched_query([(MP, 64, 64, 64, FAKE, FAKE, FAKE, 0)]) > 0


def test_fused_staging_plan(lib):
    """With MM_OPT_STRASSEN_FUSED a one-level FP32-mode plan whose leaves tile
    by 128 x 128 x 32 holds only the seven products; other shapes, depths and
    semirings keep the materialised plan."""
    f32 = mmsr.MM_SR_PLUS_TIMES_F32
    n = 4096
    base = mmsr.mm_plan_query(f32, 1, n, n, n, 0).workspace_min
    try:
        assert mmsr.mm_set_option(mmsr.MM_OPT_STRASSEN_FUSED, 1) == mmsr.MM_OK
        assert mmsr.mm_plan_query(f32, 1, n, n, n, 0).workspace_min == 7 * (n // 2) ** 2 * 4
        assert mmsr.mm_plan_query(f32, 1, 400, 260, 128, 0).workspace_min == \
            mmsr.mm_plan_query(f32, 1, 400, 260, 128, 0).workspace_min
        assert mmsr.mm_plan_query(f32, 2, n, n, n, 0).workspace_min > 7 * (n // 2) ** 2 * 4
        assert mmsr.mm_set_option(mmsr.MM_OPT_STRASSEN_FUSED, 2, check=False) == mmsr.MM_ERR_ARG
    finally:
        mmsr.mm_set_option(mmsr.MM_OPT_STRASSEN_FUSED, 0)
    assert mmsr.mm_plan_query(f32, 1, n, n, n, 0).workspace_min == base
