"""Pins for the CPU oracle: each check compares the oracle with something
other than itself -- closed forms, exact rational arithmetic, library
routines (numpy / scipy), independent algorithms (Strassen, Winograd,
Floyd-Warshall, graph search) and exhaustive enumeration -- so that a
dropped term, a wrong sign or index, or a transposed operand in the oracle
fails at least one of them."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1911_05328_gb300 import inputs

INF = oracle.INF
GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


# ----------------------------------------------------------------- (+,x) FP64
# Each pin is a function of the implementation under test (the oracle by
# default), so that tests/test_oracle_mutations.py can show that planted
# mistakes fail them.
def pin_f64_identity_and_zero(mm=oracle.mm_f64):
    A, B = inputs.uniform_f64(7, 5, 9, seed=11)
    np.testing.assert_array_equal(mm(A, np.eye(5)), A)
    np.testing.assert_array_equal(mm(np.eye(9)[:7, :7], A), A)
    np.testing.assert_array_equal(mm(A, np.zeros((5, 3))), np.zeros((7, 3)))


def pin_f64_rank1_closed_form(mm=oracle.mm_f64):
    # (u v^T)(w x^T) = (v . w) u x^T ; distinct m, k, n catch a transposed operand.
    rng = np.random.default_rng(3)
    u, v = rng.integers(-9, 10, 6), rng.integers(-9, 10, 4)
    w, x = rng.integers(-9, 10, 4), rng.integers(-9, 10, 11)
    A = np.outer(u, v).astype(np.float64)
    B = np.outer(w, x).astype(np.float64)
    expect = float(np.dot(v, w)) * np.outer(u, x).astype(np.float64)
    np.testing.assert_array_equal(mm(A, B), expect)


def pin_f64_exact_rational_error_bound(mm=oracle.mm_f64):
    # Exact rational sum of exact rational products; the oracle must sit
    # within the classical recursive-summation bound gamma_k * sum|a||b|.
    A, B = inputs.uniform_f64(5, 37, 6, seed=4)
    C = mm(A, B)
    u = 2.0 ** -53
    g = 37 * u / (1 - 37 * u)
    for i in range(5):
        for j in range(6):
            exact = sum(Fraction(A[i, t]) * Fraction(B[t, j]) for t in range(37))
            bound = g * sum(abs(A[i, t] * B[t, j]) for t in range(37))
            assert abs(Fraction(C[i, j]) - exact) <= Fraction(bound)


def test_f64_identity_and_zero_exact():
    pin_f64_identity_and_zero()


def test_f64_rank1_closed_form_nonsquare():
    pin_f64_rank1_closed_form()


def test_f64_exact_rational_error_bound():
    pin_f64_exact_rational_error_bound()


def test_f64_ascending_order_bitwise():
    # ascending-t recursive summation reproduced with a fused-free scalar loop
    # in Python's own float arithmetic: identical bits.
    A, B = inputs.uniform_f64(3, 50, 4, seed=8)
    C = oracle.mm_f64(A, B)
    for i in range(3):
        for j in range(4):
            s = 0.0
            for t in range(50):
                s = s + float(A[i, t]) * float(B[t, j])
            assert C[i, j] == s


def test_f64_matches_blas_within_bound():
    A, B = inputs.uniform_f64(64, 300, 48, seed=9)
    ref = A @ B
    C = oracle.mm_f64(A, B)
    bound = 300 * 2.0 ** -52 * (np.abs(A) @ np.abs(B))
    assert np.all(np.abs(C - ref) <= bound)


def test_f64_row_sampling_matches_full():
    A, B = inputs.uniform_f64(40, 17, 13, seed=10)
    rows = [0, 5, 19, 20, 39]
    np.testing.assert_array_equal(oracle.mm_f64(A, B, rows=rows), oracle.mm_f64(A, B)[rows])


def test_f32_inputs_widen_exactly():
    A, B = inputs.normal_f32(9, 33, 7, seed=2)
    np.testing.assert_array_equal(oracle.mm_f64(A, B), oracle.mm_f64(A.astype(np.float64), B.astype(np.float64)))


def test_sample_rows_cover_quadrant_edges():
    rows = oracle.sample_rows(16384)
    for lvl in range(1, 5):
        q = 16384 >> lvl
        for b in range(q, 16384, q):
            assert b - 1 in rows and b in rows
    assert rows[0] == 0 and rows[-1] == 16383 and 480 <= len(rows) <= 560


# ---------------------------------------------------------------- (+,x) int64
def test_i64_matches_numpy_exact():
    rng = np.random.default_rng(12)
    A = rng.integers(-1000, 1000, size=(23, 31))
    B = rng.integers(-1000, 1000, size=(31, 19))
    np.testing.assert_array_equal(oracle.mm_i64(A, B), A @ B)


@pytest.mark.parametrize("variant", ["strassen", "winograd"])
@pytest.mark.parametrize("levels", [1, 2, 3])
def test_strassen_variants_equal_classic(variant, levels):
    rng = np.random.default_rng(100 + levels)
    m, k, n = 8 * 3, 8 * 5, 8 * 2
    A = rng.integers(-100, 101, size=(m, k))
    B = rng.integers(-100, 101, size=(k, n))
    np.testing.assert_array_equal(oracle.strassen_i64(A, B, levels, variant), oracle.mm_i64(A, B))


def _golden_strassen():
    S, T, Cq = {}, {}, {}
    with open(__import__("os").path.join(GOLDEN, "strassen_paper_formulas.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "S":
                S[int(tok[1])] = [int(x) for x in tok[2:]]
            elif tok[0] == "T":
                T[int(tok[1])] = [int(x) for x in tok[2:]]
            else:
                Cq[tok[1]] = [int(x) for x in tok[2:]]
    return S, T, Cq


def test_golden_paper_table_is_matrix_product_and_matches_oracle():
    # Section 5 formulas as printed (golden table): evaluate them on random
    # integer quadrants and compare both to the classic product and to the
    # oracle's one-level Strassen.
    S, T, Cq = _golden_strassen()
    rng = np.random.default_rng(5)
    h = 3
    A = rng.integers(-50, 51, size=(2 * h, 2 * h))
    B = rng.integers(-50, 51, size=(2 * h, 2 * h))
    qa = [A[:h, :h], A[:h, h:], A[h:, :h], A[h:, h:]]
    qb = [B[:h, :h], B[:h, h:], B[h:, :h], B[h:, h:]]
    P = {r: sum(c * x for c, x in zip(S[r], qa)) @ sum(c * x for c, x in zip(T[r], qb)) for r in range(1, 8)}
    C = np.block([[sum(g * P[r + 1] for r, g in enumerate(Cq["00"])), sum(g * P[r + 1] for r, g in enumerate(Cq["01"]))],
                  [sum(g * P[r + 1] for r, g in enumerate(Cq["10"])), sum(g * P[r + 1] for r, g in enumerate(Cq["11"]))]])
    np.testing.assert_array_equal(C, A @ B)
    np.testing.assert_array_equal(oracle.strassen_i64(A, B, 1, "strassen"), C)


def test_strassen_rejects_bad_shape():
    with pytest.raises(RuntimeError):
        oracle.strassen_i64(np.ones((6, 6)), np.ones((6, 6)), 2)


# ------------------------------------------------------------------- (min,+)
def _tropical_identity(n):
    E = np.full((n, n), INF, dtype=np.int32)
    np.fill_diagonal(E, 0)
    return E


def pin_minplus_identity_and_zero(mm=oracle.mm_minplus):
    A, _ = inputs.tropical_i32(9, 6, 1, seed=13)
    np.testing.assert_array_equal(mm(A, _tropical_identity(6)), A)
    np.testing.assert_array_equal(mm(_tropical_identity(9), A), A)
    Z = np.full((6, 4), INF, dtype=np.int32)
    np.testing.assert_array_equal(mm(A, Z), np.full((9, 4), INF, dtype=np.int32))


def pin_minplus_sentinel_saturates_without_wrap(mm=oracle.mm_minplus):
    A = np.full((3, 4), INF, dtype=np.int32)
    B = np.full((4, 5), INF, dtype=np.int32)
    np.testing.assert_array_equal(mm(A, B), np.full((3, 5), INF, dtype=np.int32))
    A[1, 2] = 7
    B[2, 3] = INF - 3  # finite sum 2^30 + 4 clamps to the sentinel
    C = mm(A, B)
    assert C[1, 3] == INF


def pin_minplus_two_hop_paths_enumerated(mm=oracle.mm_minplus):
    # (D (x) D)[i][j] is the cheapest walk of exactly two edges (with the 0
    # diagonal, at most two): enumerate every walk explicitly.
    D = inputs.graph_minplus(5, seed=14, density=0.5, hi=20)
    C = mm(D, D)
    for i, j in itertools.product(range(5), repeat=2):
        best = INF
        for v in range(5):
            if D[i, v] < INF and D[v, j] < INF:
                best = min(best, int(D[i, v]) + int(D[v, j]))
        assert C[i, j] == best


def test_minplus_identity_and_zero():
    pin_minplus_identity_and_zero()


def test_minplus_sentinel_saturates_without_wrap():
    pin_minplus_sentinel_saturates_without_wrap()


def test_minplus_two_hop_paths_enumerated():
    pin_minplus_two_hop_paths_enumerated()


def test_minplus_squaring_equals_floyd_warshall_and_scipy():
    from scipy.sparse.csgraph import shortest_path

    for seed, nv in ((15, 17), (16, 40), (17, 64)):
        D = inputs.graph_minplus(nv, seed=seed, density=0.08)
        X = D.copy()
        for _ in range(math.ceil(math.log2(nv - 1))):
            X = oracle.mm_minplus(X, X)
        fw = oracle.floyd_warshall(D)
        np.testing.assert_array_equal(X.astype(np.int64), fw)
        W = np.where(D >= INF, 0, D).astype(np.float64)  # 0 = no edge for scipy dense input
        sp = shortest_path(W, method="D", directed=True)
        sp = np.where(np.isinf(sp), INF, sp).astype(np.int64)
        np.testing.assert_array_equal(fw, sp)


def test_minplus_k_split_associativity():
    # min over k in two halves, combined by min, equals the whole; catches an
    # off-by-one in the k loop.
    A, B = inputs.tropical_i32(11, 29, 7, seed=18)
    whole = oracle.mm_minplus(A, B)
    lo = oracle.mm_minplus(A[:, :13], B[:13])
    hi = oracle.mm_minplus(A[:, 13:], B[13:])
    np.testing.assert_array_equal(whole, np.minimum(lo, hi))


def test_minplus_matches_numpy_broadcast():
    # library-routine special case: numpy reduction over an explicit 3-D sum.
    A, B = inputs.tropical_i32(12, 10, 14, seed=19)
    ref = np.minimum((A.astype(np.int64)[:, :, None] + B.astype(np.int64)[None, :, :]).min(axis=1), INF)
    np.testing.assert_array_equal(oracle.mm_minplus(A, B), ref.astype(np.int32))


def test_minplus_k_zero_gives_sentinel():
    C = oracle.mm_minplus(np.zeros((3, 0), np.int32), np.zeros((0, 2), np.int32))
    np.testing.assert_array_equal(C, np.full((3, 2), INF, dtype=np.int32))


# ------------------------------------------------------------------- boolean
def pin_orand_exhaustive_2x2(mm=oracle.mm_orand):
    mats = [np.array(bits, dtype=np.uint8).reshape(2, 2) for bits in itertools.product((0, 1), repeat=4)]
    for A in mats:
        for B in mats:
            ref = ((A.astype(np.int64) @ B.astype(np.int64)) > 0).astype(np.uint8)
            np.testing.assert_array_equal(mm(A, B), ref)


def test_orand_exhaustive_2x2():
    pin_orand_exhaustive_2x2()


def test_orand_closure_equals_reachability():
    from scipy.sparse.csgraph import shortest_path

    A, _ = inputs.boolean_u8(30, 30, 1, seed=20, density=0.06)
    R = (A | np.eye(30, dtype=np.uint8)).astype(np.uint8)
    for _ in range(5):
        R = oracle.mm_orand(R, R)
    reach = np.isfinite(shortest_path(A.astype(np.float64), unweighted=True, directed=True)).astype(np.uint8)
    np.testing.assert_array_equal(R, reach)


# ------------------------------------------------------------------ closures
def _tropical_power_series(A):
    # A* = 1 (+) A (+) A^2 (+) ... (+) A^(n-1), each power by numpy broadcasting
    # (an independent min-plus product), summed with the semiring's min.
    n = A.shape[0]
    A = np.minimum(A.astype(np.int64), INF)
    one = np.full((n, n), INF, dtype=np.int64)
    np.fill_diagonal(one, 0)
    X, P = one.copy(), one.copy()
    for _ in range(max(n - 1, 0)):
        P = np.minimum((P[:, :, None] + A[None, :, :]).min(axis=1), INF)
        X = np.minimum(X, P)
    return X


def pin_minplus_closure_power_series_tiny(closure=oracle.closure_minplus):
    # Brute force on tiny inputs, including a nonzero diagonal that only the
    # semiring's 1 term of the closure clears.
    for seed, nv in ((30, 1), (31, 2), (32, 5), (33, 9)):
        D = inputs.graph_minplus(nv, seed=seed, density=0.4)
        rng = np.random.default_rng(seed)
        np.fill_diagonal(D, rng.integers(0, 50, size=nv))
        np.testing.assert_array_equal(closure(D), _tropical_power_series(D))


def pin_minplus_closure_scipy_dijkstra(closure=oracle.closure_minplus):
    from scipy.sparse.csgraph import shortest_path

    D = inputs.graph_minplus(70, seed=34, density=0.05)
    W = np.where(D >= INF, 0, D).astype(np.float64)
    sp = shortest_path(W, method="D", directed=True)
    sp = np.where(np.isinf(sp), INF, sp).astype(np.int64)
    np.testing.assert_array_equal(closure(D), sp)


def pin_minplus_closure_special_cases(closure=oracle.closure_minplus):
    # no arcs: the closure is the semiring's 1; zero-weight complete graph: all 0.
    n = 6
    none = np.full((n, n), INF, dtype=np.int32)
    one = np.full((n, n), INF, dtype=np.int64)
    np.fill_diagonal(one, 0)
    np.testing.assert_array_equal(closure(none), one)
    np.testing.assert_array_equal(closure(np.zeros((n, n), np.int32)), np.zeros((n, n)))
    # a directed path 0 -> 1 -> ... -> n-1 of unit arcs: C[i][j] = j - i above the diagonal.
    path = np.full((n, n), INF, dtype=np.int32)
    for i in range(n - 1):
        path[i, i + 1] = 1
    C = closure(path)
    for i in range(n):
        for j in range(n):
            assert C[i, j] == (j - i if j >= i else INF)


def test_minplus_closure_equals_power_series_tiny():
    pin_minplus_closure_power_series_tiny()


def test_minplus_closure_equals_scipy_dijkstra():
    pin_minplus_closure_scipy_dijkstra()


def test_minplus_closure_special_cases():
    pin_minplus_closure_special_cases()


def test_orand_closure_equals_scipy_and_power_series():
    from scipy.sparse.csgraph import shortest_path

    for seed, nv, dens in ((35, 1, 0.5), (36, 7, 0.2), (37, 45, 0.04)):
        A, _ = inputs.boolean_u8(nv, nv, 1, seed=seed, density=dens)
        A = A * 3  # nonzero means true
        reach = np.isfinite(shortest_path((A > 0).astype(np.float64), unweighted=True, directed=True))
        R = oracle.closure_orand(A)
        np.testing.assert_array_equal(R, reach.astype(np.uint8))
        X = np.eye(nv, dtype=np.int64)
        P = np.eye(nv, dtype=np.int64)
        for _ in range(max(nv - 1, 0)):
            P = ((P @ (A > 0).astype(np.int64)) > 0).astype(np.int64)
            X |= P
        np.testing.assert_array_equal(R, X.astype(np.uint8))


def test_minplus_closure_rows_dijkstra_matches_floyd_warshall():
    # two independent algorithms for the same closure rows; zero-weight arcs,
    # a nonzero diagonal and unreachable vertices included.
    for seed, nv, dens in ((38, 1, 0.5), (39, 13, 0.2), (40, 90, 0.05)):
        D = inputs.graph_minplus(nv, seed=seed, density=dens, hi=1000)
        rng = np.random.default_rng(seed)
        D[rng.random((nv, nv)) < 0.02] = 0
        np.fill_diagonal(D, rng.integers(0, 9, size=nv))
        rows = np.arange(nv)[:: max(1, nv // 7)]
        np.testing.assert_array_equal(oracle.closure_minplus_rows(D, rows), oracle.closure_minplus(D)[rows])
