"""The library's Strassen coefficient tables (read through the C ABI, no GPU
needed): the paper variant equals the formulas printed in Section 5 (golden
table), and both variants satisfy the bilinear identity -- evaluated here on
random integer quadrants with numpy, independently of the oracle and of the
CUDA kernels -- so one level computes A*B exactly."""
import os

import numpy as np
import pytest

from paper_1911_05328_gb300 import build as mmsr_build
from paper_1911_05328_gb300 import mmsr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "strassen_paper_formulas.txt")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mmsr_build.build()


def _golden():
    S, T, C = np.zeros((7, 4), np.int64), np.zeros((7, 4), np.int64), np.zeros((4, 7), np.int64)
    qi = {"00": 0, "01": 1, "10": 2, "11": 3}
    for line in open(GOLDEN):
        if not line.strip() or line.startswith("#"):
            continue
        t = line.split()
        if t[0] == "S":
            S[int(t[1]) - 1] = [int(x) for x in t[2:]]
        elif t[0] == "T":
            T[int(t[1]) - 1] = [int(x) for x in t[2:]]
        else:
            C[qi[t[1]]] = [int(x) for x in t[2:]]
    return S, T, C


def test_paper_table_matches_section5():
    a, b, g = mmsr.mm_strassen_tables(mmsr.MM_STRASSEN_PAPER)
    S, T, C = _golden()
    np.testing.assert_array_equal(a, S)
    np.testing.assert_array_equal(b, T)
    np.testing.assert_array_equal(g, C)


@pytest.mark.parametrize("variant", [mmsr.MM_STRASSEN_PAPER, mmsr.MM_STRASSEN_WINOGRAD])
def test_bilinear_identity_exact(variant):
    a, b, g = mmsr.mm_strassen_tables(variant)
    rng = np.random.default_rng(variant + 1)
    h = 5
    A = rng.integers(-9, 10, size=(2 * h, 2 * h))
    B = rng.integers(-9, 10, size=(2 * h, 2 * h))
    qa = [A[:h, :h], A[:h, h:], A[h:, :h], A[h:, h:]]
    qb = [B[:h, :h], B[:h, h:], B[h:, :h], B[h:, h:]]
    P = [sum(a[r, q] * qa[q] for q in range(4)) @ sum(b[r, q] * qb[q] for q in range(4)) for r in range(7)]
    Cq = [sum(g[q, r] * P[r] for r in range(7)) for q in range(4)]
    np.testing.assert_array_equal(np.block([[Cq[0], Cq[1]], [Cq[2], Cq[3]]]), A @ B)


def test_winograd_term_counts():
    # fully expanded (no shared intermediates) Winograd has 14 A-terms,
    # 14 B-terms and 14 C-terms per level; the paper's Strassen 12/12/12
    for variant, cnt in ((mmsr.MM_STRASSEN_PAPER, 12), (mmsr.MM_STRASSEN_WINOGRAD, 14)):
        a, b, g = mmsr.mm_strassen_tables(variant)
        assert np.count_nonzero(a) == cnt and np.count_nonzero(b) == cnt and np.count_nonzero(g) == cnt


def test_strassen_workspace_is_reported():
    # O(n^2) for a fixed number of levels; grows with the leaf stacks
    prev = 0
    for L in range(1, 5):
        p = mmsr.mm_plan_query(mmsr.MM_SR_PLUS_TIMES_F32, L, 4096, 4096, 4096, 0)
        assert p.levels == L and p.workspace_min > prev
        assert p.workspace_min < 64 * 4096 * 4096 * 4
        prev = p.workspace_min


def test_growth_factors_of_the_standard_analysis():
    """The per-level max-norm growth of the cited worst-case analysis, from
    the tables: 12 for the printed formulas (golden table and library table
    alike), 18 for Winograd's variant; the FP32-mode Strassen tolerances are
    1e-5 x 6^L and 1e-5 x 9^L."""
    from error_bounds import fp32_strassen_tol, growth_factor

    S, T, C = _golden()
    assert growth_factor(S, T, C) == 12
    assert growth_factor(*mmsr.mm_strassen_tables(mmsr.MM_STRASSEN_PAPER)) == 12
    assert growth_factor(*mmsr.mm_strassen_tables(mmsr.MM_STRASSEN_WINOGRAD)) == 18
    assert abs(fp32_strassen_tol(mmsr.MM_STRASSEN_PAPER, 2) - 3.6e-4) < 1e-12
    assert abs(fp32_strassen_tol(mmsr.MM_STRASSEN_WINOGRAD, 4) - 1e-5 * 9 ** 4) < 1e-12
    # a plain classic block product (alpha = beta = unit rows, gamma summing
    # two products per quadrant) grows by 2 per level: (g/2)^L = 1
    a = np.zeros((8, 4), np.int64)
    b = np.zeros((8, 4), np.int64)
    g = np.zeros((4, 8), np.int64)
    for q, (i, j) in enumerate(((0, 0), (0, 1), (1, 0), (1, 1))):
        for t in range(2):
            r = 2 * q + t
            a[r, 2 * i + t] = 1
            b[r, 2 * t + j] = 1
            g[q, r] = 1
    assert growth_factor(a, b, g) == 2
