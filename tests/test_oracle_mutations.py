"""Planted mistakes in the CPU oracle fail its pins.

Each mutant is the oracle with one plausible bug planted on the CPU (a
dropped term, a wrong index, a transposed operand or transposed addressing,
a wrong sign, the wrong (+) of the semiring, a missing clamp, a
lower-precision accumulator, a shifted output); every mutant must fail at
least one of the pins in tests/test_oracle_pins.py, while the oracle itself
passes all of them.  The closure mutants (Floyd-Warshall with the pivot loop
innermost, no semiring 1 on the diagonal, one squaring too few) are checked
against the closure pins the same way."""
import numpy as np
import pytest

import oracle
from test_oracle_pins import (pin_f64_exact_rational_error_bound, pin_f64_identity_and_zero,
                              pin_f64_rank1_closed_form, pin_minplus_closure_power_series_tiny,
                              pin_minplus_closure_scipy_dijkstra, pin_minplus_closure_special_cases,
                              pin_minplus_identity_and_zero, pin_minplus_sentinel_saturates_without_wrap,
                              pin_minplus_two_hop_paths_enumerated, pin_orand_exhaustive_2x2)

INF = oracle.INF

F64_PINS = [pin_f64_identity_and_zero, pin_f64_rank1_closed_form, pin_f64_exact_rational_error_bound]
MINPLUS_PINS = [pin_minplus_identity_and_zero, pin_minplus_sentinel_saturates_without_wrap,
                pin_minplus_two_hop_paths_enumerated]
ORAND_PINS = [pin_orand_exhaustive_2x2]
CLOSURE_PINS = [pin_minplus_closure_power_series_tiny, pin_minplus_closure_scipy_dijkstra,
                pin_minplus_closure_special_cases]


def _tropical(A, B, reduce, clamp=True, dtype=np.int64):
    S = A.astype(dtype)[:, :, None] + B.astype(dtype)[None, :, :]
    R = reduce(S, axis=1) if A.shape[1] else np.full((A.shape[0], B.shape[1]), INF, dtype=dtype)
    return (np.minimum(R, INF) if clamp else R).astype(np.int64)


F64_MUTANTS = {
    "drops the last k term": lambda A, B: oracle.mm_f64(A[:, :-1], B[:-1, :]),
    "reads B's rows in reverse k order": lambda A, B: oracle.mm_f64(A, np.ascontiguousarray(B[::-1])),
    "transposes B": lambda A, B: oracle.mm_f64(A, np.ascontiguousarray(B.T)),
    "indexes B column-major": lambda A, B: oracle.mm_f64(A, _col_major(B)),
    "subtracts the first term": lambda A, B: oracle.mm_f64(A, B) - 2.0 * np.outer(A[:, 0], B[0, :]),
    "accumulates in FP32": lambda A, B: (A.astype(np.float32) @ B.astype(np.float32)).astype(np.float64),
    "writes row i to row i + 1": lambda A, B: np.roll(oracle.mm_f64(A, B), 1, axis=0),
}

MINPLUS_MUTANTS = {
    "takes max as the (+)": lambda A, B: _tropical(A, B, np.max),
    "does not clamp to the sentinel": lambda A, B: _tropical(A, B, np.min, clamp=False),
    "adds in int32 with wrap-around": lambda A, B: _tropical(A, B, np.min, dtype=np.int32),
    "drops the last k term": lambda A, B: oracle.mm_minplus(A[:, :-1], B[:-1, :]),
    "reads B's rows in reverse k order": lambda A, B: oracle.mm_minplus(A, np.ascontiguousarray(B[::-1])),
    "transposes B": lambda A, B: oracle.mm_minplus(A, np.ascontiguousarray(B.T)),
    "indexes B column-major": lambda A, B: oracle.mm_minplus(A, _col_major(B)),
}

ORAND_MUTANTS = {
    "takes XOR as the (+)": lambda A, B: ((A.astype(np.int64) @ B.astype(np.int64)) % 2).astype(np.uint8),
    "takes AND as the (+)": lambda A, B: np.all((A[:, :, None] & B[None, :, :]) != 0, axis=1).astype(np.uint8),
    "drops the last k term": lambda A, B: oracle.mm_orand(A[:, :-1], B[:-1, :]),
    "transposes B": lambda A, B: oracle.mm_orand(A, np.ascontiguousarray(B.T)),
    "indexes B column-major": lambda A, B: oracle.mm_orand(A, _col_major(B)),
}


def _fw(A, pivot_innermost=False, reflexive=True):
    # Floyd-Warshall on 1 (+) A in plain Python (tiny graphs), with an optional bug
    D = np.minimum(np.asarray(A, dtype=np.int64), INF)
    n = D.shape[0]
    if reflexive:
        np.fill_diagonal(D, 0)
    D = D.tolist()
    order = ((i, j, v) for i in range(n) for j in range(n) for v in range(n)) if pivot_innermost else \
        ((i, j, v) for v in range(n) for i in range(n) for j in range(n))
    for i, j, v in order:
        if D[i][v] < INF and D[v][j] < INF and D[i][v] + D[v][j] < D[i][j]:
            D[i][j] = D[i][v] + D[v][j]
    return np.array(D, dtype=np.int64)


def _squarings(A, count):
    # repeated squaring of 1 (+) A through the (min,+) oracle, `count` times
    X = np.minimum(np.asarray(A, dtype=np.int64), INF)
    np.fill_diagonal(X, 0)
    for _ in range(count):
        X = oracle.mm_minplus(X.astype(np.int32), X.astype(np.int32)).astype(np.int64)
    return X


def _col_major(B):
    # B's buffer read with the index bug B[j * k + t] instead of B[t * n + j]:
    # same shape, transposed addressing
    k, n = B.shape
    return np.ascontiguousarray(B.reshape(n, k).T)


CLOSURE_MUTANTS = {
    "runs the pivot loop innermost": lambda A: _fw(A, pivot_innermost=True),
    "omits the semiring's 1 (diagonal)": lambda A: _fw(A, reflexive=False),
    "squares one time too few": lambda A: _squarings(A, max(0, (len(A) - 2).bit_length() - 1)),
}


def _failures(pins, mm):
    failed = []
    for pin in pins:
        try:
            with np.errstate(over="ignore"):
                pin(mm)
        except Exception:  # a wrong value, or a shape error the bug provokes
            failed.append(pin.__name__)
    return failed


@pytest.mark.parametrize("pins,mm", [(F64_PINS, oracle.mm_f64), (MINPLUS_PINS, oracle.mm_minplus),
                                     (ORAND_PINS, oracle.mm_orand), (CLOSURE_PINS, oracle.closure_minplus)])
def test_oracle_passes_every_pin(pins, mm):
    assert _failures(pins, mm) == []


@pytest.mark.parametrize("name", list(F64_MUTANTS))
def test_f64_mutant_is_caught(name):
    assert _failures(F64_PINS, F64_MUTANTS[name]), name


@pytest.mark.parametrize("name", list(MINPLUS_MUTANTS))
def test_minplus_mutant_is_caught(name):
    assert _failures(MINPLUS_PINS, MINPLUS_MUTANTS[name]), name


@pytest.mark.parametrize("name", list(ORAND_MUTANTS))
def test_orand_mutant_is_caught(name):
    assert _failures(ORAND_PINS, ORAND_MUTANTS[name]), name


def test_correct_reference_closures_pass():
    # the planted-bug helpers are correct without their bug
    assert _failures(CLOSURE_PINS, _fw) == []
    assert _failures(CLOSURE_PINS, lambda A: _squarings(A, max(0, (len(A) - 2).bit_length()))) == []


@pytest.mark.parametrize("name", list(CLOSURE_MUTANTS))
def test_closure_mutant_is_caught(name):
    assert _failures(CLOSURE_PINS, CLOSURE_MUTANTS[name]), name
