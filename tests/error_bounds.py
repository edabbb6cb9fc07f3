"""Stated tolerances of FP32-mode Strassen levels, derived from the standard
worst-case error analysis of Strassen-like algorithms, not fitted to any
measurement.

The analysis (R. P. Brent, 1970; N. J. Higham, Accuracy and Stability of
Numerical Algorithms, 2nd ed., SIAM 2002, Section 23.2.2: Theorem 23.3 for
Strassen's method and the corresponding bound for Winograd's variant) works in
the max norm ||X|| = max |x_ij|.  One level forms S_r = sum_p alpha_rp A_p and
T_r = sum_p beta_rp B_p from quadrants, multiplies P_r = S_r T_r at half size
and adds C_q = sum_r gamma_qr P_r.  With |alpha|, |beta|, |gamma| <= 1,
||S_r|| <= nnz(alpha_r) ||A|| and ||T_r|| <= nnz(beta_r) ||B||, so an error
bound e ||S_r|| ||T_r|| on each half-size product gives at most

    g = max_q  sum_r |gamma_qr| nnz(alpha_r) nnz(beta_r)

times e ||A|| ||B|| on C, plus rounding of the sums themselves (a few units
of u = 2^-24 per level, negligible beside the leaf's error).  g is 12 for the
formulas the paper prints (Section 5) and 18 for Winograd's variant, the two
growth factors of the cited bounds.

The FP32-mode leaf (bf16 hi/lo split, three products, 256-k chunks summed in
FP32) has an error bound linear in its inner dimension k: a fixed relative
error per term (the split's residual and the dropped lo*lo term) plus the
rounding of the chunk sums.  Each level halves k, so L levels bound the error
by (g/2)^L times the bound of the classic product of the same size: 6^L for
the paper's formulas and 9^L for Winograd's.  The classic FP32-mode product is
held to the FP32-mode tolerance (1e-5 relative Frobenius error), so a product
with L Strassen levels is held to 1e-5 (g/2)^L.  The worst-case factors are
far above the typical growth, so these tolerances are loose; they still fail
on a dropped term, a wrong sign or a misplaced block (errors of order one).
"""
import numpy as np

FP32_TOL = 1e-5


def growth_factor(alpha, beta, gamma):
    """Max-norm growth of one level: max_q sum_r |gamma_qr| nnz(alpha_r) nnz(beta_r)."""
    alpha, beta, gamma = (np.asarray(x) for x in (alpha, beta, gamma))
    sa = np.count_nonzero(alpha, axis=1)
    sb = np.count_nonzero(beta, axis=1)
    return int(np.max(np.abs(gamma) @ (sa * sb)))


def fp32_strassen_tol(variant, levels):
    """1e-5 x (g/2)^L with g computed from the library's coefficient tables."""
    from paper_1911_05328_gb300 import mmsr

    g = growth_factor(*mmsr.mm_strassen_tables(variant))
    return FP32_TOL * (g / 2.0) ** levels
