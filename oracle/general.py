"""General transfer functions h(A) = sum_i c_i A^i (Appendix A, oracle).

Theorem 2 (Eq. 32-33): h(W) = U1 g(Lambda1) U1^T + h(W - U1 Lambda1 U1^T)
with g(x) = h(x) - h(0).  Here h is a polynomial given by its coefficients, so
both sides can be evaluated exactly (Horner's rule on the black box).
"""
from __future__ import annotations

import numpy as np


def poly_apply(apply_A, coeffs, y: np.ndarray) -> np.ndarray:
    """sum_i c_i A^i y by Horner's rule with black-box A."""
    acc = np.zeros_like(np.asarray(y, dtype=np.float64))
    for c in reversed(list(coeffs)):
        acc = apply_A(acc) + c * y
    return acc


def poly_scalar(coeffs, lam) -> np.ndarray:
    lam = np.asarray(lam, dtype=np.float64)
    return sum(c * lam ** i for i, c in enumerate(coeffs))


def hybrid_poly(W, U1: np.ndarray, lam1: np.ndarray, coeffs, y: np.ndarray) -> np.ndarray:
    """x = U1 g(Lambda1) U1^T y + h(W_r) y for polynomial h (Eq. 32)."""
    g = poly_scalar(coeffs, lam1) - coeffs[0]
    xs = U1 @ (g * (U1.T @ y))
    Wr = lambda z: W @ z - U1 @ (lam1 * (U1.T @ z))  # noqa: E731
    return xs + poly_apply(Wr, coeffs, y)
