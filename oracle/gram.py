"""Eq. 2.2 as one Gram product, for inputs too large for the window loop.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Eq. 2.2 adds x x^H over the window positions. With the K column-stacked window
vectors x (Eq. 2.1) as the columns of X (PQ x K), that sum is the Gram matrix
X X^H. This module evaluates it with a library primitive, BLAS's Hermitian
rank-k update (zherk, through SciPy), in FP64: the columns of X are taken in
the order of the window positions (p, then q), one group of window rows at a
time, and each group's update is added into the same upper triangle. Then,
as in ``cov_window``: R = C / K by IEEE division (COV_MEAN), the lower
triangle is the conjugate of the upper one, and the diagonal is real.

It serves as the full-size reference where ``cov_window`` (about PQ^2 K / 2
complex multiply-adds through memory) would take minutes: the 2048 x 512
input with a 32 x 32 window is 5e11 multiply-adds. Its pins
(``tests/test_oracle_pins.py``) hold it to ``cov_window`` and brute force on
every small shape, bit for bit on integer inputs, and to the closed forms.
"""
from __future__ import annotations

import numpy as np


def _window_block(A: np.ndarray, p0: int, p1: int, P: int, Q: int) -> np.ndarray:
    """X^T for the window rows p0 <= p < p1: one row per position (p, q), in
    the order of p then q, holding x[i + P*j] = A[p+i][q+j]."""
    W = np.lib.stride_tricks.sliding_window_view(A[p0:p1 + P - 1], (P, Q))  # [p, q, i, j]
    return np.ascontiguousarray(W.transpose(0, 1, 3, 2)).reshape(-1, P * Q)


def cov_gram(A, P: int, Q: int, mean: bool = True, rows_per_group: int = 0) -> np.ndarray:
    """R of Eq. 2.1-2.2 (mean over all K = (N-P+1)(M-Q+1) positions, or the
    sum with ``mean=False``) as X X^H, FP64."""
    from scipy.linalg import blas

    A = np.ascontiguousarray(np.asarray(A), dtype=np.complex128)
    if A.ndim != 2:
        raise ValueError("A must be 2-D")
    N, M = A.shape
    if not (1 <= P <= N and 1 <= Q <= M):
        raise ValueError("window larger than the input")
    D = P * Q
    npr = N - P + 1
    if rows_per_group <= 0:  # about 64 MiB of X per group
        rows_per_group = max(1, (64 << 20) // max(1, 16 * D * (M - Q + 1)))
    C = np.zeros((D, D), dtype=np.complex128, order="F")
    for p0 in range(0, npr, rows_per_group):
        p1 = min(npr, p0 + rows_per_group)
        XT = _window_block(A, p0, p1, P, Q)  # C-order (positions x D) = F-order X
        C = blas.zherk(1.0, XT.T, beta=1.0, c=C, trans=0, lower=0, overwrite_c=1)
    U = np.triu(np.asarray(C))
    if mean:  # real and imaginary parts each divided by K (a complex
        # division by K + 0i would not be correctly rounded)
        K = float((N - P + 1) * (M - Q + 1))
        V = np.empty_like(U)
        V.real = U.real / K
        V.imag = U.imag / K
        U = V
    R = U + np.conj(np.triu(U, 1)).T
    R[np.diag_indices(D)] = U.diagonal().real
    return np.ascontiguousarray(R)
