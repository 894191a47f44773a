"""Exact evaluation of Eq. 2.2 for Gaussian-integer inputs.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Uses Python integers, so the window sum is exact; the average is returned as
fractions. A correctly rounded FP64 division of that exact sum by K is the
value every exact-summing implementation must produce.
"""
from __future__ import annotations

from fractions import Fraction
from typing import List, Tuple


def window_sum_exact(A_re: List[List[int]], A_im: List[List[int]], P: int, Q: int
                     ) -> Tuple[List[List[int]], List[List[int]]]:
    """C[a][b] = sum over windows of x_a * conj(x_b), as exact integers."""
    N, M = len(A_re), len(A_re[0])
    D = P * Q
    Cre = [[0] * D for _ in range(D)]
    Cim = [[0] * D for _ in range(D)]
    for p in range(N - P + 1):
        for q in range(M - Q + 1):
            xr = [A_re[p + a % P][q + a // P] for a in range(D)]
            xi = [A_im[p + a % P][q + a // P] for a in range(D)]
            for a in range(D):
                for b in range(D):
                    Cre[a][b] += xr[a] * xr[b] + xi[a] * xi[b]
                    Cim[a][b] += xi[a] * xr[b] - xr[a] * xi[b]
    return Cre, Cim


def covariance_exact(A_re, A_im, P: int, Q: int, mean: bool = True):
    """R as Fractions (mean) or ints (sum): (R_re, R_im)."""
    Cre, Cim = window_sum_exact(A_re, A_im, P, Q)
    if not mean:
        return Cre, Cim
    N, M = len(A_re), len(A_re[0])
    K = (N - P + 1) * (M - Q + 1)
    D = P * Q
    return ([[Fraction(Cre[a][b], K) for b in range(D)] for a in range(D)],
            [[Fraction(Cim[a][b], K) for b in range(D)] for a in range(D)])
