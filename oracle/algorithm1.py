"""Algorithm 1 (Section 3.3) in the paper's own steps, in pure Python.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). For tiny inputs.

For every unique combination (Eq. 3.3), every product of an element pair at
that distance is formed once, and added to each output index that one of the
window's legal shifts maps it to (Section 3.3, "Write pattern"). The result is
the upper triangle of C (Eq. 2.2); it is then averaged over the K window
positions and mirrored, as the definition does.
"""
from __future__ import annotations

import numpy as np

from .combinations import initial_write_index, unique_combinations


def covariance_algorithm1(A, P: int, Q: int, mean: bool = True) -> np.ndarray:
    A = np.asarray(A, dtype=np.complex128)
    N, M = A.shape
    D = P * Q
    C = np.zeros((D, D), np.complex128)
    for dr, dc in unique_combinations(P, Q):
        a0, b0 = initial_write_index(P, dr, dc)
        # every element pair (r1, c1), (r2, c2) = (r1 + dr, c1 + dc) inside A
        for r1 in range(max(0, -dr), N - max(0, dr)):
            for c1 in range(0, M - dc):
                r2, c2 = r1 + dr, c1 + dc
                val = A[r1, c1] * np.conj(A[r2, c2])
                # initial placement: upper-left corner of the window that holds
                # the pair on its top and left borders
                p0, q0 = min(r1, r2), c1
                for t in range(Q - dc):            # steps leftward: +P
                    for s in range(P - abs(dr)):   # steps upward:   +1
                        p, q = p0 - s, q0 - t
                        if 0 <= p <= N - P and 0 <= q <= M - Q:
                            C[a0 + s + P * t, b0 + s + P * t] += val
    K = (N - P + 1) * (M - Q + 1)
    if mean:
        C = C / K
    R = np.triu(C) + np.conj(np.triu(C, 1)).T
    R[np.diag_indices(D)] = R.diagonal().real
    return R
