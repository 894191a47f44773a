"""The minimum-variance (Capon) spectrum of a covariance estimate.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section 2.3 names the downstream uses of the estimated covariance matrix:
the Minimum Variance Method in SAR imaging (DeGraaf, on the covariance
matrices of overlapping 25 x 25 apertures with 10 x 10 sub-apertures) and the
Capon estimator. Capon's minimum-variance spectrum at a steering vector a is
P(a) = 1 / (a^H R^{-1} a); with diagonal loading d = loading * trace(R) / D
the matrix is R + d I. Written here from that definition in FP64, with a
library solve (NumPy) as the one step.
"""
from __future__ import annotations

import numpy as np


def capon_spectrum(R, steer, loading: float = 0.0) -> np.ndarray:
    """R: (count, D, D) or (D, D) Hermitian; steer: (F, D), row f = a_f.
    Returns (count, F) (or (F,)) real spectra P_k(f) = 1 / (a_f^H (R_k + d_k I)^{-1} a_f)."""
    R = np.asarray(R, dtype=np.complex128)
    single = R.ndim == 2
    if single:
        R = R[None]
    A = np.asarray(steer, dtype=np.complex128)
    count, D, _ = R.shape
    out = np.empty((count, A.shape[0]), np.float64)
    for k in range(count):
        d = loading * np.trace(R[k]).real / D
        Rl = R[k] + d * np.eye(D)
        X = np.linalg.solve(Rl, A.T)                     # (R + dI)^{-1} a_f, one column per f
        q = np.einsum("df,df->f", A.T.conj(), X).real    # a_f^H (R + dI)^{-1} a_f
        out[k] = 1.0 / q
    return out[0] if single else out


def steering_vectors(P: int, Q: int, omegas, nus) -> np.ndarray:
    """2-D steering vectors over the column-stacked window (x[i + P j]):
    a[i + P j] = exp(i (omega i + nu j)), one row per (omega, nu) pair."""
    i = np.arange(P)[:, None]
    j = np.arange(Q)[None, :]
    rows = []
    for w, v in zip(omegas, nus):
        rows.append(np.exp(1j * (w * i + v * j)).T.reshape(-1))  # index i + P j
    return np.array(rows)
