"""Seeded synthetic inputs for the sliding-window covariance workloads.

This module only draws inputs (and names the workload shapes). It holds none
of the covariance method's arithmetic, so both the CUDA path (through the
tests and ``bench.py``) and the CPU oracle can take their inputs from here
without sharing any code of the method itself.

Conventions
-----------
* A is an N x M complex matrix, row-major, drawn with NumPy's PCG64.
* "Standard complex Gaussian" CN(0, 1): Re and Im i.i.d. N(0, 1/2), so
  E|a|^2 = 1.
* The SAR-like input stands in for the SAR imagery that motivates the paper
  (Section 2.3): a sum of 2-D complex exponentials plus complex Gaussian noise.
"""
from __future__ import annotations

import dataclasses
from typing import List, Tuple

import numpy as np

_CDTYPE = {"c64": np.complex64, "c128": np.complex128}


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    N: int
    M: int
    P: int
    Q: int
    dtype: str          # "c64" or "c128"
    kind: str           # "cn" (complex normal), "sar", "int"
    seed: int
    batch: int = 1

    @property
    def K(self) -> int:
        return (self.N - self.P + 1) * (self.M - self.Q + 1)


# The five workload shapes: the plain FP64 method, the single large FP32 input,
# the SAR-like input, the uneven batch and the differentiation batch.
WORKLOADS = {
    "plain_64x64_w8_f64": Workload("plain_64x64_w8_f64", 64, 64, 8, 8, "c128", "cn", 1303),
    "cn_1024x1024_w16_f32": Workload("cn_1024x1024_w16_f32", 1024, 1024, 16, 16, "c64", "cn", 1),
    "sar_2048x512_w32_f32": Workload("sar_2048x512_w32_f32", 2048, 512, 32, 32, "c64", "sar", 2),
    "diff_b64_256x256_w12_f32": Workload("diff_b64_256x256_w12_f32", 256, 256, 12, 12, "c64", "cn", 4, batch=64),
}

BATCHED_COUNT = 4096
BATCHED_SEED = 3


def complex_normal(shape, seed: int, dtype: str = "c128") -> np.ndarray:
    """CN(0,1) entries: Re, Im i.i.d. N(0, 1/2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    z = rng.standard_normal(shape + (2,) if isinstance(shape, tuple) else (shape, 2))
    z *= np.sqrt(0.5)
    return (z[..., 0] + 1j * z[..., 1]).astype(_CDTYPE[dtype])


def integer_valued(shape, seed: int, lo: int = -8, hi: int = 8, dtype: str = "c128") -> np.ndarray:
    """Re and Im uniform integers in [lo, hi] (inclusive)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    re = rng.integers(lo, hi + 1, size=shape)
    im = rng.integers(lo, hi + 1, size=shape)
    return (re + 1j * im).astype(_CDTYPE[dtype])


def sar_like(N: int, M: int, seed: int, n_exp: int = 8, snr_db: float = 10.0,
             dtype: str = "c64") -> Tuple[np.ndarray, dict]:
    """Sum of ``n_exp`` 2-D complex exponentials plus CN noise at ``snr_db``.

    Frequencies uniform in [-pi, pi), amplitudes uniform in [0.1, 1], phases
    uniform in [0, 2 pi). The noise variance is set from the empirical signal
    power. Returns the matrix and the drawn parameters.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    om = rng.uniform(-np.pi, np.pi, n_exp)
    nu = rng.uniform(-np.pi, np.pi, n_exp)
    amp = rng.uniform(0.1, 1.0, n_exp)
    phi = rng.uniform(0.0, 2 * np.pi, n_exp)
    n = np.arange(N)[:, None]
    m = np.arange(M)[None, :]
    s = np.zeros((N, M), np.complex128)
    for k in range(n_exp):
        s += amp[k] * np.exp(1j * (om[k] * n + nu[k] * m + phi[k]))
    p_sig = float(np.mean(np.abs(s) ** 2))
    sigma2 = p_sig / (10.0 ** (snr_db / 10.0))
    w = rng.standard_normal((N, M, 2)) * np.sqrt(sigma2 / 2.0)
    a = s + (w[..., 0] + 1j * w[..., 1])
    params = dict(omega=om, nu=nu, amp=amp, phi=phi, sigma2=sigma2)
    return a.astype(_CDTYPE[dtype]), params


def single_exponential(N: int, M: int, c: complex, omega: float, nu: float,
                       dtype: str = "c128") -> np.ndarray:
    """A[n, m] = c * exp(i (omega n + nu m))."""
    n = np.arange(N)[:, None]
    m = np.arange(M)[None, :]
    return (c * np.exp(1j * (omega * n + nu * m))).astype(_CDTYPE[dtype])


def workload_input(w: Workload, index: int = 0) -> np.ndarray:
    """The input matrix of workload ``w`` (``index`` selects a batch member)."""
    seed = w.seed + index
    if w.kind == "cn":
        return complex_normal((w.N, w.M), seed, w.dtype)
    if w.kind == "int":
        return integer_valued((w.N, w.M), seed, dtype=w.dtype)
    if w.kind == "sar":
        return sar_like(w.N, w.M, seed, dtype=w.dtype)[0]
    raise ValueError(w.kind)


def batched_shapes(count: int = BATCHED_COUNT, seed: int = BATCHED_SEED,
                   nm_range=(32, 256), pq_range=(2, 16)) -> List[Tuple[int, int, int, int]]:
    """(N, M, P, Q) per batch member: N, M uniform in nm_range and P, Q uniform
    in pq_range, each capped at half of N (resp. M)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        N = int(rng.integers(nm_range[0], nm_range[1] + 1))
        M = int(rng.integers(nm_range[0], nm_range[1] + 1))
        P = int(rng.integers(pq_range[0], pq_range[1] + 1))
        Q = int(rng.integers(pq_range[0], pq_range[1] + 1))
        out.append((N, M, min(P, N // 2), min(Q, M // 2)))
    return out


def batched_inputs(shapes, seed: int = BATCHED_SEED, dtype: str = "c64") -> List[np.ndarray]:
    """One CN(0,1) matrix per shape, member k drawn from seed (seed * 100003 + k)."""
    return [complex_normal((N, M), seed * 100003 + k, dtype)
            for k, (N, M, _, _) in enumerate(shapes)]
