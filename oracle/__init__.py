"""CPU oracle for the sliding-window covariance method (arXiv 1303.2285).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The product library
(``paper_1303_2285_gb300``) never imports, links or runs anything here, and
this package imports nothing from it.

Contents
--------
* ``cov_window``    -- the plain definition, Eq. 2.1-2.2 averaged over all
                       window positions (C, FP64, no contraction).
* ``cov_element``   -- one element of the same, bit-identical to ``cov_window``.
* ``cov_backward``  -- the adjoint dL/dA of the estimate (C, FP64).
* ``combinations``  -- the counting and indexing of Section 3 and 4.
* ``algorithm1``    -- Algorithm 1 in the paper's own steps (pure Python).
* ``exact``         -- exact Gaussian-integer evaluation of Eq. 2.2.
* ``capon``         -- the minimum-variance (Capon) spectrum of an estimate
                       (the downstream use Section 2.3 cites), FP64.
* ``gram``          -- Eq. 2.2 as the Gram product X X^H of the window vectors
                       (BLAS zherk, FP64): the full-size reference where the
                       window loop would take minutes.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against a closed form, an invariant, a library routine or brute force; none
is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIBPATH = os.path.join(_LIBDIR, "libcov_oracle.so")
_SRC = os.path.join(_HERE, "cov_oracle.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (FP64, -ffp-contract=off, OpenMP)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIBPATH)
            and os.path.getmtime(_LIBPATH) >= os.path.getmtime(_SRC)):
        return _LIBPATH
    tmp = _LIBPATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-std=c11", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIBPATH)
    return _LIBPATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            L, I = ctypes.c_long, ctypes.c_int
            lib.cov_oracle_window.argtypes = [dp, L, L, L, I, I, I, I, dp]
            lib.cov_oracle_window.restype = I
            lib.cov_oracle_element.argtypes = [dp, L, L, L, I, I, I, L, L, dp]
            lib.cov_oracle_element.restype = I
            lib.cov_oracle_backward.argtypes = [dp, dp, L, L, L, I, I, I, dp]
            lib.cov_oracle_backward.restype = I
            lib.cov_oracle_max_threads.argtypes = []
            lib.cov_oracle_max_threads.restype = I
            _lib = lib
    return _lib


def _as_c128(A) -> np.ndarray:
    A = np.ascontiguousarray(np.asarray(A), dtype=np.complex128)
    if A.ndim != 2:
        raise ValueError("A must be 2-D")
    return A


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def max_threads() -> int:
    return int(_load().cov_oracle_max_threads())


def cov_window(A, P: int, Q: int, mean: bool = True, threads: int = 1) -> np.ndarray:
    """R = (1/K) sum_{p,q} x x^H (Eq. 2.1-2.2); ``mean=False`` gives the sum."""
    A = _as_c128(A)
    N, M = A.shape
    D = P * Q
    R = np.empty((D, D), np.complex128)
    rc = _load().cov_oracle_window(_ptr(A), N, M, M, P, Q, int(mean), int(threads), _ptr(R))
    if rc != 0:
        raise ValueError("cov_oracle_window: bad arguments")
    return R


def cov_element(A, P: int, Q: int, a: int, b: int, mean: bool = True) -> complex:
    """R[a, b] alone, bit-identical to ``cov_window(A, P, Q)[a, b]``."""
    A = _as_c128(A)
    N, M = A.shape
    out = np.zeros(2, np.float64)
    rc = _load().cov_oracle_element(_ptr(A), N, M, M, P, Q, int(mean), int(a), int(b), _ptr(out))
    if rc != 0:
        raise ValueError("cov_oracle_element: bad arguments")
    return complex(out[0], out[1])


def cov_backward(A, G, P: int, Q: int, mean: bool = True) -> np.ndarray:
    """dL/dA given G = dL/dR (both in the dRe + i dIm convention)."""
    A = _as_c128(A)
    G = np.ascontiguousarray(np.asarray(G), dtype=np.complex128)
    N, M = A.shape
    D = P * Q
    if G.shape != (D, D):
        raise ValueError("G must be PQ x PQ")
    dA = np.empty((N, M), np.complex128)
    rc = _load().cov_oracle_backward(_ptr(A), _ptr(G), N, M, M, P, Q, int(mean), _ptr(dA))
    if rc != 0:
        raise ValueError("cov_oracle_backward: bad arguments")
    return dA
