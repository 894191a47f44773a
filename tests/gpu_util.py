"""Helpers for the GPU tests: device tensors with guard bands (canaries) in
place of a memory checker, and comparisons against the oracle."""
import numpy as np
import torch

CANARY = 64  # complex elements of guard band on each side


def guarded(shape, dtype, fill=np.nan):
    """A CUDA tensor view of `shape` inside a larger buffer whose borders hold
    a known pattern; `check()` verifies the borders are untouched."""
    n = int(np.prod(shape))
    base = torch.empty(n + 2 * CANARY, dtype=dtype, device="cuda")
    pat = complex(fill, -7.25) if dtype.is_complex else fill
    base.fill_(pat)
    view = base[CANARY:CANARY + n].view(*shape)

    def check():
        lo = base[:CANARY].cpu().numpy()
        hi = base[CANARY + n:].cpu().numpy()
        for band in (lo, hi):
            ok = np.all(np.isnan(band.real)) & np.all(band.imag == -7.25)
            assert ok, "guard band overwritten"
    return view, check


def to_dev(A, dtype):
    return torch.from_numpy(np.ascontiguousarray(A)).to(device="cuda", dtype=dtype)


def rel_fro(X, Y):
    return float(np.linalg.norm(X - Y) / max(np.linalg.norm(Y), 1e-300))


def oracle_R(oracle_mod, A, P, Q, mean=True):
    """The oracle's estimate, using every host core (bit-identical to one)."""
    import os
    return oracle_mod.cov_window(np.asarray(A, np.complex128), P, Q, mean=mean,
                                 threads=os.cpu_count() or 1)
