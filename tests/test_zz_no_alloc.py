"""cov_estimate_noalloc: the entry point for callers that must not allocate
device memory during a call (for example a plugin whose host application's
memory pool already owns the device memory, or a real-time processing loop
with a device-memory budget fixed at start-up). Its scratch space is a static
device array inside the library.

Checked through the C ABI: two calls in a row give the same R as
cov_estimate_ex (the entry point with a caller workspace) within the
tolerances of the other parity tests, and a problem larger than the static
array is rejected before any work is queued. This file is collected last so a
run that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

import cov_workloads as wl
import paper_1303_2285_gb300 as cov

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5
F64_TOL = 1e-12
COV_EWORKSPACE = 3

CASES = [
    (1024, 1024, 16, 16, "c64"),   # the bench workload
    (100, 70, 8, 3, "c64"),
    (64, 64, 8, 8, "c128"),
    (300, 101, 12, 12, "c128"),
]


def _stream():
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("N,M,P,Q,dt", CASES)
def test_noalloc_matches_workspace_entry_point(N, M, P, Q, dt):
    lib = cov.load()
    tdt = torch.complex64 if dt == "c64" else torch.complex128
    A_np = wl.complex_normal((N, M), 7 * N + M, dtype=dt)
    A = torch.from_numpy(A_np).cuda()
    D = P * Q
    dtype_code = cov.DTYPES[dt]
    # existing entry point with a caller-provided workspace
    ws = torch.empty(cov.workspace_size(dt, N, M, P, Q, "recurrence"), dtype=torch.uint8, device="cuda")
    R_ref = torch.empty((D, D), dtype=tdt, device="cuda")
    assert lib.cov_estimate_ex(A.data_ptr(), dtype_code, N, M, M, P, Q, R_ref.data_ptr(),
                               cov.ALGOS["recurrence"], cov.NORMS["mean"], ws.data_ptr(),
                               ws.numel(), _stream()) == 0
    ref = R_ref.cpu().numpy()
    tol = F32_TOL if dt == "c64" else F64_TOL
    for _ in range(2):  # two calls in a row share the static scratch
        R = torch.full((D, D), complex(np.nan, np.nan), dtype=tdt, device="cuda")
        code = lib.cov_estimate_noalloc(A.data_ptr(), dtype_code, N, M, M, P, Q, R.data_ptr(),
                                        cov.NORMS["mean"], _stream())
        assert code == 0, cov.STATUS.get(code, code)
        got = R.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol


def test_noalloc_rejects_problems_beyond_the_static_scratch():
    lib = cov.load()
    N, M, P, Q = 2048, 512, 32, 32
    assert cov.workspace_size("c64", N, M, P, Q, "recurrence") > 16 << 20
    A = torch.zeros((N, M), dtype=torch.complex64, device="cuda")
    R = torch.zeros((P * Q, P * Q), dtype=torch.complex64, device="cuda")
    code = lib.cov_estimate_noalloc(A.data_ptr(), 0, N, M, M, P, Q, R.data_ptr(), 0, _stream())
    assert code == COV_EWORKSPACE
    torch.cuda.synchronize()
    assert bool((R == 0).all())  # nothing was queued
