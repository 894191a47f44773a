"""cov_estimate_noalloc: the entry point for callers that must not allocate
device memory during a call (for example a plugin whose host application's
memory pool already owns the device memory, or a real-time processing loop
with a device-memory budget fixed at start-up). Its scratch space is a static
device array inside the library.

Checked through the C ABI. cov_estimate_noalloc and cov_estimate_ex (the
entry point with a caller workspace) run the same plan and the same kernels,
so their results must agree bit for bit; every call runs twice in a row, and
the problems run from the largest to the smallest, so that later calls find
the shared scratch still holding an earlier, larger problem's partial sums
(a region the kernels fail to overwrite, or a counter they fail to clear,
would show). One case has lda > M. The static array's status word reads
COV_OK after normal calls, and a problem larger than the array is rejected
before any work is queued. This file is collected last so a run that stops
at the first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

import cov_workloads as wl
import paper_1303_2285_gb300 as cov

pytestmark = pytest.mark.gpu

COV_EWORKSPACE = 3

# (N, M, lda, P, Q, dtype), run from the largest scratch need to the smallest
CASES = [
    (1024, 1024, 1024, 16, 16, "c64"),   # the 1024 x 1024 workload
    (300, 101, 101, 12, 12, "c128"),
    (100, 70, 96, 8, 3, "c64"),          # lda > M
    (64, 64, 64, 8, 8, "c128"),
    (15, 9, 9, 8, 5, "c64"),
]


def _stream():
    return torch.cuda.current_stream().cuda_stream


def test_noalloc_matches_workspace_entry_point_bit_for_bit():
    lib = cov.load()
    cases = sorted(CASES, key=lambda c: -cov.workspace_size(c[5], c[0], c[1], c[3], c[4],
                                                            "recurrence"))
    for N, M, lda, P, Q, dt in cases:
        tdt = torch.complex64 if dt == "c64" else torch.complex128
        A_full = torch.from_numpy(wl.complex_normal((N, lda), 7 * N + M, dtype=dt)).cuda()
        A = A_full[:, :M]  # leading dimension lda
        D = P * Q
        dtype_code = cov.DTYPES[dt]
        ws = torch.empty(cov.workspace_size(dt, N, M, P, Q, "recurrence"), dtype=torch.uint8,
                         device="cuda")
        R_ref = torch.empty((D, D), dtype=tdt, device="cuda")
        assert lib.cov_estimate_ex(A.data_ptr(), dtype_code, N, M, lda, P, Q, R_ref.data_ptr(),
                                   cov.ALGOS["recurrence"], cov.NORMS["mean"], ws.data_ptr(),
                                   ws.numel(), _stream()) == 0
        ref = R_ref.cpu().numpy()
        assert np.all(np.isfinite(ref))
        for _ in range(2):  # two calls in a row share the static scratch
            R = torch.full((D, D), complex(np.nan, np.nan), dtype=tdt, device="cuda")
            code = lib.cov_estimate_noalloc(A.data_ptr(), dtype_code, N, M, lda, P, Q, R.data_ptr(),
                                            cov.NORMS["mean"], _stream())
            assert code == 0, cov.STATUS.get(code, code)
            assert lib.cov_noalloc_check_status(_stream()) == 0
            assert np.array_equal(R.cpu().numpy(), ref), (N, M, lda, P, Q, dt)


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
