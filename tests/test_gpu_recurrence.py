"""Parity of the CUDA combination path (and the plain FP64 direct path) with
the CPU oracle, through the C ABI.

Bars: FP64 results are bit-identical to the oracle on small-integer inputs
(every partial sum is an exact integer, so every summation order gives the
same value) and within 1e-12 relative Frobenius on Gaussian inputs; FP32
results are within 1e-5 relative Frobenius error of the FP64 oracle and
exact on small-integer inputs whose sums stay below 2^24.
"""
import numpy as np
import pytest
import torch

import cov_workloads as wl
import paper_1303_2285_gb300 as cov

pytestmark = pytest.mark.gpu

from gpu_util import guarded, oracle_R, rel_fro, to_dev  # noqa: E402

F32_TOL = 1e-5
F64_TOL = 1e-12

# shapes spanning several tiles, ragged row / column tails, the smallest
# shapes the path takes (N = 2P-1, M = 2Q-1) and P or Q equal to 1
SHAPES = [
    (64, 64, 8, 8), (37, 45, 5, 7), (100, 70, 8, 3), (20, 300, 4, 9), (15, 9, 8, 5),
    (33, 65, 1, 6), (40, 17, 7, 1), (1, 1, 1, 1), (130, 200, 16, 16), (77, 129, 12, 12),
    (300, 101, 2, 2), (95, 95, 32, 32), (63, 70, 32, 3),
]

# shapes without inner rows (N < 2P-1) or inner columns (M < 2Q-1), or both:
# every row / column is a fringe one. N = 2P-2 and M = 2Q-2 keep the scan
# form of the column sums with no inner column; below that the window form;
# a single window (N = P, M = Q); wide and tall ones put every product in the
# fringe-row kernel or the product kernel's column sums.
SHORT_SHAPES = [
    (9, 9, 9, 9), (7, 30, 5, 3), (30, 7, 2, 6), (12, 12, 7, 7), (5, 5, 1, 5), (14, 16, 8, 9),
    (40, 40, 32, 32), (32, 32, 32, 32), (40, 3000, 32, 4), (3000, 40, 4, 32), (62, 600, 32, 20),
    (5, 200, 3, 2), (200, 5, 2, 3), (1, 40, 1, 32),
]


def run(A_np, P, Q, dtype, algo="recurrence", norm="mean"):
    A = to_dev(A_np, dtype)
    D = P * Q
    R, check = guarded((D, D), dtype)
    ws_n = cov.workspace_size("c64" if dtype == torch.complex64 else "c128", *A_np.shape, P, Q, algo)
    ws = torch.empty(ws_n + 512, dtype=torch.uint8, device="cuda")
    cov.estimate_into(A, R, P, Q, algo=algo, norm=norm, workspace=ws[:ws_n] if ws_n else ws)
    torch.cuda.synchronize()
    cov.check_device_status(ws)
    check()
    return R.cpu().numpy()


@pytest.mark.parametrize("N,M,P,Q", SHAPES + SHORT_SHAPES)
def test_f64_integer_bit_exact(oracle_mod, N, M, P, Q):
    A = wl.integer_valued((N, M), 2285 + N + 7 * M)
    for norm in ("mean", "sum"):
        got = run(A, P, Q, torch.complex128, norm=norm)
        want = oracle_R(oracle_mod, A, P, Q, mean=(norm == "mean"))
        assert np.array_equal(got, want), f"max diff {np.abs(got - want).max()}"


@pytest.mark.parametrize("N,M,P,Q", SHAPES + SHORT_SHAPES)
def test_f64_gaussian(oracle_mod, N, M, P, Q):
    A = wl.complex_normal((N, M), 1303 + N + M)
    got = run(A, P, Q, torch.complex128)
    want = oracle_R(oracle_mod, A, P, Q)
    assert rel_fro(got, want) < F64_TOL
    assert np.array_equal(got, got.conj().T)
    assert np.all(got.diagonal().imag == 0)


@pytest.mark.parametrize("N,M,P,Q", SHAPES + SHORT_SHAPES)
def test_f32_gaussian(oracle_mod, N, M, P, Q):
    A = wl.complex_normal((N, M), 1 + N * M, dtype="c64")
    got = run(A, P, Q, torch.complex64)
    want = oracle_R(oracle_mod, A.astype(np.complex128), P, Q)
    assert rel_fro(got, want) < F32_TOL
    assert np.array_equal(got, got.conj().T)
    assert np.all(got.diagonal().imag == 0)


@pytest.mark.parametrize("N,M,P,Q", [(64, 64, 8, 8), (37, 45, 5, 7), (95, 95, 32, 32), (130, 200, 16, 16)])
def test_f32_integer_exact(oracle_mod, N, M, P, Q):
    # |products| <= 128 and K * 128 < 2^24: every FP32 partial sum is exact.
    A = wl.integer_valued((N, M), 99 + N, dtype="c64")
    K = (N - P + 1) * (M - Q + 1)
    assert K * 256 < 2 ** 24
    S = oracle_R(oracle_mod, A.astype(np.complex128), P, Q, mean=False)
    assert np.array_equal(run(A, P, Q, torch.complex64, norm="sum"), S.astype(np.complex64))
    want = (S.real.astype(np.float32) / np.float32(K)) + 1j * (S.imag.astype(np.float32) / np.float32(K))
    assert np.array_equal(run(A, P, Q, torch.complex64, norm="mean"), want.astype(np.complex64))


@pytest.mark.parametrize("N,M,P,Q", [(9, 9, 9, 9), (7, 30, 5, 3), (30, 7, 2, 6), (12, 12, 7, 7),
                                     (5, 5, 1, 5)])
def test_auto_takes_the_combination_path_without_inner_rows_or_columns(oracle_mod, N, M, P, Q):
    assert cov.plan_info(N, M, P, Q)["recurrence_ok"] == 1
    A = wl.integer_valued((N, M), 5 + N)
    got = run(A, P, Q, torch.complex128, algo="auto")
    assert np.array_equal(got, run(A, P, Q, torch.complex128, algo="recurrence"))
    assert np.array_equal(got, oracle_R(oracle_mod, A, P, Q))
    A32 = wl.complex_normal((N, M), 6 + N, dtype="c64")
    got = run(A32, P, Q, torch.complex64, algo="auto")
    assert rel_fro(got, oracle_R(oracle_mod, A32.astype(np.complex128), P, Q)) < 1e-6


@pytest.mark.parametrize("N,M,P,Q", [(12, 40, 7, 5), (20, 20, 16, 6), (62, 600, 32, 20)])
@pytest.mark.parametrize("kernels", [1, 4])
def test_short_rows_fused_and_four_kernels(oracle_mod, N, M, P, Q, kernels):
    # N < 2P - 1 with inner columns: the fused kernel takes it (no product
    # tasks), as do the four kernels; both exact on integers
    key = ("c64", N, M, P, Q)
    cov.tuning_set(*key, {"lag_group": 8, "rows_per_task": 16, "reseed_interval": 4,
                          "kernels": kernels})
    try:
        A = wl.integer_valued((N, M), 41 + M)
        K = (N - P + 1) * (M - Q + 1)
        assert K * 256 < 2 ** 24
        S = oracle_R(oracle_mod, A, P, Q, mean=False)
        assert np.array_equal(run(A.astype(np.complex64), P, Q, torch.complex64, norm="sum"),
                              S.astype(np.complex64))
    finally:
        cov.tuning_set(*key, None)


@pytest.mark.parametrize("N,M,P,Q", [(64, 64, 8, 8), (31, 17, 4, 6)])
def test_direct_f64(oracle_mod, N, M, P, Q):
    A = wl.integer_valued((N, M), 17 + M)
    assert np.array_equal(run(A, P, Q, torch.complex128, algo="direct"), oracle_R(oracle_mod, A, P, Q))
    A = wl.complex_normal((N, M), 18 + M)
    assert rel_fro(run(A, P, Q, torch.complex128, algo="direct"), oracle_R(oracle_mod, A, P, Q)) < 1e-14


def test_leading_dimension(oracle_mod):
    N, M, P, Q = 50, 40, 6, 5
    big = wl.complex_normal((N, M + 13), 4)
    A = to_dev(big, torch.complex128)[:, 3:3 + M]
    assert A.stride(0) == M + 13
    R = cov.estimate(A, P, Q, algo="recurrence")
    want = oracle_R(oracle_mod, big[:, 3:3 + M], P, Q)
    assert rel_fro(R.cpu().numpy(), want) < F64_TOL


def test_convenience_entry_point(oracle_mod):
    A_np = wl.complex_normal((40, 40), 8, dtype="c64")
    A = to_dev(A_np, torch.complex64)
    R = torch.empty((36, 36), dtype=torch.complex64, device="cuda")
    lib = cov.load()
    code = lib.cov_estimate(A.data_ptr(), 0, 40, 40, 6, 6, R.data_ptr(),
                            torch.cuda.current_stream().cuda_stream)
    assert code == 0
    torch.cuda.synchronize()
    assert rel_fro(R.cpu().numpy(), oracle_R(oracle_mod, A_np.astype(np.complex128), 6, 6)) < F32_TOL


def test_workspace_errors():
    A = torch.zeros((64, 64), dtype=torch.complex64, device="cuda")
    R = torch.empty((64, 64), dtype=torch.complex64, device="cuda")
    small = torch.empty(512, dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError):
        cov.estimate_into(A, R, 8, 8, algo="recurrence", workspace=small)
    lib = cov.load()
    s = torch.cuda.current_stream().cuda_stream
    code = lib.cov_estimate_ex(A.data_ptr(), 0, 64, 64, 64, 8, 8, R.data_ptr(), 1, 0,
                               small.data_ptr(), small.numel(), s)
    assert code == 3  # COV_EWORKSPACE
    code = lib.cov_estimate_ex(A.data_ptr(), 0, 64, 64, 64, 8, 8, R.data_ptr(), 1, 0,
                               small.data_ptr() + 8, 1 << 30, s)
    assert code == 3  # misaligned


def test_repeated_calls_reuse_workspace(oracle_mod):
    A_np = wl.complex_normal((70, 80), 9, dtype="c64")
    A = to_dev(A_np, torch.complex64)
    ws = torch.full((cov.workspace_size("c64", 70, 80, 9, 9),), 0xAB, dtype=torch.uint8, device="cuda")
    r1 = cov.estimate(A, 9, 9, workspace=ws).cpu().numpy()
    r2 = cov.estimate(A, 9, 9, workspace=ws).cpu().numpy()
    assert np.array_equal(r1, r2)
