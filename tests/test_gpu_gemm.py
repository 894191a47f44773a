"""Parity of the dense contraction form (R = X X^H on tcgen05 tensor cores,
TF32 hi/lo or BF16 hi/mid/lo split products, FP32 accumulation, split-K)
with the CPU oracle."""
import numpy as np
import pytest
import torch

import cov_workloads as wl
import paper_1303_2285_gb300 as cov

pytestmark = pytest.mark.gpu

from gpu_util import guarded, oracle_R, rel_fro, to_dev  # noqa: E402

F32_TOL = 1e-5


def run_gemm(A_np, P, Q, norm="mean", algo="gemm_tf32x3"):
    A = to_dev(A_np, torch.complex64)
    D = P * Q
    R, check = guarded((D, D), torch.complex64)
    n = cov.workspace_size("c64", *A_np.shape, P, Q, algo)
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    cov.estimate_into(A, R, P, Q, algo=algo, norm=norm, workspace=ws)
    torch.cuda.synchronize()
    cov.check_device_status(ws)
    check()
    return R.cpu().numpy()


@pytest.mark.parametrize("algo", ["gemm_tf32x3", "gemm_bf16x3"])
@pytest.mark.parametrize("N,M,P,Q", [(20, 20, 4, 4), (64, 64, 8, 8), (100, 70, 8, 12),
                                     (130, 200, 16, 16), (95, 95, 32, 32), (300, 41, 3, 2),
                                     (9, 9, 9, 9), (40, 1, 7, 1)])
def test_gemm_gaussian(oracle_mod, N, M, P, Q, algo):
    A = wl.complex_normal((N, M), 77 + N + M, dtype="c64")
    got = run_gemm(A, P, Q, algo=algo)
    want = oracle_R(oracle_mod, A, P, Q)
    assert rel_fro(got, want) < F32_TOL
    assert np.array_equal(got, got.conj().T)
    assert np.all(got.diagonal().imag == 0)


@pytest.mark.parametrize("algo", ["gemm_tf32x3", "gemm_bf16x3"])
def test_gemm_sum_mode_integer(oracle_mod, algo):
    # small integers: hi holds them exactly, every partial sum is exact in FP32
    A = wl.integer_valued((40, 33), 9, dtype="c64")
    got = run_gemm(A, 6, 5, norm="sum", algo=algo)
    want = oracle_R(oracle_mod, A, 6, 5, mean=False)
    assert np.array_equal(got, want.astype(np.complex64))
