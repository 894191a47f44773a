"""Parity of the adjoint kernels (dL/dA) with the CPU oracle's gradient and
with FP64 finite differences of the oracle's loss, through the C ABI and the
torch.autograd.Function wrapper."""
import numpy as np
import pytest
import torch

import cov_workloads as wl
import paper_1303_2285_gb300 as cov

pytestmark = pytest.mark.gpu

from gpu_util import rel_fro  # noqa: E402

F32_TOL = 1e-5


SHAPES = [(20, 17, 4, 3), (16, 16, 4, 4), (37, 50, 7, 5), (9, 9, 9, 9), (30, 12, 1, 1),
          (64, 70, 12, 12), (47, 33, 24, 2), (100, 37, 3, 19), (11, 13, 6, 7)]


def _stencil_ok(N, M, P, Q):
    return N >= 2 * P - 1 and M >= 2 * Q - 1 and (2 * P - 1) * (2 * Q - 1) <= 2048


@pytest.mark.parametrize("N,M,P,Q", SHAPES)
@pytest.mark.parametrize("norm", ["mean", "sum"])
@pytest.mark.parametrize("form", ["dense", "stencil", "auto"])
def test_backward_matches_oracle(oracle_mod, N, M, P, Q, norm, form):
    if form == "stencil" and not _stencil_ok(N, M, P, Q):
        pytest.skip("the stencil form needs N >= 2P-1, M >= 2Q-1")
    A = wl.complex_normal((N, M), 11 + N, dtype="c64")
    G = wl.complex_normal((P * Q, P * Q), 12 + M, dtype="c64")
    dA = cov.estimate_backward(torch.from_numpy(A).cuda(), torch.from_numpy(G).cuda(), P, Q, norm=norm,
                               form=form)
    want = oracle_mod.cov_backward(A.astype(np.complex128), G.astype(np.complex128), P, Q,
                                   mean=(norm == "mean"))
    assert rel_fro(dA.cpu().numpy(), want) < F32_TOL


def test_stencil_form_refuses_small_shapes():
    with pytest.raises(cov.CovError) as e:
        cov.estimate_backward(torch.zeros((9, 9), dtype=torch.complex64, device="cuda"),
                              torch.zeros((81, 81), dtype=torch.complex64, device="cuda"), 9, 9,
                              form="stencil")
    assert e.value.code == 5


def test_autograd_against_fd_fp64(oracle_mod):
    # loss = ||R - T||_F^2 with T from a second seed; A 16x16, window 4x4
    N = M = 16
    P = Q = 4
    A = wl.complex_normal((N, M), 4, dtype="c128")
    T = oracle_mod.cov_window(wl.complex_normal((N, M), 5000, dtype="c128"), P, Q)
    At = torch.tensor(A.astype(np.complex64), device="cuda", requires_grad=True)
    Tt = torch.tensor(T.astype(np.complex64), device="cuda")
    R = cov.covariance(At, P, Q)
    loss = (R - Tt).abs().pow(2).sum()
    loss.backward()
    got = At.grad.cpu().numpy()

    def L(X):
        return float(np.sum(np.abs(oracle_mod.cov_window(X, P, Q) - T) ** 2))

    h = 1e-6
    fd = np.zeros((N, M), np.complex128)
    for n in range(N):
        for m in range(M):
            for unit in (1.0, 1j):
                E = np.zeros((N, M), np.complex128)
                E[n, m] = unit * h
                d = (L(A + E) - L(A - E)) / (2 * h)
                fd[n, m] += d * (1.0 if unit == 1.0 else 1j)
    assert rel_fro(got, fd) < 1e-5


def test_autograd_matches_oracle_gradient_workload_shape(oracle_mod):
    # one member of the differentiation workload: 256 x 256, window 12 x 12
    N = M = 256
    P = Q = 12
    A = wl.complex_normal((N, M), 4, dtype="c64")
    T = wl.complex_normal((N, M), 5000, dtype="c64")
    At = torch.tensor(A, device="cuda", requires_grad=True)
    with torch.no_grad():
        Tt = cov.estimate(torch.from_numpy(T).cuda(), P, Q)
    R = cov.covariance(At, P, Q)
    loss = (R - Tt).abs().pow(2).sum()
    loss.backward()
    G = 2.0 * (R.detach() - Tt).cpu().numpy().astype(np.complex128)
    want = oracle_mod.cov_backward(A.astype(np.complex128), G, P, Q)
    assert rel_fro(At.grad.cpu().numpy(), want) < F32_TOL


@pytest.mark.parametrize("B,N,M,P,Q", [(5, 40, 33, 5, 4), (3, 64, 70, 12, 12), (4, 11, 13, 6, 7)])
@pytest.mark.parametrize("norm", ["mean", "sum"])
def test_strided_batch_matches_oracle(oracle_mod, B, N, M, P, Q, norm):
    A = np.stack([wl.complex_normal((N, M), 50 + k, dtype="c64") for k in range(B)])
    G = np.stack([wl.complex_normal((P * Q, P * Q), 90 + k, dtype="c64") for k in range(B)])
    dA = cov.estimate_backward_batch(torch.from_numpy(A).cuda(), torch.from_numpy(G).cuda(), P, Q,
                                     norm=norm).cpu().numpy()
    for k in range(B):
        want = oracle_mod.cov_backward(A[k].astype(np.complex128), G[k].astype(np.complex128), P, Q,
                                       mean=(norm == "mean"))
        assert rel_fro(dA[k], want) < F32_TOL


# complex128: the dense form in FP64
@pytest.mark.parametrize("N,M,P,Q", [(20, 17, 4, 3), (9, 9, 9, 9), (37, 50, 7, 5), (30, 12, 1, 1),
                                     (64, 70, 12, 12), (11, 13, 6, 7)])
def test_backward_complex128_integer_exact_and_gaussian(oracle_mod, N, M, P, Q):
    # small integers, plain sum: every partial sum is an exact integer in FP64
    A = wl.integer_valued((N, M), 21 + N)
    G = wl.integer_valued((P * Q, P * Q), 22 + M)
    dA = cov.estimate_backward(torch.from_numpy(A).cuda(), torch.from_numpy(G).cuda(), P, Q,
                               norm="sum")
    assert dA.dtype == torch.complex128
    want = oracle_mod.cov_backward(A, G, P, Q, mean=False)
    assert np.array_equal(dA.cpu().numpy(), want)
    A = wl.complex_normal((N, M), 23 + N)
    G = wl.complex_normal((P * Q, P * Q), 24 + M)
    dA = cov.estimate_backward(torch.from_numpy(A).cuda(), torch.from_numpy(G).cuda(), P, Q)
    assert rel_fro(dA.cpu().numpy(), oracle_mod.cov_backward(A, G, P, Q)) < 1e-12


def test_backward_complex128_refuses_the_stencil_form():
    with pytest.raises(cov.CovError) as e:
        cov.estimate_backward(torch.zeros((40, 40), dtype=torch.complex128, device="cuda"),
                              torch.zeros((16, 16), dtype=torch.complex128, device="cuda"), 4, 4,
                              form="stencil")
    assert e.value.code == 5


def test_autograd_complex128_against_fd(oracle_mod):
    # the whole differentiable estimate in FP64: forward (combination path)
    # and adjoint (dense form), against central differences of the oracle's loss
    N = M = 12
    P = Q = 3
    A = wl.complex_normal((N, M), 31, dtype="c128")
    T = oracle_mod.cov_window(wl.complex_normal((N, M), 5001, dtype="c128"), P, Q)
    At = torch.tensor(A, device="cuda", requires_grad=True)
    R = cov.covariance(At, P, Q)
    loss = (R - torch.tensor(T, device="cuda")).abs().pow(2).sum()
    loss.backward()
    got = At.grad.cpu().numpy()

    def L(X):
        return float(np.sum(np.abs(oracle_mod.cov_window(X, P, Q) - T) ** 2))

    h = 1e-6
    fd = np.zeros((N, M), np.complex128)
    for n in range(N):
        for m in range(M):
            for unit in (1.0, 1j):
                E = np.zeros((N, M), np.complex128)
                E[n, m] = unit * h
                d = (L(A + E) - L(A - E)) / (2 * h)
                fd[n, m] += d * (1.0 if unit == 1.0 else 1j)
    assert rel_fro(got, fd) < 1e-7
