"""Minimum-variance (Capon) spectra of the estimates (the downstream use of R
that Section 2.3 cites) through the C ABI, against the FP64 oracle applied to
the same R.

Bar: the kernel factorises R + dI in FP32, so its relative error is bounded
by about cond(R + dI) x D x 2^-24 (backward-stable Cholesky and triangular
solve); each test computes the condition number in FP64 and checks the
largest relative error of the spectrum against 8 x cond x D x 2^-24."""
import numpy as np
import pytest
import torch

import cov_workloads as wl
import paper_1303_2285_gb300 as cov
from oracle.capon import capon_spectrum as oracle_capon, steering_vectors

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


def _bound(R64, loading):
    out = []
    for Rk in R64:
        D = Rk.shape[0]
        Rl = Rk + loading * np.trace(Rk).real / D * np.eye(D)
        out.append(8.0 * np.linalg.cond(Rl) * D * EPS32)
    return np.array(out)[:, None]


@pytest.mark.parametrize("P,Q,loading", [(10, 10, 0.01), (4, 3, 0.0), (8, 16, 0.05), (11, 11, 0.1)])
def test_capon_on_aperture_estimates(P, Q, loading):
    # estimates of apertures of one image (25 x 25, P x Q windows) as the input
    img = torch.from_numpy(wl.complex_normal((65, 90), 3 + P, dtype="c64")).cuda()
    ap = (max(25, 2 * P + 5), max(25, 2 * Q + 5))
    plan, R = cov.aperture_batch(img, ap, (10, 10), P, Q)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.upload(ws)
    plan.run(ws)
    torch.cuda.synchronize()
    rng = np.random.default_rng(P * Q)
    A = steering_vectors(P, Q, rng.uniform(-np.pi, np.pi, 70), rng.uniform(-np.pi, np.pi, 70))
    steer = torch.from_numpy(A.astype(np.complex64)).cuda()
    got = cov.capon_spectrum(R, steer, loading).cpu().numpy()
    R64 = R.cpu().numpy().astype(np.complex128)
    want = oracle_capon(R64, A.astype(np.complex64).astype(np.complex128), loading)
    rel = np.abs(got - want) / want
    assert np.all(np.isfinite(got)) and np.all(got > 0)
    assert np.all(rel <= _bound(R64, loading)), float(rel.max())


def test_capon_closed_form_white_noise():
    D, s2 = 36, 1.7
    R = torch.from_numpy((s2 * np.eye(D)).astype(np.complex64)).cuda().expand(5, D, D).contiguous()
    A = steering_vectors(6, 6, np.linspace(-3, 3, 40), np.linspace(3, -3, 40))
    got = cov.capon_spectrum(R, torch.from_numpy(A.astype(np.complex64)).cuda(), 0.0).cpu().numpy()
    assert np.allclose(got, s2 / D, rtol=1e-5)


def test_capon_not_positive_definite_gives_nan():
    D = 12
    v = np.ones(D, np.complex64)
    R = torch.from_numpy(np.stack([np.outer(v, v.conj()), np.eye(D, dtype=np.complex64)])).cuda()
    A = steering_vectors(3, 4, [0.1, 0.2], [0.3, -0.4])
    got = cov.capon_spectrum(R, torch.from_numpy(A.astype(np.complex64)).cuda(), 0.0).cpu().numpy()
    assert np.all(np.isnan(got[0]))          # rank one: a zero pivot
    assert np.allclose(got[1], 1.0 / D, rtol=1e-5)


def test_capon_rejects_bad_arguments():
    lib = cov.load()
    R = torch.zeros((2, 8, 8), dtype=torch.complex64, device="cuda")
    A = torch.zeros((3, 8), dtype=torch.complex64, device="cuda")
    out = torch.zeros((2, 3), dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert lib.cov_capon_spectrum(R.data_ptr(), 2, 129, A.data_ptr(), 3, 0.0, out.data_ptr(), s) == 1
    assert lib.cov_capon_spectrum(R.data_ptr(), 2, 8, A.data_ptr(), 3, -1.0, out.data_ptr(), s) == 1
    assert lib.cov_capon_spectrum(None, 2, 8, A.data_ptr(), 3, 0.0, out.data_ptr(), s) == 1
