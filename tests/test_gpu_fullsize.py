"""Parity at the workloads' full sizes, in the launch configuration the bench
times (knobs autotuned first), on sampled outputs the oracle computes one by
one, plus properties that hold at any size: R exactly Hermitian with a real
diagonal. Also the largest inputs of the suite (4096 x 4096) and a sample of
the 4096-member batched workload."""
import numpy as np
import pytest
import torch

import cov_workloads as wl
import paper_1303_2285_gb300 as cov

pytestmark = pytest.mark.gpu

from gpu_util import oracle_R, rel_fro, to_dev  # noqa: E402


def sample_pairs(D, n, seed):
    rng = np.random.default_rng(seed)
    fixed = [(0, 0), (0, D - 1), (D - 1, 0), (D - 1, D - 1), (D // 2, D // 2), (1, 0)]
    rand = [tuple(int(x) for x in rng.integers(0, D, 2)) for _ in range(n)]
    return fixed + rand


def check_sampled(oracle_mod, A_np, R, P, Q, pairs, tol):
    A128 = np.ascontiguousarray(A_np.astype(np.complex128))
    scale = np.abs(R).max()
    for a, b in pairs:
        want = oracle_mod.cov_element(A128, P, Q, a, b)
        assert abs(R[a, b] - want) <= tol * scale, (a, b, R[a, b], want)
    assert np.array_equal(R, R.conj().T)
    assert np.all(R.diagonal().imag == 0)


@pytest.mark.parametrize("name,tol", [("cn_1024x1024_w16_f32", 1e-5), ("sar_2048x512_w32_f32", 1e-5),
                                      ("plain_64x64_w8_f64", 1e-12)])
def test_workload_full_size_sampled(oracle_mod, name, tol):
    w = wl.WORKLOADS[name]
    dt = torch.complex64 if w.dtype == "c64" else torch.complex128
    A_np = wl.workload_input(w)
    A = to_dev(A_np, dt)
    cov.tuning_clear()
    try:
        cov.autotune(A, w.P, w.Q, reps=2)
        R = cov.estimate(A, w.P, w.Q, algo="recurrence")
        torch.cuda.synchronize()
    finally:
        cov.tuning_clear()
    check_sampled(oracle_mod, A_np, R.cpu().numpy(), w.P, w.Q, sample_pairs(w.P * w.Q, 40, 7), tol)


@pytest.mark.parametrize("kernels", [1, 4])
def test_largest_input_sampled(oracle_mod, kernels):
    N = M = 4096
    P = Q = 8
    A_np = wl.complex_normal((N, M), 2024, dtype="c64")
    cov.tuning_set("c64", N, M, P, Q, {"lag_group": 8, "rows_per_task": 128, "reseed_interval": 8,
                                       "kernels": kernels})
    try:
        R = cov.estimate(to_dev(A_np, torch.complex64), P, Q, algo="recurrence")
        torch.cuda.synchronize()
    finally:
        cov.tuning_clear()
    check_sampled(oracle_mod, A_np, R.cpu().numpy(), P, Q, sample_pairs(P * Q, 12, 8), 1e-5)


def test_batched_workload_sampled_members(oracle_mod):
    shapes = wl.batched_shapes()
    items, host = [], []
    for k, (N, M, P, Q) in enumerate(shapes):
        A = wl.complex_normal((N, M), wl.BATCHED_SEED * 100003 + k, "c64")
        items.append((torch.from_numpy(A).cuda(),
                      torch.empty((P * Q, P * Q), dtype=torch.complex64, device="cuda"), P, Q))
        host.append(A)
    plan = cov.BatchedPlan(items)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.upload(ws)
    plan.run(ws)
    torch.cuda.synchronize()
    cov.check_device_status(ws)
    rng = np.random.default_rng(11)
    for k in rng.choice(len(shapes), 8, replace=False):
        N, M, P, Q = shapes[k]
        got = items[k][1].cpu().numpy()
        assert rel_fro(got, oracle_R(oracle_mod, host[k], P, Q)) < 1e-5, shapes[k]
