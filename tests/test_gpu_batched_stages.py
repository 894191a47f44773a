"""Parity of the batched plan's stage form (form 3: the single-matrix stages,
each one launch over all members) with the CPU oracle, through the C ABI:
complex64 within 1e-5 relative Frobenius and exact on small integers;
complex128 bit-identical on small integers and within 1e-12 on Gaussian
inputs; members beyond the other forms' limits (P or Q up to 32, no inner
rows or columns, M above 512); CUDA-graph capture."""
import numpy as np
import pytest
import torch

import cov_workloads as wl
import paper_1303_2285_gb300 as cov

pytestmark = pytest.mark.gpu

from gpu_util import oracle_R, rel_fro  # noqa: E402

F32_TOL = 1e-5
F64_TOL = 1e-12


def random_shapes(count, seed, nm=(8, 90), pq_max=16, short=False):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        N, M = (int(x) for x in rng.integers(nm[0], nm[1] + 1, 2))
        cap_p = N if short else (N + 1) // 2
        cap_q = M if short else (M + 1) // 2
        P = int(rng.integers(1, min(pq_max, cap_p) + 1))
        Q = int(rng.integers(1, min(pq_max, cap_q) + 1))
        out.append((N, M, P, Q))
    return out


def make_batch(shapes, kind, seed, dtype=torch.complex64):
    items, host = [], []
    np_dt = "c64" if dtype == torch.complex64 else "c128"
    for k, (N, M, P, Q) in enumerate(shapes):
        if kind == "int":
            A = wl.integer_valued((N, M), seed + k, dtype=np_dt)
        else:
            A = wl.complex_normal((N, M), seed + k, dtype=np_dt)
        At = torch.from_numpy(A).cuda()
        Rt = torch.full((P * Q, P * Q), complex(np.nan, np.nan), dtype=dtype, device="cuda")
        items.append((At, Rt, P, Q))
        host.append(A)
    return items, host


def run_stages(items, norm="mean"):
    plan = cov.BatchedPlan(items, norm=norm)
    plan.set_tuning(3)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.upload(ws)
    plan.run(ws)
    torch.cuda.synchronize()
    cov.check_device_status(ws)
    assert plan.tuning["form"] == 3
    return plan, ws


def test_stages_gaussian(oracle_mod):
    shapes = random_shapes(40, 11) + [(256, 256, 16, 16), (31, 200, 16, 2), (200, 33, 3, 16),
                                      (32, 32, 16, 16), (5, 9, 1, 1), (144, 150, 9, 9)]
    items, host = make_batch(shapes, "cn", 700)
    run_stages(items)
    for (At, Rt, P, Q), A in zip(items, host):
        got = Rt.cpu().numpy()
        want = oracle_R(oracle_mod, A.astype(np.complex128), P, Q)
        assert rel_fro(got, want) < F32_TOL, (A.shape, P, Q)
        assert np.array_equal(got, got.conj().T)
        assert np.all(got.diagonal().imag == 0)


def test_stages_integer_exact(oracle_mod):
    shapes = random_shapes(30, 12, nm=(8, 60))
    items, host = make_batch(shapes, "int", 800)
    run_stages(items, norm="sum")
    for (At, Rt, P, Q), A in zip(items, host):
        S = oracle_R(oracle_mod, A.astype(np.complex128), P, Q, mean=False)
        assert np.array_equal(Rt.cpu().numpy(), S.astype(np.complex64)), (A.shape, P, Q)


def test_stages_members_beyond_the_other_forms(oracle_mod):
    # P or Q above 16, no inner rows / columns, M above 512, a single window
    shapes = [(64, 64, 20, 4), (30, 40, 16, 3), (100, 600, 4, 4), (40, 40, 32, 32),
              (9, 9, 9, 9), (7, 30, 5, 3), (30, 7, 2, 6), (70, 1100, 3, 30), (32, 32, 32, 32),
              (12, 12, 7, 7)] + random_shapes(12, 13, nm=(4, 40), pq_max=32, short=True)
    items, host = make_batch(shapes, "int", 900)
    plan = cov.BatchedPlan(items, norm="sum")
    assert plan.tuning["form"] == 3  # the only form these members fit
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.upload(ws)
    plan.run(ws)
    torch.cuda.synchronize()
    cov.check_device_status(ws)
    for (At, Rt, P, Q), A in zip(items, host):
        N, M = A.shape
        S = oracle_R(oracle_mod, A.astype(np.complex128), P, Q, mean=False)
        if (N - P + 1) * (M - Q + 1) * 256 < 2 ** 24:  # every FP32 partial sum exact
            assert np.array_equal(Rt.cpu().numpy(), S.astype(np.complex64)), (N, M, P, Q)
        else:
            assert rel_fro(Rt.cpu().numpy(), S) < F32_TOL, (N, M, P, Q)


def test_stages_complex128_integer_bit_exact(oracle_mod):
    shapes = random_shapes(20, 14, nm=(4, 70), pq_max=32, short=True) + [
        (64, 64, 8, 8), (40, 40, 32, 32), (100, 300, 16, 3), (9, 9, 9, 9)]
    items, host = make_batch(shapes, "int", 1000, dtype=torch.complex128)
    for norm in ("mean", "sum"):
        plan = cov.BatchedPlan(items, norm=norm)
        assert plan.tuning["form"] == 3
        ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
        plan.upload(ws)
        plan.run(ws)
        torch.cuda.synchronize()
        cov.check_device_status(ws)
        for (At, Rt, P, Q), A in zip(items, host):
            want = oracle_R(oracle_mod, A, P, Q, mean=(norm == "mean"))
            assert np.array_equal(Rt.cpu().numpy(), want), (A.shape, P, Q, norm)


def test_stages_complex128_gaussian(oracle_mod):
    shapes = random_shapes(16, 15, nm=(8, 80)) + [(150, 140, 12, 10)]
    items, host = make_batch(shapes, "cn", 1100, dtype=torch.complex128)
    run_stages(items)
    for (At, Rt, P, Q), A in zip(items, host):
        assert rel_fro(Rt.cpu().numpy(), oracle_R(oracle_mod, A, P, Q)) < F64_TOL, (A.shape, P, Q)


def test_stages_graph_capture_and_repeat(oracle_mod):
    shapes = random_shapes(24, 16)
    items, host = make_batch(shapes, "cn", 1200)
    plan, ws = run_stages(items)
    first = [Rt.cpu().numpy().copy() for _, Rt, _, _ in items]
    for _, Rt, _, _ in items:
        Rt.fill_(complex(np.nan, np.nan))
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        plan.run(ws, stream=s)
    g.replay()
    torch.cuda.synchronize()
    cov.check_device_status(ws)
    for (At, Rt, P, Q), R0 in zip(items, first):
        assert np.array_equal(Rt.cpu().numpy(), R0)  # same plan, same kernels, same sums


def test_stages_agree_with_the_cta_form(oracle_mod):
    # both forms against the oracle on the same members, and with each other
    shapes = random_shapes(20, 17, nm=(16, 120))
    items, host = make_batch(shapes, "cn", 1300)
    plan = cov.BatchedPlan(items)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    out = {}
    for form in (0, 3):
        plan.set_tuning(form)
        plan.upload(ws)
        plan.run(ws)
        torch.cuda.synchronize()
        cov.check_device_status(ws)
        out[form] = [Rt.cpu().numpy().copy() for _, Rt, _, _ in items]
    for k, ((At, Rt, P, Q), A) in enumerate(zip(items, host)):
        want = oracle_R(oracle_mod, A.astype(np.complex128), P, Q)
        assert rel_fro(out[3][k], want) < F32_TOL and rel_fro(out[0][k], want) < F32_TOL
        assert rel_fro(out[3][k], out[0][k]) < 2 * F32_TOL


def test_autotune_considers_the_stage_form(oracle_mod):
    shapes = random_shapes(30, 18, nm=(40, 150))
    items, host = make_batch(shapes, "cn", 1400)
    plan = cov.BatchedPlan(items)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.upload(ws)
    best = plan.autotune(ws, reps=1)
    assert best["form"] in (0, 3)
    plan.run(ws)
    torch.cuda.synchronize()
    cov.check_device_status(ws)
    for (At, Rt, P, Q), A in zip(items, host):
        assert rel_fro(Rt.cpu().numpy(), oracle_R(oracle_mod, A.astype(np.complex128), P, Q)) < F32_TOL
