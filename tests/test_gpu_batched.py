"""Parity of the batched persistent launch (many uneven matrices, one kernel)
with the CPU oracle, through the C ABI; and its capture in a CUDA graph."""
import numpy as np
import pytest
import torch

import cov_workloads as wl
import paper_1303_2285_gb300 as cov

pytestmark = pytest.mark.gpu

from gpu_util import oracle_R, rel_fro  # noqa: E402

F32_TOL = 1e-5


def random_shapes(count, seed, nm=(8, 70), pq_max=16):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        N, M = (int(x) for x in rng.integers(nm[0], nm[1] + 1, 2))
        P = int(rng.integers(1, min(pq_max, (N + 1) // 2) + 1))
        Q = int(rng.integers(1, min(pq_max, (M + 1) // 2) + 1))
        out.append((N, M, P, Q))
    return out


def make_batch(shapes, kind, seed):
    items, host = [], []
    for k, (N, M, P, Q) in enumerate(shapes):
        if kind == "int":
            A = wl.integer_valued((N, M), seed + k, dtype="c64")
        else:
            A = wl.complex_normal((N, M), seed + k, dtype="c64")
        At = torch.from_numpy(A).cuda()
        Rt = torch.full((P * Q, P * Q), complex(np.nan, np.nan), dtype=torch.complex64, device="cuda")
        items.append((At, Rt, P, Q))
        host.append(A)
    return items, host


def run_plan(items, norm="mean"):
    plan = cov.BatchedPlan(items, norm=norm)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.upload(ws)
    plan.run(ws)
    torch.cuda.synchronize()
    cov.check_device_status(ws)
    return plan, ws


def test_batched_gaussian(oracle_mod):
    shapes = random_shapes(40, 1) + [(256, 256, 16, 16), (31, 200, 16, 2), (200, 33, 3, 16),
                                     (32, 32, 16, 16), (5, 9, 1, 1)]
    items, host = make_batch(shapes, "cn", 100)
    run_plan(items)
    for (At, Rt, P, Q), A in zip(items, host):
        got = Rt.cpu().numpy()
        want = oracle_R(oracle_mod, A, P, Q)
        assert rel_fro(got, want) < F32_TOL, (A.shape, P, Q)
        assert np.array_equal(got, got.conj().T)


def test_batched_integer_exact(oracle_mod):
    shapes = random_shapes(25, 2, nm=(8, 60))
    items, host = make_batch(shapes, "int", 300)
    run_plan(items, norm="sum")
    for (At, Rt, P, Q), A in zip(items, host):
        N, M = A.shape
        S = oracle_R(oracle_mod, A, P, Q, mean=False)
        assert np.array_equal(Rt.cpu().numpy(), S.astype(np.complex64)), (N, M, P, Q)


def test_batched_graph_capture(oracle_mod):
    shapes = random_shapes(16, 3)
    items, host = make_batch(shapes, "cn", 500)
    plan = cov.BatchedPlan(items)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.upload(ws)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.run(ws, stream=s)
    for _ in range(2):
        for _, Rt, _, _ in items:
            Rt.fill_(complex(np.nan, np.nan))
        g.replay()
        torch.cuda.synchronize()
        for (At, Rt, P, Q), A in zip(items, host):
            assert rel_fro(Rt.cpu().numpy(), oracle_R(oracle_mod, A, P, Q)) < F32_TOL


def narrow_shapes(count, seed):
    """Members with M <= 32, N M <= 1024 and P, Q <= 16: the batch then runs
    one warp per member."""
    rng = np.random.default_rng(seed)
    out = [(31, 32, 16, 16), (33, 31, 3, 16), (9, 1, 5, 1), (1, 1, 1, 1), (25, 25, 10, 10),
           (64, 2, 7, 1), (17, 32, 9, 2)]
    while len(out) < count:
        N, M = int(rng.integers(1, 81)), int(rng.integers(1, 33))
        if N * M > 1024:
            continue
        P = int(rng.integers(1, min(16, (N + 1) // 2) + 1))
        Q = int(rng.integers(1, min(16, (M + 1) // 2) + 1))
        out.append((N, M, P, Q))
    return out


def test_batched_narrow_members_gaussian(oracle_mod):
    shapes = narrow_shapes(60, 21)
    assert all(M <= 32 and N * M <= 1024 and P <= 16 and Q <= 16 for N, M, P, Q in shapes)
    items, host = make_batch(shapes, "cn", 700)
    run_plan(items)
    for (At, Rt, P, Q), A in zip(items, host):
        got = Rt.cpu().numpy()
        assert rel_fro(got, oracle_R(oracle_mod, A, P, Q)) < F32_TOL, (A.shape, P, Q)
        assert np.array_equal(got, got.conj().T)
        assert np.all(got.diagonal().imag == 0)


def test_batched_narrow_members_integer_exact(oracle_mod):
    # small integers: every product, column sum, scan prefix and difference is
    # an exact integer in FP32, so the SUM result is exact
    shapes = narrow_shapes(30, 22)
    items, host = make_batch(shapes, "int", 900)
    run_plan(items, norm="sum")
    for (At, Rt, P, Q), A in zip(items, host):
        S = oracle_R(oracle_mod, A, P, Q, mean=False)
        assert np.array_equal(Rt.cpu().numpy(), S.astype(np.complex64)), (A.shape, P, Q)


@pytest.mark.parametrize("L,rs", [(0, 1), (1, 4), (3, 2), (16, 4), (2, 1)])
def test_batched_cta_form_knobs(oracle_mod, L, rs):
    shapes = random_shapes(24, 31) + [(256, 200, 16, 16), (40, 33, 16, 3)]
    items, host = make_batch(shapes, "cn", 1100)
    plan = cov.BatchedPlan(items)
    plan.set_tuning(0, L, rs)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.upload(ws)
    plan.run(ws)
    torch.cuda.synchronize()
    cov.check_device_status(ws)
    for (At, Rt, P, Q), A in zip(items, host):
        got = Rt.cpu().numpy()
        assert rel_fro(got, oracle_R(oracle_mod, A, P, Q)) < F32_TOL, (A.shape, P, Q, L, rs)
        assert np.array_equal(got, got.conj().T)


def test_batched_narrow_both_forms_and_autotune(oracle_mod):
    shapes = narrow_shapes(40, 41)
    items, host = make_batch(shapes, "cn", 1300)
    plan = cov.BatchedPlan(items)
    assert plan.tuning["form"] == 1
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    for form, L in [(1, 0), (0, 0), (0, 4), (3, 0)]:
        plan.set_tuning(form, L, 4)
        plan.upload(ws)
        for _, Rt, _, _ in items:
            Rt.fill_(complex(np.nan, np.nan))
        plan.run(ws)
        torch.cuda.synchronize()
        cov.check_device_status(ws)
        for (At, Rt, P, Q), A in zip(items, host):
            assert rel_fro(Rt.cpu().numpy(), oracle_R(oracle_mod, A, P, Q)) < F32_TOL, (form, L)
    best = plan.autotune(ws, reps=2)
    assert best["form"] in (0, 1, 3) and best["row_ranges"] in (2, 4)
    for _, Rt, _, _ in items:
        Rt.fill_(complex(np.nan, np.nan))
    plan.run(ws)
    torch.cuda.synchronize()
    cov.check_device_status(ws)
    for (At, Rt, P, Q), A in zip(items, host):
        assert rel_fro(Rt.cpu().numpy(), oracle_R(oracle_mod, A, P, Q)) < F32_TOL


def box_shapes(count, seed):
    """Members the box form takes (M <= 32, N M <= 1024, P, Q <= 16,
    PQ <= 100), including the smallest and the widest windows."""
    rng = np.random.default_rng(seed)
    out = [(25, 25, 10, 10), (19, 32, 10, 10), (31, 32, 16, 6), (33, 31, 6, 16), (9, 1, 5, 1),
           (1, 1, 1, 1), (64, 2, 7, 1), (21, 17, 11, 9), (8, 32, 1, 16), (40, 25, 20, 5)]
    out = [s for s in out if s[2] <= 16 and s[3] <= 16]
    while len(out) < count:
        N, M = int(rng.integers(1, 81)), int(rng.integers(1, 33))
        if N * M > 1024:
            continue
        P = int(rng.integers(1, min(16, (N + 1) // 2) + 1))
        Q = int(rng.integers(1, min(16, (M + 1) // 2) + 1))
        if P * Q <= 100:
            out.append((N, M, P, Q))
    return out


@pytest.mark.parametrize("form", [2, 1, 0])
def test_batched_box_form_members(oracle_mod, form):
    shapes = box_shapes(48, 51)
    items, host = make_batch(shapes, "cn", 1500)
    plan = cov.BatchedPlan(items)
    assert plan.tuning["form"] == 2  # the default where every member fits it
    plan.set_tuning(form, 0, 4)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.upload(ws)
    plan.run(ws)
    torch.cuda.synchronize()
    cov.check_device_status(ws)
    for (At, Rt, P, Q), A in zip(items, host):
        got = Rt.cpu().numpy()
        assert rel_fro(got, oracle_R(oracle_mod, A, P, Q)) < F32_TOL, (A.shape, P, Q, form)
        assert np.array_equal(got, got.conj().T)
        assert np.all(got.diagonal().imag == 0)


def test_batched_box_form_integer_exact(oracle_mod):
    # small integers: products, column sums, walks and lane-window sums are
    # exact integers in FP32, so the SUM result is exact
    shapes = box_shapes(30, 52)
    items, host = make_batch(shapes, "int", 1700)
    plan, _ = run_plan(items, norm="sum")
    assert plan.tuning["form"] == 2
    for (At, Rt, P, Q), A in zip(items, host):
        S = oracle_R(oracle_mod, A, P, Q, mean=False)
        assert np.array_equal(Rt.cpu().numpy(), S.astype(np.complex64)), (A.shape, P, Q)
