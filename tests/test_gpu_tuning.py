"""GPU behaviour of the tuned knobs and the failure-detection self-test.

Every knob value the tuner may pick must give the same estimate: each
setting is checked against the CPU oracle (FP64 on integer-valued input
bit-exact, FP32 on Gaussian input within 1e-5 relative Frobenius error)."""
import numpy as np
import pytest
import torch

import cov_workloads as wl
import paper_1303_2285_gb300 as cov

pytestmark = pytest.mark.gpu

from gpu_util import oracle_R, rel_fro, to_dev  # noqa: E402

KNOBS = [
    {"lag_group": 4, "rows_per_task": 8, "reseed_interval": 1, "kernels": 4, "tile_cols": 64},
    {"lag_group": 8, "rows_per_task": 16, "reseed_interval": 2, "kernels": 4, "tile_cols": 64},
    {"lag_group": 16, "rows_per_task": 24, "reseed_interval": 32, "kernels": 4, "tile_cols": 64},
    {"lag_group": 4, "rows_per_task": 64, "reseed_interval": 3, "kernels": 4, "tile_cols": 64},
    {"lag_group": 8, "rows_per_task": 128, "reseed_interval": 16, "kernels": 4, "tile_cols": 64},
    {"lag_group": 16, "rows_per_task": 256, "reseed_interval": 5, "kernels": 4, "tile_cols": 64},
    {"lag_group": 4, "rows_per_task": 8, "reseed_interval": 1, "kernels": 1, "tile_cols": 64},
    {"lag_group": 8, "rows_per_task": 32, "reseed_interval": 4, "kernels": 1, "tile_cols": 64},
    {"lag_group": 16, "rows_per_task": 128, "reseed_interval": 8, "kernels": 1, "tile_cols": 64},
    {"lag_group": 16, "rows_per_task": 48, "reseed_interval": 32, "kernels": 1, "tile_cols": 64},
    # 32-column tiles (taller row blocks fit)
    {"lag_group": 4, "rows_per_task": 8, "reseed_interval": 2, "kernels": 4, "tile_cols": 32},
    {"lag_group": 8, "rows_per_task": 192, "reseed_interval": 7, "kernels": 4, "tile_cols": 32},
    {"lag_group": 16, "rows_per_task": 160, "reseed_interval": 16, "kernels": 4, "tile_cols": 32},
    {"lag_group": 8, "rows_per_task": 40, "reseed_interval": 1, "kernels": 1, "tile_cols": 32},
    {"lag_group": 16, "rows_per_task": 224, "reseed_interval": 32, "kernels": 1, "tile_cols": 32},
]


@pytest.fixture(autouse=True)
def _clean_cache():
    cov.tuning_clear()
    yield
    cov.tuning_clear()


def _run(A_np, P, Q, dtype):
    A = to_dev(A_np, dtype)
    R = cov.estimate(A, P, Q, algo="recurrence")
    torch.cuda.synchronize()
    return R.cpu().numpy()


@pytest.mark.parametrize("knobs", KNOBS)
@pytest.mark.parametrize("N,M,P,Q", [(300, 101, 7, 5), (200, 150, 16, 16), (95, 95, 32, 32),
                                     (40, 33, 17, 3), (64, 100, 2, 17)])
def test_knobs_fp32_parity(oracle_mod, knobs, N, M, P, Q):
    A = wl.complex_normal((N, M), 31 + N, dtype="c64")
    cov.tuning_set("c64", N, M, P, Q, knobs)
    got = _run(A, P, Q, torch.complex64)
    assert rel_fro(got, oracle_R(oracle_mod, A, P, Q)) < 1e-5


@pytest.mark.parametrize("knobs", [k for k in KNOBS if k["lag_group"] <= 8 and k["kernels"] == 4])
def test_knobs_fp64_integer_exact(oracle_mod, knobs):
    N, M, P, Q = 211, 97, 9, 6
    A = wl.integer_valued((N, M), 17, dtype="c128")
    cov.tuning_set("c128", N, M, P, Q, knobs)
    A_dev = to_dev(A, torch.complex128)
    R = cov.estimate(A_dev, P, Q, algo="recurrence", norm="sum")
    torch.cuda.synchronize()
    want = oracle_R(oracle_mod, A, P, Q, mean=False)
    assert np.array_equal(R.cpu().numpy(), want)


def test_autotune_caches_and_stays_correct(oracle_mod):
    N, M, P, Q = 512, 384, 12, 10
    A = wl.complex_normal((N, M), 5, dtype="c64")
    A_dev = to_dev(A, torch.complex64)
    best, ms = cov.autotune(A_dev, P, Q, reps=2)
    assert ms > 0
    got, cached = cov.tuning_get("c64", N, M, P, Q)
    assert cached and got == best and best["kernels"] in (1, 4)
    R = cov.estimate(A_dev, P, Q, algo="recurrence")
    torch.cuda.synchronize()
    assert rel_fro(R.cpu().numpy(), oracle_R(oracle_mod, A, P, Q)) < 1e-5


def test_autotune_small_workspace_skips_candidates():
    N, M, P, Q = 256, 256, 8, 8
    A = to_dev(wl.complex_normal((N, M), 6, dtype="c64"), torch.complex64)
    lib = cov.load()
    need = cov.workspace_size("c64", N, M, P, Q, "recurrence")
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    R = torch.empty((P * Q, P * Q), dtype=torch.complex64, device="cuda")
    import ctypes
    best, ms = cov.Tuning(), ctypes.c_float(0)
    code = lib.cov_autotune(A.data_ptr(), 0, N, M, M, P, Q, R.data_ptr(), ws.data_ptr(),
                            ws.numel(), 1, torch.cuda.current_stream().cuda_stream,
                            ctypes.byref(best), ctypes.byref(ms))
    assert code == 0
    # whatever it picked fits the workspace it was given
    assert cov.workspace_size("c64", N, M, P, Q, "recurrence") <= need


def test_timeout_selftest_reports_and_context_survives(oracle_mod):
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    cov.selftest_timeout(ws, limit_us=20000)
    with pytest.raises(cov.CovError) as e:
        cov.check_device_status(ws)
    assert e.value.code == 4
    # the status word was cleared by the read and the context still computes
    cov.check_device_status(ws)
    A = wl.complex_normal((64, 64), 8, dtype="c64")
    got = _run(A, 8, 8, torch.complex64)
    assert rel_fro(got, oracle_R(oracle_mod, A, 8, 8)) < 1e-5


def test_timeout_selftest_argument_checks():
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    for bad in (0, 1000001):
        with pytest.raises(cov.CovError):
            cov.selftest_timeout(ws, limit_us=bad)
