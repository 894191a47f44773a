"""The typed short forms cov_estimate_c64 / cov_estimate_c128 (Eq. 2.1-2.2,
Section 2.2) called through the C ABI against the oracle, and the FMA-rate
instrumentation the roofline figures use.

Bars as in test_gpu_recurrence.py: complex128 bit-identical to the oracle on
small-integer inputs; complex64 within 1e-5 relative Frobenius of the FP64
oracle. Shapes without inner rows or columns run the combination path as
well; shapes it does not take (P or Q above 32) go through COV_DIRECT
(COV_AUTO), which is held to the same bars.
"""
import ctypes

import numpy as np
import pytest
import torch

import cov_workloads as wl
import paper_1303_2285_gb300 as cov

from gpu_util import guarded, oracle_R, rel_fro, to_dev  # noqa: E402

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5


def _stream():
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("N,M,P,Q", [(64, 64, 8, 8), (100, 70, 8, 3), (40, 17, 7, 1),
                                     (9, 30, 6, 4), (1, 1, 1, 1), (40, 36, 33, 1)])
def test_typed_c128_integer_bit_exact(oracle_mod, N, M, P, Q):
    lib = cov.load()
    A_np = wl.integer_valued((N, M), 91 + N * M)
    A = to_dev(A_np, torch.complex128)
    R, check = guarded((P * Q, P * Q), torch.complex128)
    assert lib.cov_estimate_c128(A.data_ptr(), N, M, P, Q, R.data_ptr(), _stream()) == 0
    torch.cuda.synchronize()
    check()
    assert np.array_equal(R.cpu().numpy(), oracle_R(oracle_mod, A_np, P, Q))


@pytest.mark.parametrize("N,M,P,Q", [(64, 64, 8, 8), (130, 200, 16, 16), (37, 45, 5, 7),
                                     (9, 30, 6, 4)])
def test_typed_c64_gaussian(oracle_mod, N, M, P, Q):
    lib = cov.load()
    A_np = wl.complex_normal((N, M), 17 + N + M, dtype="c64")
    A = to_dev(A_np, torch.complex64)
    R, check = guarded((P * Q, P * Q), torch.complex64)
    assert lib.cov_estimate_c64(A.data_ptr(), N, M, P, Q, R.data_ptr(), _stream()) == 0
    torch.cuda.synchronize()
    check()
    assert rel_fro(R.cpu().numpy().astype(np.complex128), oracle_R(oracle_mod, A_np, P, Q)) < F32_TOL


def test_typed_forms_reject_bad_arguments():
    lib = cov.load()
    A = torch.zeros((8, 8), dtype=torch.complex64, device="cuda")
    R = torch.zeros((16, 16), dtype=torch.complex64, device="cuda")
    assert lib.cov_estimate_c64(None, 8, 8, 4, 4, R.data_ptr(), _stream()) == 1
    assert lib.cov_estimate_c64(A.data_ptr(), 8, 8, 9, 4, R.data_ptr(), _stream()) == 1
    assert lib.cov_estimate_c128(A.data_ptr(), 8, 8, 4, 0, R.data_ptr(), _stream()) == 1


def test_fma_rate_measurement():
    lib = cov.load()
    f32, f64 = ctypes.c_double(0), ctypes.c_double(0)
    assert lib.cov_measure_fma_rate(0, 3, ctypes.byref(f32), _stream()) == 0
    assert lib.cov_measure_fma_rate(1, 3, ctypes.byref(f64), _stream()) == 0
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # at most 128 FP32 lanes per SM at 2.2 GHz; FP64 well below FP32
    assert 0.2 * sms * 128 * 1.0e9 < f32.value < sms * 128 * 2.2e9
    assert 0 < f64.value < f32.value
    assert lib.cov_measure_fma_rate(0, 0, ctypes.byref(f32), _stream()) == 1
