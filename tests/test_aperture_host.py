"""Host-side construction of the aperture descriptors (every overlapping
aperture of one image, read in place): counts, pointer offsets, strides and
argument checks. No device memory is touched."""
import ctypes

import pytest

import paper_1303_2285_gb300 as cov


def test_count_and_offsets():
    img, R = 0x10000000, 0x20000000
    H, W, ld = 64, 80, 96
    arr = cov.aperture_descs(img, "c64", H, W, ld, (25, 20), (10, 7), 5, 4, R)
    nr, nc = (H - 25) // 10 + 1, (W - 20) // 7 + 1
    assert len(arr) == nr * nc
    for a in range(nr):
        for b in range(nc):
            d = arr[a * nc + b]
            assert d.A == img + ((a * 10) * ld + b * 7) * 8
            assert d.R == R + (a * nc + b) * (20 * 20) * 8
            assert (d.lda, d.N, d.M, d.P, d.Q) == (ld, 25, 20, 5, 4)


def test_c128_element_size():
    arr = cov.aperture_descs(0x1000, "c128", 10, 10, 10, (5, 5), (5, 5), 2, 2, 0x9000)
    assert len(arr) == 4
    assert arr[3].A == 0x1000 + (5 * 10 + 5) * 16
    assert arr[3].R == 0x9000 + 3 * 16 * 16


@pytest.mark.parametrize("H,W,ld,an,am,sr,sc,P,Q", [
    (5, 30, 30, 30, 10, 1, 1, 2, 2),     # aperture taller than the image
    (30, 30, 29, 10, 10, 1, 1, 2, 2),    # ld < W
    (30, 30, 30, 10, 10, 0, 1, 2, 2),    # zero step
    (30, 30, 30, 10, 10, 1, 1, 11, 2),   # P > aperture rows
])
def test_argument_checks(H, W, ld, an, am, sr, sc, P, Q):
    n = ctypes.c_int(0)
    assert cov.load().cov_aperture_descs(None, 0, H, W, ld, an, am, sr, sc, P, Q, None, None, 0,
                                         ctypes.byref(n)) == 1


def test_too_small_output_array():
    lib = cov.load()
    n = ctypes.c_int(0)
    arr = (cov.CovDesc * 2)()
    assert lib.cov_aperture_descs(0x1000, 0, 30, 30, 30, 10, 10, 10, 10, 2, 2, 0x2000, arr, 2,
                                  ctypes.byref(n)) == 1
    assert n.value == 9


def test_quarter_million_apertures_plan():
    # The large image-processing case of Section 2.3: an 8000 x 8000 image cut
    # into about 250,000 overlapping apertures. R offsets pass 2^31 elements,
    # so descriptor addresses must be 64-bit; the plan is built on the host.
    img, R = 0x10000000, 0x7000000000
    arr = cov.aperture_descs(img, "c64", 8000, 8000, 8000, (25, 25), (16, 16), 10, 10, R)
    n = len(arr)
    assert n == 499 * 499
    assert arr[n - 1].R == R + (n - 1) * 100 * 100 * 8
    assert arr[n - 1].A == img + (498 * 16 * 8000 + 498 * 16) * 8
    plan = cov.BatchedPlan(None, descs=arr)
    assert plan.tuning["form"] == 2  # the box form: 25 x 25 apertures, 10 x 10 windows
    assert plan.workspace_bytes >= n * ctypes.sizeof(cov.CovDesc)


@pytest.mark.parametrize("args,status", [
    # (image, dtype, H, W, ld, an, am, sr, sc, P, Q, R, norm): checks made before any CUDA call
    ((None, 0, 64, 64, 64, 25, 25, 10, 10, 10, 10, 0x2000, 0), 1),     # null image
    ((0x1000, 0, 64, 64, 64, 25, 25, 10, 10, 10, 10, None, 0), 1),     # null R
    ((0x1004, 0, 64, 64, 64, 25, 25, 10, 10, 10, 10, 0x2000, 0), 1),   # misaligned image
    ((0x1000, 0, 64, 64, 64, 25, 25, 10, 10, 10, 10, 0x2000, 2), 1),   # bad norm
    ((0x1000, 0, 64, 64, 63, 25, 25, 10, 10, 10, 10, 0x2000, 0), 1),   # ld < W
    ((0x1000, 0, 64, 64, 64, 25, 25, 10, 10, 26, 10, 0x2000, 0), 1),   # P > aperture rows
    ((0x1000, 1, 64, 64, 64, 25, 25, 10, 10, 10, 10, 0x2000, 0), 5),   # complex128
    ((0x1000, 0, 64, 64, 64, 25, 25, 10, 10, 17, 10, 0x2000, 0), 5),   # P above 16
    ((0x1000, 0, 99, 99, 99, 65, 25, 10, 10, 10, 10, 0x2000, 0), 5),   # 65 aperture rows
    ((0x1000, 0, 99, 99, 99, 25, 65, 10, 10, 10, 10, 0x2000, 0), 5),   # 65 aperture columns
])
def test_strip_argument_checks(args, status):
    assert cov.load().cov_estimate_apertures(*args, None) == status


def test_strip_wrapper_rejects_host_and_wrong_dtype_images():
    import torch
    with pytest.raises(ValueError):
        cov.apertures(torch.zeros((30, 30), dtype=torch.complex64), (10, 10), (10, 10), 4, 4)
    with pytest.raises(ValueError):
        cov.apertures(torch.zeros((30, 30), dtype=torch.complex128), (10, 10), (10, 10), 4, 4)
