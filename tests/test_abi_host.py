"""Host-only checks of the C ABI: the library builds and loads, exports every
entry point of include/cov.h, its plan layer agrees with the oracle's
counting (an independent implementation), and argument checks fail before any
CUDA call. No GPU is used."""
import ctypes
import os
import re

import pytest

import paper_1303_2285_gb300 as cov
from oracle import combinations as cb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "cov.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(cov_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_function():
    lib = cov.load()
    names = header_functions()
    assert len(names) >= 14
    bound = {n for n, _, _ in cov.SIGNATURES}
    for n in names:
        assert hasattr(lib, n), n
        assert n in bound, f"{n} has no binding"
    assert bound == set(names), "binding names a function the header does not declare"
    # the package exposes each entry point under the C name
    for n in names:
        assert getattr(cov, n) is getattr(lib, n)
    with pytest.raises(AttributeError):
        cov.cov_not_a_function


def test_status_strings_and_version():
    lib = cov.load()
    for code in range(7):
        assert lib.cov_status_string(code).decode().startswith(cov.STATUS[code])
    assert lib.cov_version() >= 100


@pytest.mark.parametrize("N,M,P,Q", [(64, 64, 8, 8), (1024, 1024, 16, 16), (2048, 512, 32, 32),
                                     (256, 256, 12, 12), (20, 20, 8, 8), (32, 32, 13, 13),
                                     (37, 11, 5, 6), (9, 9, 9, 9), (5, 1, 2, 1)])
def test_plan_counts_match_oracle(N, M, P, Q):
    info = cov.plan_info(N, M, P, Q)
    assert info["K"] == (N - P + 1) * (M - Q + 1)
    assert info["n_combinations"] == cb.n_unique_combinations(P, Q)
    assert info["distinct_products"] == cb.um_enumerated(N, M, P, Q)
    assert info["r_elements"] == (P * Q) ** 2
    D = P * Q
    assert info["naive_macs"] == info["K"] * D * (D + 1) // 2
    # the combination path takes every shape with P, Q <= 32, including those
    # without inner rows (N < 2P - 1) or inner columns (M < 2Q - 1)
    assert info["recurrence_ok"] == int(P <= 32 and Q <= 32)


@pytest.mark.parametrize("N,M,P,Q", [(64, 64, 8, 8), (1024, 1024, 16, 16), (2048, 512, 32, 32),
                                     (33, 70, 3, 11), (15, 31, 8, 16), (9, 9, 9, 9), (7, 30, 5, 3),
                                     (30, 7, 2, 6), (12, 12, 7, 7), (5, 5, 1, 5), (62, 900, 32, 4),
                                     (40, 40, 32, 32)])
def test_plan_products_cover_um(N, M, P, Q):
    # Every distinct product is formed by exactly one of the two product
    # kernels; the rest of UM is the fringe-row x fringe-column corner
    # products, which the fringe-row kernel also forms.
    info = cov.plan_info(N, M, P, Q)
    assert info["products_inner"] + info["products_fringe"] == info["distinct_products"]


def test_workspace_sizes():
    n1 = cov.workspace_size("c64", 1024, 1024, 16, 16, "recurrence")
    n2 = cov.workspace_size("c128", 1024, 1024, 16, 16, "recurrence")
    assert n1 > 256 and n1 % 256 == 0 and n2 > n1
    assert cov.workspace_size("c64", 40, 40, 33, 1, "auto") == 256  # direct path (P > 32)
    assert cov.workspace_size("c64", 9, 9, 9, 9, "auto") > 256  # no inner rows or columns
    with pytest.raises(cov.CovError) as e:
        cov.workspace_size("c64", 40, 40, 33, 1, "recurrence")
    assert e.value.code == 5


def test_argument_checks_fail_before_cuda():
    lib = cov.load()
    fake = ctypes.c_void_p(0x1000)
    # null input
    assert lib.cov_estimate_ex(None, 0, 8, 8, 8, 2, 2, fake, 0, 0, None, 0, None) == 1
    # P > N
    assert lib.cov_estimate_ex(fake, 0, 8, 8, 8, 9, 2, fake, 0, 0, None, 0, None) == 1
    # lda < M
    assert lib.cov_estimate_ex(fake, 0, 8, 8, 7, 2, 2, fake, 0, 0, None, 0, None) == 1
    # bad dtype / norm
    assert lib.cov_estimate_ex(fake, 7, 8, 8, 8, 2, 2, fake, 0, 0, None, 0, None) == 1
    assert lib.cov_estimate_ex(fake, 0, 8, 8, 8, 2, 2, fake, 0, 9, None, 0, None) == 1
    # recurrence without a workspace
    assert lib.cov_estimate_ex(fake, 0, 64, 64, 64, 8, 8, fake, 1, 0, None, 0, None) == 3
    # misaligned workspace
    assert lib.cov_estimate_ex(fake, 0, 64, 64, 64, 8, 8, fake, 1, 0,
                               ctypes.c_void_p(0x1008), 1 << 30, None) == 3
    # recurrence on a shape it does not take
    assert lib.cov_estimate_ex(fake, 0, 40, 40, 40, 33, 1, fake, 1, 0, None, 0, None) == 5
    info = cov.PlanInfo()
    assert lib.cov_plan_info(0, 5, 1, 1, ctypes.byref(info)) == 1
    assert lib.cov_plan_info(5, 5, 1, 1, None) == 1


def test_batched_plan_validation_host_only():
    lib = cov.load()
    fake = 0x1000

    def plan(shapes):
        arr = (cov.CovDesc * len(shapes))()
        for k, (N, M, P, Q) in enumerate(shapes):
            arr[k] = cov.CovDesc(fake, fake, M, N, M, P, Q)
        ptr = ctypes.c_void_p()
        code = lib.cov_batched_plan_create(arr, len(shapes), 0, 0, 0, ctypes.byref(ptr))
        return code, ptr

    def form_after(shapes, form):
        code, ptr = plan(shapes)
        assert code == 0, shapes
        t = cov.BatchedTuning(form, 0, 4)
        ok = lib.cov_batched_set_tuning(ptr, ctypes.byref(t)) == 0
        lib.cov_batched_plan_destroy(ptr)
        return ok

    code, ptr = plan([(64, 64, 8, 8), (33, 40, 16, 2), (200, 512, 3, 16)])
    assert code == 0
    n = ctypes.c_size_t(0)
    assert lib.cov_batched_workspace_size(ptr, ctypes.byref(n)) == 0 and n.value > 256
    lib.cov_batched_plan_destroy(ptr)
    # beyond the CTA form's limits (P or Q above 16, no inner rows, M above
    # 512): only the stage form takes the batch
    for wide in ([(64, 64, 17, 8)], [(30, 64, 16, 2)], [(64, 513, 2, 2)], [(40, 40, 32, 32)]):
        assert form_after(wide, 3) and not form_after(wide, 0), wide
    assert form_after([(64, 64, 8, 8)], 0) and form_after([(64, 64, 8, 8)], 3)
    for bad in ([(8, 8, 0, 1)], [(64, 64, 33, 2)], [(8, 8, 9, 2)]):
        assert plan(bad)[0] == 1, bad
    arr = (cov.CovDesc * 1)(cov.CovDesc(fake, fake, 8, 8, 8, 2, 2))
    ptr = ctypes.c_void_p()
    assert lib.cov_batched_plan_create(arr, 1, 1, 0, 0, ctypes.byref(ptr)) == 0  # c128: stage form
    t = cov.BatchedTuning()
    assert lib.cov_batched_get_tuning(ptr, ctypes.byref(t)) == 0 and t.form == 3
    t.form = 0
    assert lib.cov_batched_set_tuning(ptr, ctypes.byref(t)) == 1
    lib.cov_batched_plan_destroy(ptr)
    assert lib.cov_batched_plan_create(arr, 1, 0, 2, 0, ctypes.byref(ptr)) == 5  # gemm algo


def test_backward_workspace_by_form():
    # the stencil form tabulates (2P-1)(2Q-1) weights per class pair; the
    # dense form keeps Y = H X (PQ x windows)
    st = cov.backward_workspace_size(256, 256, 12, 12, "stencil")
    de = cov.backward_workspace_size(256, 256, 12, 12, "dense")
    assert st >= 23 ** 4 * 8 and de >= 144 * 245 * 245 * 8
    assert cov.backward_workspace_size(256, 256, 12, 12) == st  # auto picks the stencil
    assert cov.backward_workspace_size(9, 9, 9, 9) == cov.backward_workspace_size(9, 9, 9, 9, "dense")
    # complex128: the dense form (FP64), Y twice the bytes; no stencil form
    d128 = cov.backward_workspace_size(256, 256, 12, 12, "auto", "c128")
    assert d128 == cov.backward_workspace_size(256, 256, 12, 12, "dense", "c128")
    assert d128 - 256 >= 2 * (de - 256) - 256
    with pytest.raises(cov.CovError):
        cov.backward_workspace_size(256, 256, 12, 12, "stencil", "c128")
    with pytest.raises(cov.CovError):
        cov.backward_workspace_size(9, 9, 9, 9, "stencil")
