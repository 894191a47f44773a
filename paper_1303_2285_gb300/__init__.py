"""GB300 (sm_103a) covariance-method library: Python binding.

A thin ctypes layer over the C ABI of ``include/cov.h`` (``libcov.so``). It
marshals arguments only: torch tensors supply device memory and the current
CUDA stream, and every step of the computation runs in the library's CUDA
kernels. There is no CPU fallback: without the built library or a CUDA
device the calls raise.

The estimate (arXiv 1303.2285, Section 2.2, Eq. 2.1-2.2):
    R = (1/K) * sum over all K = (N-P+1)(M-Q+1) window positions of x x^H,
with x the column stack of the P x Q window (x[i + P*j] = A[p+i, q+j]).
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

from . import _build

__all__ = ["load", "estimate", "estimate_into", "workspace_size", "plan_info",
           "check_device_status", "CovError", "ALGOS", "NORMS", "DTYPES", "STATUS", "autotune",
           "tuning_get", "tuning_set", "tuning_clear", "tuning_save", "tuning_load",
           "covariance", "estimate_backward", "estimate_backward_batch",
           "backward_workspace_size", "BatchedPlan", "aperture_descs", "aperture_batch", "apertures",
           "selftest_timeout", "set_stage_events", "capon_spectrum", "SIGNATURES"]

ALGOS = {"auto": 0, "recurrence": 1, "gemm_tf32x3": 2, "gemm_bf16x3": 3, "direct": 4}
NORMS = {"mean": 0, "sum": 1}
DTYPES = {"c64": 0, "c128": 1}
STATUS = {0: "COV_OK", 1: "COV_EINVAL", 2: "COV_ECUDA", 3: "COV_EWORKSPACE",
          4: "COV_ETIMEOUT", 5: "COV_EUNSUPPORTED", 6: "COV_EDEVICE"}


class CovError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {STATUS.get(code, code)}")


class PlanInfo(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int64), ("n_combinations", ctypes.c_int64),
                ("distinct_products", ctypes.c_int64), ("r_elements", ctypes.c_int64),
                ("naive_macs", ctypes.c_int64), ("recurrence_ok", ctypes.c_int32),
                ("n_groups", ctypes.c_int32), ("n_tasks", ctypes.c_int64),
                ("products_inner", ctypes.c_int64), ("products_fringe", ctypes.c_int64)]


class Tuning(ctypes.Structure):
    """Knobs of the combination path: lags per group, rows per product task,
    walk re-seed interval, kernels per call (1 fused or 4), columns per
    shared-memory tile (32 or 64) (cov_tuning_t)."""
    _fields_ = [("lag_group", ctypes.c_int32), ("rows_per_task", ctypes.c_int32),
                ("reseed_interval", ctypes.c_int32), ("kernels", ctypes.c_int32),
                ("tile_cols", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class BatchedTuning(ctypes.Structure):
    """Knobs of a batched plan: kernel form (0 CTA per member, 1 warp per
    member, 2 box sums of small members in shared memory, 3 the single-matrix
    stages over all members), walk re-seed interval of form 0 (0: one seed
    per segment), row ranges per column block of form 0
    (cov_batched_tuning_t)."""
    _fields_ = [("form", ctypes.c_int32), ("reseed_interval", ctypes.c_int32),
                ("row_ranges", ctypes.c_int32)]


class CovDesc(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("R", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("N", ctypes.c_int32), ("M", ctypes.c_int32), ("P", ctypes.c_int32),
                ("Q", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None

# (name, restype, argtypes) of every exported entry point of include/cov.h
_VP, _I64, _I, _SZ = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
SIGNATURES = [
    ("cov_status_string", ctypes.c_char_p, [_I]),
    ("cov_version", _I, []),
    ("cov_plan_info", _I, [_I64, _I64, _I, _I, ctypes.POINTER(PlanInfo)]),
    ("cov_workspace_size", _I, [_I, _I64, _I64, _I, _I, _I, ctypes.POINTER(_SZ)]),
    ("cov_estimate_ex", _I, [_VP, _I, _I64, _I64, _I64, _I, _I, _VP, _I, _I, _VP, _SZ, _VP]),
    ("cov_estimate", _I, [_VP, _I, _I64, _I64, _I, _I, _VP, _VP]),
    ("cov_check_device_status", _I, [_VP, _VP]),
    ("cov_estimate_c64", _I, [_VP, _I64, _I64, _I, _I, _VP, _VP]),
    ("cov_estimate_c128", _I, [_VP, _I64, _I64, _I, _I, _VP, _VP]),
    ("cov_estimate_noalloc", _I, [_VP, _I, _I64, _I64, _I64, _I, _I, _VP, _I, _VP]),
    ("cov_noalloc_check_status", _I, [_VP]),
    ("cov_measure_fma_rate", _I, [_I, _I, ctypes.POINTER(ctypes.c_double), _VP]),
    ("cov_set_stage_events", _I, [ctypes.POINTER(_VP), _I]),
    ("cov_batched_plan_create", _I, [ctypes.POINTER(CovDesc), _I, _I, _I, _I,
                                     ctypes.POINTER(_VP)]),
    ("cov_batched_workspace_size", _I, [_VP, ctypes.POINTER(_SZ)]),
    ("cov_aperture_descs", _I, [_VP, _I, _I64, _I64, _I64, _I, _I, _I, _I, _I, _I, _VP,
                                ctypes.POINTER(CovDesc), _I, ctypes.POINTER(ctypes.c_int)]),
    ("cov_estimate_apertures", _I, [_VP, _I, _I64, _I64, _I64, _I, _I, _I, _I, _I, _I, _VP, _I,
                                    _VP]),
    ("cov_batched_upload", _I, [_VP, _VP, _SZ, _VP]),
    ("cov_estimate_batched", _I, [_VP, _VP, _SZ, _VP]),
    ("cov_batched_plan_destroy", None, [_VP]),
    ("cov_batched_get_tuning", _I, [_VP, ctypes.POINTER(BatchedTuning)]),
    ("cov_batched_set_tuning", _I, [_VP, ctypes.POINTER(BatchedTuning)]),
    ("cov_batched_autotune", _I, [_VP, _VP, _SZ, _I, _VP]),
    ("cov_backward_workspace_size", _I, [_I, _I64, _I64, _I, _I, ctypes.POINTER(_SZ)]),
    ("cov_estimate_backward", _I, [_VP, _VP, _I, _I64, _I64, _I, _I, _I, _VP, _VP, _SZ, _VP]),
    ("cov_backward_strided_workspace_size", _I, [_I, _I64, _I64, _I, _I, ctypes.POINTER(_SZ)]),
    ("cov_estimate_backward_strided", _I, [_VP, _I64, _VP, _I64, _VP, _I64, _I, _I64, _I64, _I,
                                           _I, _I, _VP, _SZ, _VP]),
    ("cov_backward_workspace_size_ex", _I, [_I, _I64, _I64, _I, _I, _I, ctypes.POINTER(_SZ)]),
    ("cov_estimate_backward_ex", _I, [_VP, _VP, _I, _I64, _I64, _I, _I, _I, _I, _VP, _VP, _SZ,
                                      _VP]),
    ("cov_selftest_timeout", _I, [_VP, _SZ, ctypes.c_uint32, _VP]),
    ("cov_capon_spectrum", _I, [_VP, _I, _I, _VP, _I, ctypes.c_float, _VP, _VP]),
    ("cov_partition_lags", _I, [_I64, _I64, _I, _I, _I, ctypes.POINTER(ctypes.c_int32),
                                ctypes.POINTER(ctypes.c_int64)]),
    ("cov_estimate_shard", _I, [_VP, _I, _I64, _I64, _I64, _I, _I, _I, _I, _VP, _I, _VP, _SZ,
                                _VP]),
    ("cov_shard_packed_size", _I, [_I, _I, _I, _I, _I, ctypes.POINTER(_SZ)]),
    ("cov_shard_pack", _I, [_VP, _I, _I, _I, _I, _I, _VP, _VP]),
    ("cov_shard_unpack", _I, [_VP, _I, _I, _I, _I, _I, _VP, _VP]),
    ("cov_partition_matrices", _I, [ctypes.POINTER(CovDesc), _I, _I,
                                    ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_int64)]),
    ("cov_partition_rows", _I, [_I64, _I, _I, ctypes.POINTER(ctypes.c_int64),
                                ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    ("cov_tuning_get", _I, [_I, _I64, _I64, _I, _I, ctypes.POINTER(Tuning),
                            ctypes.POINTER(ctypes.c_int)]),
    ("cov_tuning_set", _I, [_I, _I64, _I64, _I, _I, ctypes.POINTER(Tuning)]),
    ("cov_tuning_clear", None, []),
    ("cov_tuning_save", _I, [ctypes.c_char_p]),
    ("cov_tuning_load", _I, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_int)]),
    ("cov_autotune_workspace_size", _I, [_I, _I64, _I64, _I, _I, ctypes.POINTER(_SZ)]),
    ("cov_autotune", _I, [_VP, _I, _I64, _I64, _I64, _I, _I, _VP, _VP, _SZ, _I, _VP,
                          ctypes.POINTER(Tuning), ctypes.POINTER(ctypes.c_float)]),
]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libcov.so (building it with nvcc first when missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing and _build.needs_build():
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError("libcov.so is not built; run __graft_entry__.build()")
            lib = ctypes.CDLL(_build.LIB)
            for name, res, args in SIGNATURES:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


_C_NAMES = frozenset(n for n, _, _ in SIGNATURES)


def __getattr__(name: str):
    """Every C entry point under its own name (``paper_1303_2285_gb300.cov_estimate_ex``
    and so on): the typed ctypes function of the loaded library."""
    if name in _C_NAMES:
        return getattr(load(), name)
    raise AttributeError(f"module {__name__!r} has no attribute {name!r}")


def _check(code: int, what: str):
    if code != 0:
        raise CovError(code, what)


def plan_info(N: int, M: int, P: int, Q: int) -> dict:
    """Counts of the plan layer (host only): K, |UC|, UM, ... ."""
    info = PlanInfo()
    _check(load().cov_plan_info(N, M, P, Q, ctypes.byref(info)), "cov_plan_info")
    return {f: getattr(info, f) for f, _ in PlanInfo._fields_}


def workspace_size(dtype: str, N: int, M: int, P: int, Q: int, algo: str = "auto") -> int:
    out = ctypes.c_size_t(0)
    _check(load().cov_workspace_size(DTYPES[dtype], N, M, P, Q, ALGOS[algo], ctypes.byref(out)),
           "cov_workspace_size")
    return int(out.value)


def _torch():
    import torch
    return torch


def _dtype_of(A) -> str:
    torch = _torch()
    if A.dtype == torch.complex64:
        return "c64"
    if A.dtype == torch.complex128:
        return "c128"
    raise TypeError("A must be complex64 or complex128")


def _stream_ptr(stream) -> Optional[int]:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def estimate_into(A, R, P: int, Q: int, algo: str = "auto", norm: str = "mean",
                  workspace=None, stream=None):
    """R <- estimate of A (device tensors). ``workspace`` is a uint8 CUDA tensor
    of at least ``workspace_size`` bytes (allocated here when None)."""
    torch = _torch()
    if not (A.is_cuda and R.is_cuda):
        raise ValueError("A and R must be CUDA tensors (no CPU fallback)")
    if A.dim() != 2 or A.stride(1) != 1:
        raise ValueError("A must be 2-D with unit column stride")
    dt = _dtype_of(A)
    if R.dtype != A.dtype or not R.is_contiguous() or tuple(R.shape) != (P * Q, P * Q):
        raise ValueError("R must be a contiguous PQ x PQ tensor of A's dtype")
    N, M = A.shape
    need = workspace_size(dt, N, M, P, Q, algo)
    if workspace is None:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=A.device)
    if workspace.numel() < need:
        raise ValueError(f"workspace too small: {workspace.numel()} < {need}")
    code = load().cov_estimate_ex(A.data_ptr(), DTYPES[dt], N, M, A.stride(0), P, Q,
                                  R.data_ptr(), ALGOS[algo], NORMS[norm],
                                  workspace.data_ptr(), workspace.numel(), _stream_ptr(stream))
    _check(code, "cov_estimate_ex")
    return R


def estimate(A, P: int, Q: int, algo: str = "auto", norm: str = "mean", workspace=None,
             stream=None):
    """Returns R (PQ x PQ, A's dtype) for the device tensor A."""
    torch = _torch()
    R = torch.empty((P * Q, P * Q), dtype=A.dtype, device=A.device)
    return estimate_into(A, R, P, Q, algo, norm, workspace, stream)


BWD_FORMS = {"auto": 0, "dense": 1, "stencil": 2}


def backward_workspace_size(N: int, M: int, P: int, Q: int, form: str = "auto",
                            dtype: str = "c64") -> int:
    out = ctypes.c_size_t(0)
    _check(load().cov_backward_workspace_size_ex(DTYPES[dtype], N, M, P, Q, BWD_FORMS[form],
                                                 ctypes.byref(out)),
           "cov_backward_workspace_size")
    return int(out.value)


def estimate_backward(A, G, P: int, Q: int, norm: str = "mean", workspace=None, stream=None,
                      form: str = "auto"):
    """dL/dA for G = dL/dR (CUDA tensors, both complex64 or both complex128;
    dL/dRe + i dL/dIm convention). ``form``: "auto" (complex64: the stencil
    where it applies; complex128: the dense form in FP64), "stencil" or
    "dense"."""
    torch = _torch()
    if not (A.is_cuda and G.is_cuda) or A.dtype != G.dtype:
        raise ValueError("A and G must be CUDA tensors of one dtype")
    dt = _dtype_of(A)
    A = A.contiguous()
    G = G.contiguous()
    N, M = A.shape
    if tuple(G.shape) != (P * Q, P * Q):
        raise ValueError("G must be PQ x PQ")
    need = backward_workspace_size(N, M, P, Q, form, dt)
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=A.device)
    dA = torch.empty_like(A)
    _check(load().cov_estimate_backward_ex(A.data_ptr(), G.data_ptr(), DTYPES[dt], N, M, P, Q,
                                           NORMS[norm], BWD_FORMS[form], dA.data_ptr(),
                                           workspace.data_ptr(), workspace.numel(),
                                           _stream_ptr(stream)),
           "cov_estimate_backward")
    return dA


def estimate_backward_batch(A, G, P: int, Q: int, norm: str = "mean", workspace=None,
                            stream=None):
    """dL/dA for a batch: A (B, N, M) and G (B, PQ, PQ) contiguous complex64
    CUDA tensors; one launch sequence of the stencil form."""
    torch = _torch()
    if not (A.is_cuda and G.is_cuda) or A.dtype != torch.complex64 or G.dtype != torch.complex64:
        raise ValueError("A and G must be complex64 CUDA tensors")
    if A.dim() != 3 or G.dim() != 3 or A.shape[0] != G.shape[0]:
        raise ValueError("A must be (B, N, M) and G (B, PQ, PQ)")
    A = A.contiguous()
    G = G.contiguous()
    B, N, M = A.shape
    need = ctypes.c_size_t(0)
    _check(load().cov_backward_strided_workspace_size(B, N, M, P, Q, ctypes.byref(need)),
           "cov_backward_strided_workspace_size")
    if workspace is None:
        workspace = torch.empty(int(need.value), dtype=torch.uint8, device=A.device)
    dA = torch.empty_like(A)
    _check(load().cov_estimate_backward_strided(A.data_ptr(), N * M, G.data_ptr(), P * Q * P * Q,
                                                dA.data_ptr(), N * M, B, N, M, P, Q, NORMS[norm],
                                                workspace.data_ptr(), workspace.numel(),
                                                _stream_ptr(stream)),
           "cov_estimate_backward_strided")
    return dA


def _make_autograd():
    torch = _torch()

    class CovarianceEstimate(torch.autograd.Function):
        """R = estimate(A) with the library's adjoint kernels as backward."""

        @staticmethod
        def forward(ctx, A, P, Q, norm):
            ctx.save_for_backward(A)
            ctx.P, ctx.Q, ctx.norm = P, Q, norm
            return estimate(A.detach().contiguous(), P, Q, algo="auto", norm=norm)

        @staticmethod
        def backward(ctx, G):
            (A,) = ctx.saved_tensors
            dA = estimate_backward(A.detach(), G.contiguous(), ctx.P, ctx.Q, ctx.norm)
            return dA, None, None, None

    return CovarianceEstimate


_autograd_fn = None


def covariance(A, P: int, Q: int, norm: str = "mean"):
    """Differentiable estimate: R = covariance(A, P, Q); backward runs the
    library's adjoint (the stencil form where it applies, else (G + G^H) X
    with a gather col2im). complex64 or complex128 CUDA tensors."""
    global _autograd_fn
    if _autograd_fn is None:
        _autograd_fn = _make_autograd()
    return _autograd_fn.apply(A, P, Q, norm)


class BatchedPlan:
    """Many matrices of uneven shapes in one persistent launch (cov_batched_*).

    ``items``: sequence of (A, R, P, Q) with A an N x M complex64 (or, all of
    them, complex128) CUDA tensor (unit column stride) and R a contiguous
    PQ x PQ CUDA tensor of the same dtype. The plan keeps the device pointers:
    the tensors must outlive it. complex128 batches run the stage form only.
    """

    def __init__(self, items, norm: str = "mean", descs=None, dtype: Optional[str] = None):
        lib = load()
        if descs is not None:  # prepared descriptors (e.g. aperture_batch)
            arr, n = descs, len(descs)
            dtype = dtype or "c64"
        else:
            n = len(items)
            arr = (CovDesc * n)()
            kinds = set()
            for k, (A, R, P, Q) in enumerate(items):
                if not (A.is_cuda and R.is_cuda) or A.stride(1) != 1 or not R.is_contiguous():
                    raise ValueError("A and R must be CUDA tensors (A unit column stride, "
                                     "R contiguous)")
                kinds.add((str(A.dtype), str(R.dtype)))
                arr[k] = CovDesc(A.data_ptr(), R.data_ptr(), A.stride(0), A.shape[0], A.shape[1],
                                 P, Q)
            if kinds == {("torch.complex128", "torch.complex128")}:
                dtype = "c128"
            elif kinds == {("torch.complex64", "torch.complex64")}:
                dtype = "c64"
            else:
                raise ValueError("A and R must all be complex64, or all complex128")
        ptr = ctypes.c_void_p()
        _check(lib.cov_batched_plan_create(arr, n, DTYPES[dtype], ALGOS["auto"], NORMS[norm],
                                           ctypes.byref(ptr)), "cov_batched_plan_create")
        self._lib = lib
        self.ptr = ptr
        out = ctypes.c_size_t(0)
        _check(lib.cov_batched_workspace_size(ptr, ctypes.byref(out)), "cov_batched_workspace_size")
        self.workspace_bytes = int(out.value)

    def upload(self, workspace, stream=None) -> None:
        _check(self._lib.cov_batched_upload(self.ptr, workspace.data_ptr(), workspace.numel(),
                                            _stream_ptr(stream)), "cov_batched_upload")

    def run(self, workspace, stream=None) -> None:
        _check(self._lib.cov_estimate_batched(self.ptr, workspace.data_ptr(), workspace.numel(),
                                              _stream_ptr(stream)), "cov_estimate_batched")

    @property
    def tuning(self) -> dict:
        t = BatchedTuning()
        _check(self._lib.cov_batched_get_tuning(self.ptr, ctypes.byref(t)), "cov_batched_get_tuning")
        return {"form": t.form, "reseed_interval": t.reseed_interval, "row_ranges": t.row_ranges}

    def set_tuning(self, form: int, reseed_interval: int = 0, row_ranges: int = 4) -> None:
        """Sets the knobs (rebuilding the schedule): upload() again before run()."""
        t = BatchedTuning(form, reseed_interval, row_ranges)
        _check(self._lib.cov_batched_set_tuning(self.ptr, ctypes.byref(t)), "cov_batched_set_tuning")

    def autotune(self, workspace, reps: int = 3, stream=None) -> dict:
        """Times the candidate knob settings on this plan's members (writing
        their R), keeps the fastest and uploads it; returns it."""
        _check(self._lib.cov_batched_autotune(self.ptr, workspace.data_ptr(), workspace.numel(), reps,
                                              _stream_ptr(stream)), "cov_batched_autotune")
        return self.tuning

    def __del__(self):
        if getattr(self, "ptr", None) is not None and self.ptr.value:
            self._lib.cov_batched_plan_destroy(self.ptr)
            self.ptr = None


def aperture_descs(image_ptr: int, dtype: str, H: int, W: int, ld: int, ap: tuple, step: tuple,
                   P: int, Q: int, R_ptr: int):
    """Descriptors of every ap[0] x ap[1] aperture at stride step of an image
    (device pointers; host-side construction only)."""
    lib = load()
    n = ctypes.c_int(0)
    _check(lib.cov_aperture_descs(None, DTYPES[dtype], H, W, ld, ap[0], ap[1], step[0], step[1],
                                  P, Q, None, None, 0, ctypes.byref(n)), "cov_aperture_descs")
    arr = (CovDesc * n.value)()
    _check(lib.cov_aperture_descs(image_ptr, DTYPES[dtype], H, W, ld, ap[0], ap[1], step[0],
                                  step[1], P, Q, R_ptr, arr, n.value, ctypes.byref(n)),
           "cov_aperture_descs")
    return arr


def aperture_batch(image, ap: tuple, step: tuple, P: int, Q: int, norm: str = "mean"):
    """One batched plan over every aperture of a complex64 CUDA image, read in
    place: returns (plan, R) with R of shape (count, PQ, PQ); run the plan to
    fill R (plan.upload once, then plan.run)."""
    torch = _torch()
    if not image.is_cuda or image.dtype != torch.complex64 or image.stride(1) != 1:
        raise ValueError("image must be a complex64 CUDA tensor with unit column stride")
    H, W = image.shape
    n = ctypes.c_int(0)
    _check(load().cov_aperture_descs(None, DTYPES["c64"], H, W, image.stride(0), ap[0], ap[1],
                                     step[0], step[1], P, Q, None, None, 0, ctypes.byref(n)),
           "cov_aperture_descs")
    R = torch.empty((n.value, P * Q, P * Q), dtype=torch.complex64, device=image.device)
    arr = aperture_descs(image.data_ptr(), "c64", H, W, image.stride(0), ap, step, P, Q,
                         R.data_ptr())
    plan = BatchedPlan(None, norm=norm, descs=arr)
    plan._keep = (image, R)
    return plan, R


def apertures(image, ap: tuple, step: tuple, P: int, Q: int, norm: str = "mean", out=None,
              stream=None):
    """Estimates of every ap[0] x ap[1] aperture at stride step of a complex64
    CUDA image in one launch (cov_estimate_apertures); returns R of shape
    (count, PQ, PQ), apertures in row-major order (out: a tensor of that
    shape to overwrite)."""
    torch = _torch()
    if not image.is_cuda or image.dtype != torch.complex64 or image.stride(1) != 1:
        raise ValueError("image must be a complex64 CUDA tensor with unit column stride")
    H, W = image.shape
    n = ctypes.c_int(0)
    _check(load().cov_aperture_descs(None, DTYPES["c64"], H, W, image.stride(0), ap[0], ap[1],
                                     step[0], step[1], P, Q, None, None, 0, ctypes.byref(n)),
           "cov_aperture_descs")
    shape = (n.value, P * Q, P * Q)
    if out is None:
        out = torch.empty(shape, dtype=torch.complex64, device=image.device)
    elif tuple(out.shape) != shape or out.dtype != torch.complex64 or not out.is_contiguous():
        raise ValueError(f"out must be a contiguous complex64 tensor of shape {shape}")
    _check(load().cov_estimate_apertures(image.data_ptr(), DTYPES["c64"], H, W, image.stride(0),
                                         ap[0], ap[1], step[0], step[1], P, Q, out.data_ptr(),
                                         NORMS[norm], _stream_ptr(stream)),
           "cov_estimate_apertures")
    return out


def set_stage_events(events) -> None:
    """Instrumentation: record the given torch.cuda.Events (5, created) around
    the four kernels of each following recurrence call; None switches off."""
    lib = load()
    if events is None:
        _check(lib.cov_set_stage_events(None, 0), "cov_set_stage_events")
        return
    arr = (ctypes.c_void_p * len(events))(*[e.cuda_event for e in events])
    _check(lib.cov_set_stage_events(arr, len(events)), "cov_set_stage_events")


def tuning_get(dtype: str, N: int, M: int, P: int, Q: int):
    """(knobs planning uses now, whether they come from the tuning cache)."""
    t, cached = Tuning(), ctypes.c_int(0)
    _check(load().cov_tuning_get(DTYPES[dtype], N, M, P, Q, ctypes.byref(t), ctypes.byref(cached)),
           "cov_tuning_get")
    return t.as_dict(), bool(cached.value)


def tuning_set(dtype: str, N: int, M: int, P: int, Q: int, knobs: Optional[dict]) -> None:
    """Stores knobs for the shape in the tuning cache; None removes the entry."""
    t = None if knobs is None else ctypes.byref(Tuning(**knobs))
    _check(load().cov_tuning_set(DTYPES[dtype], N, M, P, Q, t), "cov_tuning_set")


def tuning_clear() -> None:
    load().cov_tuning_clear()


def tuning_save(path: str) -> None:
    _check(load().cov_tuning_save(os.fsencode(path)), "cov_tuning_save")


def tuning_load(path: str) -> int:
    n = ctypes.c_int(0)
    _check(load().cov_tuning_load(os.fsencode(path), ctypes.byref(n)), "cov_tuning_load")
    return int(n.value)


def autotune(A, P: int, Q: int, reps: int = 5, stream=None):
    """Times the combination path's candidate knobs on the device tensor A,
    caches the fastest for A's shape and returns (knobs, ms per call)."""
    torch = _torch()
    if not A.is_cuda or A.dim() != 2 or A.stride(1) != 1:
        raise ValueError("A must be a 2-D CUDA tensor with unit column stride")
    dt = _dtype_of(A)
    N, M = A.shape
    need = ctypes.c_size_t(0)
    _check(load().cov_autotune_workspace_size(DTYPES[dt], N, M, P, Q, ctypes.byref(need)),
           "cov_autotune_workspace_size")
    ws = torch.empty(max(int(need.value), 256), dtype=torch.uint8, device=A.device)
    R = torch.empty((P * Q, P * Q), dtype=A.dtype, device=A.device)
    best, ms = Tuning(), ctypes.c_float(0)
    _check(load().cov_autotune(A.data_ptr(), DTYPES[dt], N, M, A.stride(0), P, Q, R.data_ptr(),
                               ws.data_ptr(), ws.numel(), reps, _stream_ptr(stream),
                               ctypes.byref(best), ctypes.byref(ms)), "cov_autotune")
    return best.as_dict(), float(ms.value)


def selftest_timeout(workspace, limit_us: int = 20000, stream=None) -> None:
    """Queues the bounded-wait self-test kernel; its timeout is reported by the
    next check_device_status on the same workspace."""
    _check(load().cov_selftest_timeout(workspace.data_ptr(), workspace.numel(), limit_us,
                                       _stream_ptr(stream)), "cov_selftest_timeout")


def check_device_status(workspace, stream=None) -> None:
    """Raises CovError if a kernel recorded a device-side failure in workspace."""
    _check(load().cov_check_device_status(workspace.data_ptr(), _stream_ptr(stream)),
           "device status")


def capon_spectrum(R, steer, loading: float = 0.0, out=None, stream=None):
    """Minimum-variance (Capon) spectra P_k(f) = 1 / (a_f^H (R_k + d_k I)^{-1} a_f)
    of a batch of estimates R (CUDA complex64, (count, D, D) or (D, D)) for
    the steering vectors ``steer`` (CUDA complex64, (F, D)); d_k = loading
    trace(R_k) / D. Returns a (count, F) float32 CUDA tensor."""
    torch = _torch()
    if not (R.is_cuda and steer.is_cuda) or R.dtype != torch.complex64 or steer.dtype != torch.complex64:
        raise ValueError("R and steer must be complex64 CUDA tensors (no CPU fallback)")
    Rb = R if R.dim() == 3 else R.unsqueeze(0)
    if not Rb.is_contiguous() or Rb.shape[1] != Rb.shape[2]:
        raise ValueError("R must be contiguous (count, D, D)")
    st = steer.contiguous()
    count, D = Rb.shape[0], Rb.shape[1]
    if st.dim() != 2 or st.shape[1] != D:
        raise ValueError("steer must be (F, D)")
    F = st.shape[0]
    if out is None:
        out = torch.empty((count, F), dtype=torch.float32, device=R.device)
    _check(load().cov_capon_spectrum(Rb.data_ptr(), count, D, st.data_ptr(), F, float(loading),
                                     out.data_ptr(), _stream_ptr(stream)), "cov_capon_spectrum")
    return out if R.dim() == 3 else out[0]
