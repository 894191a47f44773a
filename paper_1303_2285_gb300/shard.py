"""Sharding of the covariance estimate across processes (one per GPU).

Section 4.2 gives every combination (dr, dc) its own outputs of R
(Eq. 3.7-3.8), so ranks that own disjoint sets of combinations write
disjoint parts of R: the only exchange is a gather of those parts, with no
reduction. The shard unit is a column lag dc, whose combinations own the
P x P blocks (a, b) of R with |b - a| = dc. Every rank needs all of A.

This module holds the host logic: the partition (through the C ABI's
planner), packing a rank's blocks with a CRC-32 checksum, the gather through
a ``torch.distributed`` key-value store with a deadline, and the assembly on
rank 0. A rank that dies, misses the deadline or sends a corrupted shard is
reported by name (``ShardError``); nothing waits without a limit.
"""
from __future__ import annotations

import ctypes
import struct
import time
import zlib
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np

from . import CovDesc, DTYPES, NORMS, _check, _dtype_of, _stream_ptr, load, workspace_size

_HDR = struct.Struct("<4sIIqqII")  # magic, rank, crc32, dc_lo, dc_hi, nbytes, dtype code
_MAGIC = b"CVSH"


class ShardError(RuntimeError):
    """A shard is missing, late or corrupted."""

    def __init__(self, kind: str, rank: int, detail: str):
        self.kind, self.rank = kind, rank
        super().__init__(f"shard of rank {rank}: {kind} ({detail})")


# ---------------------------------------------------------------------------
# partitions (C ABI planner)
# ---------------------------------------------------------------------------
def partition_lags(N: int, M: int, P: int, Q: int, n_ranks: int):
    """[(dc_lo, dc_hi)] per rank (contiguous, covering [0, Q)) and the costs."""
    b = (ctypes.c_int32 * (n_ranks + 1))()
    c = (ctypes.c_int64 * n_ranks)()
    _check(load().cov_partition_lags(N, M, P, Q, n_ranks, b, c), "cov_partition_lags")
    return [(b[r], b[r + 1]) for r in range(n_ranks)], list(c)


def partition_matrices(shapes: Sequence[Tuple[int, int, int, int]], n_ranks: int):
    """Rank of each (N, M, P, Q) matrix (LPT by cost) and the per-rank costs."""
    descs = (CovDesc * len(shapes))()
    for i, (N, M, P, Q) in enumerate(shapes):
        descs[i].N, descs[i].M, descs[i].P, descs[i].Q = N, M, P, Q
        descs[i].lda = M
    rank_of = (ctypes.c_int32 * len(shapes))()
    c = (ctypes.c_int64 * n_ranks)()
    _check(load().cov_partition_matrices(descs, len(shapes), n_ranks, rank_of, c),
           "cov_partition_matrices")
    return list(rank_of), list(c)


def partition_rows(N: int, P: int, n_ranks: int):
    """Adjoint: [(row_lo, row_hi)] bands of dA and [(halo_lo, halo_hi)] rows of A."""
    b = (ctypes.c_int64 * (n_ranks + 1))()
    lo = (ctypes.c_int64 * n_ranks)()
    hi = (ctypes.c_int64 * n_ranks)()
    _check(load().cov_partition_rows(N, P, n_ranks, b, lo, hi), "cov_partition_rows")
    return [(b[r], b[r + 1]) for r in range(n_ranks)], [(lo[r], hi[r]) for r in range(n_ranks)]


# ---------------------------------------------------------------------------
# blocks of R owned by a range of column lags
# ---------------------------------------------------------------------------
def owned_blocks(Q: int, dc_lo: int, dc_hi: int) -> List[Tuple[int, int]]:
    """Blocks (a, b) with dc_lo <= |b - a| < dc_hi, in a fixed order."""
    out = []
    for dc in range(dc_lo, dc_hi):
        for a in range(Q - dc):
            out.append((a, a + dc))
            if dc > 0:
                out.append((a + dc, a))
    return out


def pack_blocks(R: np.ndarray, P: int, Q: int, dc_lo: int, dc_hi: int) -> np.ndarray:
    """The shard's blocks of R, concatenated (len(blocks) x P x P)."""
    blocks = owned_blocks(Q, dc_lo, dc_hi)
    out = np.empty((len(blocks), P, P), dtype=R.dtype)
    for k, (a, b) in enumerate(blocks):
        out[k] = R[a * P:(a + 1) * P, b * P:(b + 1) * P]
    return out


def unpack_blocks(R: np.ndarray, packed: np.ndarray, P: int, Q: int, dc_lo: int, dc_hi: int):
    for k, (a, b) in enumerate(owned_blocks(Q, dc_lo, dc_hi)):
        R[a * P:(a + 1) * P, b * P:(b + 1) * P] = packed[k]


def encode_shard(rank: int, dc_lo: int, dc_hi: int, packed: np.ndarray) -> bytes:
    payload = np.ascontiguousarray(packed).tobytes()
    code = 1 if packed.dtype == np.complex128 else 0
    return _HDR.pack(_MAGIC, rank, zlib.crc32(payload), dc_lo, dc_hi, len(payload), code) + payload


def decode_shard(blob: bytes, P: int, expect_rank: int, expect_range: Tuple[int, int]):
    if len(blob) < _HDR.size:
        raise ShardError("corrupted", expect_rank, "short message")
    magic, rank, crc, lo, hi, n, code = _HDR.unpack_from(blob)
    payload = blob[_HDR.size:]
    if magic != _MAGIC or rank != expect_rank or (lo, hi) != tuple(expect_range):
        raise ShardError("corrupted", expect_rank, "header does not match the partition")
    if len(payload) != n or zlib.crc32(payload) != crc:
        raise ShardError("corrupted", expect_rank, "checksum mismatch")
    dt = np.complex128 if code == 1 else np.complex64
    return np.frombuffer(payload, dtype=dt).reshape(-1, P, P)


# ---------------------------------------------------------------------------
# gather through a key-value store (torch.distributed.TCPStore or any Store)
# ---------------------------------------------------------------------------
def gather_shards(store, rank: int, world: int, tag: str, blob: bytes, P: int,
                  ranges: Sequence[Tuple[int, int]], timeout_s: float = 30.0,
                  poll_s: float = 0.01) -> Optional[list]:
    """Every rank publishes its encoded shard; rank 0 collects all of them
    within ``timeout_s`` and returns the decoded blocks per rank (None on the
    other ranks). Raises ShardError naming the first missing or corrupted
    rank."""
    store.set(f"{tag}/{rank}", blob)
    if rank != 0:
        return None
    deadline = time.monotonic() + timeout_s
    out: list = [None] * world
    pending = set(range(world))
    while pending:
        for r in sorted(pending):
            if store.check([f"{tag}/{r}"]):
                out[r] = decode_shard(store.get(f"{tag}/{r}"), P, r, ranges[r])
                pending.discard(r)
        if pending:
            if time.monotonic() > deadline:
                r = min(pending)
                raise ShardError("missing", r, f"no shard within {timeout_s} s")
            time.sleep(poll_s)
    return out


def assemble(P: int, Q: int, ranges: Sequence[Tuple[int, int]], shards: Sequence[np.ndarray],
             dtype=np.complex64) -> np.ndarray:
    D = P * Q
    R = np.full((D, D), np.nan, dtype=dtype)
    for (lo, hi), packed in zip(ranges, shards):
        unpack_blocks(R, packed, P, Q, lo, hi)
    return R


# ---------------------------------------------------------------------------
# gather through one collective (NCCL for device tensors, gloo on the host)
# ---------------------------------------------------------------------------
def packed_elements(P: int, Q: int, dc_lo: int, dc_hi: int) -> int:
    """Complex elements of a lag range's packed blocks (len(owned_blocks) P^2)."""
    return len(owned_blocks(Q, dc_lo, dc_hi)) * P * P


def device_pack(R, P: int, Q: int, dc_lo: int, dc_hi: int, out, stream=None) -> None:
    """The library's pack kernel: R's blocks of [dc_lo, dc_hi) into `out`
    (device tensors of R's dtype, `out` with packed_elements(...) entries)."""
    if not (R.is_cuda and out.is_cuda):
        raise ValueError("device tensors expected (no CPU fallback)")
    _check(load().cov_shard_pack(R.data_ptr(), DTYPES[_dtype_of(R)], P, Q, dc_lo, dc_hi,
                                 out.data_ptr(), _stream_ptr(stream)), "cov_shard_pack")


def device_unpack(packed, R, P: int, Q: int, dc_lo: int, dc_hi: int, stream=None) -> None:
    if not (R.is_cuda and packed.is_cuda):
        raise ValueError("device tensors expected (no CPU fallback)")
    _check(load().cov_shard_unpack(packed.data_ptr(), DTYPES[_dtype_of(R)], P, Q, dc_lo, dc_hi,
                                   R.data_ptr(), _stream_ptr(stream)), "cov_shard_unpack")


def host_pack(R, P: int, Q: int, dc_lo: int, dc_hi: int, out) -> None:
    """The same layout on host tensors (for CPU process groups)."""
    import torch
    out.copy_(torch.from_numpy(pack_blocks(R.numpy(), P, Q, dc_lo, dc_hi).reshape(-1)))


def host_unpack(packed, R, P: int, Q: int, dc_lo: int, dc_hi: int) -> None:
    Rn = R.numpy()
    unpack_blocks(Rn, packed.numpy().reshape(-1, P, P), P, Q, dc_lo, dc_hi)


def allgather_blocks(R, P: int, Q: int, ranges: Sequence[Tuple[int, int]], rank: int,
                     group=None, pack=None, unpack=None, scratch=None):
    """Every rank holds its own blocks of R (the lag range ranges[rank]); after
    this call every rank holds all of R. One all-gather of equal-size packed
    buffers (each rank's blocks, zero-padded to the largest share); `pack`
    and `unpack` default to the library's kernels (device tensors); pass
    host_pack / host_unpack for host tensors on a CPU process group.
    `scratch` may hold (send, recv) buffers from an earlier call."""
    import torch
    import torch.distributed as dist
    pack = pack or device_pack
    unpack = unpack or device_unpack
    world = len(ranges)
    sizes = [packed_elements(P, Q, lo, hi) for lo, hi in ranges]
    mx = max(sizes)
    if scratch is None:
        send = torch.zeros(mx, dtype=R.dtype, device=R.device)
        recv = [torch.empty(mx, dtype=R.dtype, device=R.device) for _ in range(world)]
    else:
        send, recv = scratch
    lo, hi = ranges[rank]
    if sizes[rank]:
        pack(R, P, Q, lo, hi, send[:sizes[rank]])
    # collectives carry the real and imaginary parts as a real tensor
    dist.all_gather([torch.view_as_real(x) for x in recv], torch.view_as_real(send), group=group)
    for r, (lo_r, hi_r) in enumerate(ranges):
        if r != rank and sizes[r]:
            unpack(recv[r][:sizes[r]], R, P, Q, lo_r, hi_r)
    return send, recv


# ---------------------------------------------------------------------------
# the device side of one rank
# ---------------------------------------------------------------------------
def estimate_shard_into(A, R, P: int, Q: int, dc_lo: int, dc_hi: int, norm: str = "mean",
                        workspace=None, stream=None):
    """Writes the blocks of the column lags [dc_lo, dc_hi) of R (device
    tensors); the rest of R is left as it was."""
    import torch
    if not (A.is_cuda and R.is_cuda):
        raise ValueError("A and R must be CUDA tensors (no CPU fallback)")
    if A.dim() != 2 or A.stride(1) != 1:
        raise ValueError("A must be 2-D with unit column stride")
    dt = _dtype_of(A)
    if R.dtype != A.dtype or not R.is_contiguous() or tuple(R.shape) != (P * Q, P * Q):
        raise ValueError("R must be a contiguous PQ x PQ tensor of A's dtype")
    N, M = A.shape
    need = workspace_size(dt, N, M, P, Q, "recurrence")
    if workspace is None:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=A.device)
    _check(load().cov_estimate_shard(A.data_ptr(), DTYPES[dt], N, M, A.stride(0), P, Q, dc_lo,
                                     dc_hi, R.data_ptr(), NORMS[norm], workspace.data_ptr(),
                                     workspace.numel(), _stream_ptr(stream)),
           "cov_estimate_shard")
    return R


def run_rank(store, rank: int, world: int, N: int, M: int, P: int, Q: int,
             compute: Callable[[int, int], np.ndarray], tag: str = "cov",
             timeout_s: float = 30.0) -> Optional[np.ndarray]:
    """One rank of a sharded estimate: partition, ``compute(dc_lo, dc_hi)``
    (returns the packed blocks of the rank's lags), gather, and on rank 0 the
    assembled R (None elsewhere)."""
    ranges, _ = partition_lags(N, M, P, Q, world)
    lo, hi = ranges[rank]
    packed = compute(lo, hi)
    blob = encode_shard(rank, lo, hi, packed)
    shards = gather_shards(store, rank, world, tag, blob, P, ranges, timeout_s)
    if shards is None:
        return None
    return assemble(P, Q, ranges, shards, dtype=packed.dtype)
