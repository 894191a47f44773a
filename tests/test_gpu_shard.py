"""The per-rank device work of the sharded estimate, on one GPU.

Each shard of a partition runs in turn (nothing waits on another shard) into
an R prefilled with NaN: a shard must write exactly its blocks, bit-identical
to the unsharded call, and leave every other element untouched; the shards
together must give the whole matrix. The adjoint's row bands are checked the
same way against the unsharded gradient."""
import numpy as np
import pytest
import torch

import cov_workloads as wl
import paper_1303_2285_gb300 as cov
from paper_1303_2285_gb300 import shard

pytestmark = pytest.mark.gpu

from gpu_util import oracle_R, rel_fro, to_dev  # noqa: E402


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("N,M,P,Q,ranks", [(300, 101, 7, 5, 2), (200, 150, 16, 16, 3),
                                           (95, 95, 32, 32, 8), (64, 64, 8, 8, 12),
                                           (1024, 1024, 16, 16, 8)])
def test_shards_write_exactly_their_blocks(oracle_mod, dtype, N, M, P, Q, ranks):
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    A_np = wl.complex_normal((N, M), 7 + N + Q, dtype=dtype)
    A = to_dev(A_np, tdt)
    D = P * Q
    full = cov.estimate(A, P, Q, algo="recurrence").cpu().numpy()
    ranges, _ = shard.partition_lags(N, M, P, Q, ranks)
    ws = torch.empty(cov.workspace_size(dtype, N, M, P, Q, "recurrence"), dtype=torch.uint8,
                     device="cuda")
    pieces = []
    for lo, hi in ranges:
        R = torch.full((D, D), float("nan"), dtype=tdt, device="cuda")
        shard.estimate_shard_into(A, R, P, Q, lo, hi, workspace=ws)
        torch.cuda.synchronize()
        cov.check_device_status(ws)
        Rn = R.cpu().numpy()
        mask = np.zeros((D, D), bool)
        for a, b in shard.owned_blocks(Q, lo, hi):
            mask[a * P:(a + 1) * P, b * P:(b + 1) * P] = True
        assert np.all(np.isnan(Rn[~mask])), "a shard wrote outside its blocks"
        assert np.array_equal(Rn[mask], full[mask]), "shard differs from the unsharded call"
        pieces.append(shard.pack_blocks(Rn, P, Q, lo, hi))
    R_all = shard.assemble(P, Q, ranges, pieces, dtype=full.dtype)
    assert np.array_equal(R_all, full)
    if N * M * D * D <= 4e9:
        tol = 1e-5 if dtype == "c64" else 1e-12
        assert rel_fro(R_all, oracle_R(oracle_mod, A_np, P, Q)) < tol


def test_empty_shard_touches_nothing():
    N, M, P, Q = 64, 64, 4, 4
    A = to_dev(wl.complex_normal((N, M), 1, dtype="c64"), torch.complex64)
    R = torch.full((P * Q, P * Q), float("nan"), dtype=torch.complex64, device="cuda")
    shard.estimate_shard_into(A, R, P, Q, 2, 2)
    torch.cuda.synchronize()
    assert torch.isnan(R.real).all()


@pytest.mark.parametrize("N,M,P,Q,ranks", [(40, 33, 5, 4, 3), (64, 70, 12, 12, 4), (20, 17, 4, 3, 7)])
@pytest.mark.parametrize("norm", ["mean", "sum"])
def test_adjoint_row_bands(N, M, P, Q, ranks, norm):
    A = to_dev(wl.complex_normal((N, M), 21 + N, dtype="c64"), torch.complex64)
    G = to_dev(wl.complex_normal((P * Q, P * Q), 22, dtype="c64"), torch.complex64)
    full = cov.estimate_backward(A, G, P, Q, norm=norm).cpu().numpy()
    K = (N - P + 1) * (M - Q + 1)
    Gs = G / K if norm == "mean" else G
    bands, halos = shard.partition_rows(N, P, ranks)
    got = np.full((N, M), np.nan, np.complex64)
    for (lo, hi), (hl, hh) in zip(bands, halos):
        if lo == hi:
            continue
        sub = A[hl:hh].contiguous()
        dA = cov.estimate_backward(sub, Gs.contiguous(), P, Q, norm="sum").cpu().numpy()
        got[lo:hi] = dA[lo - hl:hi - hl]
    assert not np.isnan(got).any()
    assert rel_fro(got, full) < 1e-5


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("P,Q,ranks", [(7, 5, 2), (16, 16, 3), (32, 32, 8), (4, 1, 2)])
def test_device_pack_unpack_assembles_R(dtype, P, Q, ranks):
    # the library's pack kernel must give the host layout (shard.pack_blocks)
    # bit for bit, and unpacking every rank's packed blocks into a NaN-filled
    # R must rebuild the unsharded estimate
    N, M = 2 * P + 40, 2 * Q + 33
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    A = to_dev(wl.complex_normal((N, M), 11 + P * Q, dtype=dtype), tdt)
    full = cov.estimate(A, P, Q, algo="recurrence")
    ranges, _ = shard.partition_lags(N, M, P, Q, ranks)
    D = P * Q
    out = torch.full((D, D), complex(np.nan, np.nan), dtype=tdt, device="cuda")
    for lo, hi in ranges:
        buf = torch.full((shard.packed_elements(P, Q, lo, hi),), complex(np.nan, np.nan),
                         dtype=tdt, device="cuda")
        shard.device_pack(full, P, Q, lo, hi, buf)
        torch.cuda.synchronize()
        want = shard.pack_blocks(full.cpu().numpy(), P, Q, lo, hi).reshape(-1)
        assert np.array_equal(buf.cpu().numpy(), want)
        shard.device_unpack(buf, out, P, Q, lo, hi)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), full.cpu().numpy())


def test_nccl_allgather_of_one_rank_round_trips():
    # the collective path of the sharded bench (NCCL, complex viewed as real)
    # with a one-rank group: the rank's own blocks come back untouched
    import datetime
    import socket
    import torch.distributed as dist
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    store = dist.TCPStore("127.0.0.1", port, 1, True, timeout=datetime.timedelta(seconds=30))
    pg_was = dist.is_initialized()
    if not pg_was:
        dist.init_process_group("nccl", store=store, rank=0, world_size=1)
    try:
        N, M, P, Q = 120, 90, 8, 6
        A = to_dev(wl.complex_normal((N, M), 5, dtype="c64"), torch.complex64)
        want = cov.estimate(A, P, Q, algo="recurrence")
        ranges, _ = shard.partition_lags(N, M, P, Q, 1)
        R = torch.full_like(want, complex(np.nan, np.nan))
        shard.estimate_shard_into(A, R, P, Q, *ranges[0])
        shard.allgather_blocks(R, P, Q, ranges, 0)
        torch.cuda.synchronize()
        assert np.array_equal(R.cpu().numpy(), want.cpu().numpy())
    finally:
        if not pg_was:
            dist.destroy_process_group()
