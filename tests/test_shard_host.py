"""Host logic of the sharded estimate, on CPU ranks.

The partition functions are checked against brute force and coverage
invariants; then world_size-2 process groups (gloo) run the sharded estimate
with each rank computing its own blocks through the oracle's element
function, and rank 0's assembly must equal the oracle's whole matrix. Fault
injection happens on the host only: a rank that exits without sending, a rank
that misses the deadline, and a rank whose shard is corrupted after its
checksum was taken. Each must be reported as a ShardError naming that rank.
"""
import itertools
import multiprocessing as mp
import os
import socket
import time

import numpy as np
import pytest

import cov_workloads as wl
from paper_1303_2285_gb300 import shard


# ---------------------------------------------------------------------------
# partitions
# ---------------------------------------------------------------------------
def _lag_costs(N, M, P, Q):
    # distinct products of each column lag's combinations (Eq. 3.3) plus a
    # fixed share of 2000 per combination, as the planner's cost states
    out = []
    for dc in range(Q):
        drs = range(0, P) if dc == 0 else range(-(P - 1), P)
        out.append(sum((N - abs(dr)) * (M - dc) + 2000 for dr in drs))
    return out


@pytest.mark.parametrize("N,M,P,Q,R", [(64, 64, 8, 8, 3), (100, 70, 5, 7, 2), (1024, 1024, 16, 16, 8),
                                       (40, 50, 3, 9, 4), (64, 64, 8, 8, 12), (33, 33, 4, 1, 2)])
def test_partition_lags_optimal_contiguous(N, M, P, Q, R):
    ranges, costs = shard.partition_lags(N, M, P, Q, R)
    assert ranges[0][0] == 0 and ranges[-1][1] == Q
    for (a, b), (c, d) in zip(ranges, ranges[1:]):
        assert b == c and a <= b
    lc = _lag_costs(N, M, P, Q)
    assert costs == [sum(lc[a:b]) for a, b in ranges]
    # brute force over every contiguous split into R ranges (small Q only)
    if Q <= 16 and R <= 8:
        best = None
        for cuts in itertools.combinations_with_replacement(range(Q + 1), R - 1):
            bounds = (0,) + cuts + (Q,)
            m = max(sum(lc[bounds[i]:bounds[i + 1]]) for i in range(R))
            best = m if best is None else min(best, m)
        assert max(costs) == best


def test_owned_blocks_cover_R_once():
    Q = 7
    ranges, _ = shard.partition_lags(50, 60, 4, Q, 3)
    seen = {}
    for lo, hi in ranges:
        for blk in shard.owned_blocks(Q, lo, hi):
            seen[blk] = seen.get(blk, 0) + 1
    assert seen == {(a, b): 1 for a in range(Q) for b in range(Q)}


def test_partition_matrices_lpt():
    shapes = wl.batched_shapes(300, 7)
    for n in (1, 2, 5, 16):
        rank_of, loads = shard.partition_matrices(shapes, n)
        assert len(rank_of) == len(shapes) and all(0 <= r < n for r in rank_of)
        cost = [shard_cost(*s) for s in shapes]
        got = [0] * n
        for c, r in zip(cost, rank_of):
            got[r] += c
        assert got == loads
        # Graham's bound for LPT: at most 4/3 - 1/(3n) of the optimum, and the
        # optimum is at least max(mean load, largest item)
        lower = max(sum(cost) / n, max(cost))
        assert max(loads) <= (4 / 3 - 1 / (3 * n)) * lower + 1


def shard_cost(N, M, P, Q):
    from oracle import combinations as cb
    return cb.um_enumerated(N, M, P, Q) + 2000 * cb.n_unique_combinations(P, Q) + 20000


@pytest.mark.parametrize("N,P,R", [(100, 5, 3), (10, 10, 2), (7, 3, 9), (256, 12, 8)])
def test_partition_rows_bands_and_halos(N, P, R):
    bands, halos = shard.partition_rows(N, P, R)
    assert bands[0][0] == 0 and bands[-1][1] == N
    for (a, b), (c, d) in zip(bands, bands[1:]):
        assert b == c
    for (lo, hi), (hl, hh) in zip(bands, halos):
        if lo == hi:
            continue
        # every window (rows p .. p+P-1, 0 <= p <= N-P) that covers a band row
        # lies inside the halo
        for n in range(lo, hi):
            for p in range(max(0, n - P + 1), min(N - P, n) + 1):
                assert hl <= p and p + P <= hh
        assert 0 <= hl <= lo and hi <= hh <= N


def test_encode_decode_and_corruption():
    P, Q = 3, 4
    R = wl.complex_normal((P * Q, P * Q), 3, dtype="c64")
    packed = shard.pack_blocks(R, P, Q, 1, 3)
    blob = shard.encode_shard(1, 1, 3, packed)
    back = shard.decode_shard(blob, P, 1, (1, 3))
    assert np.array_equal(back, packed)
    bad = bytearray(blob)
    bad[-1] ^= 0x01
    with pytest.raises(shard.ShardError) as e:
        shard.decode_shard(bytes(bad), P, 1, (1, 3))
    assert e.value.kind == "corrupted" and e.value.rank == 1
    with pytest.raises(shard.ShardError):
        shard.decode_shard(blob, P, 1, (0, 3))  # not the range the partition gave


# ---------------------------------------------------------------------------
# world_size-2 process groups
# ---------------------------------------------------------------------------
SHAPE = (24, 21, 4, 5)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _oracle_blocks(A, P, Q, lo, hi):
    import oracle
    D = P * Q
    R = np.zeros((D, D), np.complex128)
    for a, b in shard.owned_blocks(Q, lo, hi):
        for i in range(P):
            for j in range(P):
                R[a * P + i, b * P + j] = oracle.cov_element(A, P, Q, a * P + i, b * P + j)
    return shard.pack_blocks(R, P, Q, lo, hi)


def _rank_main(rank, world, port, fault, q):
    import torch.distributed as dist
    try:
        import torch
        store = dist.TCPStore("127.0.0.1", port, world, rank == 0,
                              timeout=__import__("datetime").timedelta(seconds=30))
        dist.init_process_group("gloo", store=dist.PrefixStore("pg", store), rank=rank,
                                world_size=world)
        # every rank plans the same partition
        N, M, P, Q = SHAPE
        plan = [None] * world
        dist.all_gather_object(plan, shard.partition_lags(N, M, P, Q, world)[0])
        assert all(p == plan[0] for p in plan)
        A = wl.complex_normal((N, M), 99, dtype="c128")

        def compute(lo, hi):
            packed = _oracle_blocks(A, P, Q, lo, hi)
            if rank == 1 and fault == "die":
                os._exit(0)  # leaves without sending and without the barrier
            if rank == 1 and fault == "late":
                time.sleep(4.0)
            return packed

        if rank == 1 and fault == "corrupt":
            ranges, _ = shard.partition_lags(N, M, P, Q, world)
            lo, hi = ranges[rank]
            blob = bytearray(shard.encode_shard(rank, lo, hi, compute(lo, hi)))
            blob[-3] ^= 0x40  # after the checksum was taken
            store.set(f"cov/{rank}", bytes(blob))
            q.put((rank, "sent"))
            time.sleep(3.0)  # keep the store's clients alive while rank 0 reads
            return
        out = shard.run_rank(store, rank, world, N, M, P, Q, compute, tag="cov",
                             timeout_s=1.5 if fault else 30.0)
        if rank == 0:
            import oracle
            want = oracle.cov_window(A, P, Q)
            q.put((0, "equal" if np.array_equal(out, want) else "differs"))
        else:
            q.put((rank, "sent"))
        if not fault:
            dist.barrier()
            dist.destroy_process_group()
    except shard.ShardError as e:
        q.put((rank, f"ShardError:{e.kind}:{e.rank}"))
    except Exception as e:  # noqa: BLE001 - reported to the parent
        q.put((rank, f"error:{type(e).__name__}:{e}"))


def _run_world(fault, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, fault, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    deadline = time.monotonic() + 120
    while len(res) < world and time.monotonic() < deadline:
        try:
            r, msg = q.get(timeout=1.0)
            res[r] = msg
        except Exception:  # noqa: BLE001 - queue.Empty
            if fault == "die" and 0 in res:
                break
    for p in procs:
        p.join(timeout=30)
        if p.is_alive():
            p.kill()
            p.join()
    return res


def test_two_ranks_assemble_oracle():
    res = _run_world(None)
    assert res == {0: "equal", 1: "sent"}


@pytest.mark.parametrize("fault,kind", [("die", "missing"), ("late", "missing"),
                                        ("corrupt", "corrupted")])
def test_two_ranks_fault_detected(fault, kind):
    res = _run_world(fault)
    assert res.get(0) == f"ShardError:{kind}:1"


# ---------------------------------------------------------------------------
# the collective exchange (one all-gather of padded packed blocks), on gloo
# ---------------------------------------------------------------------------
def _rank_allgather(rank, world, port, q):
    import torch
    import torch.distributed as dist
    try:
        dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                                world_size=world)
        N, M, P, Q = SHAPE
        ranges, _ = shard.partition_lags(N, M, P, Q, world)
        A = wl.complex_normal((N, M), 99, dtype="c128")
        D = P * Q
        R = np.full((D, D), np.nan + 0j, np.complex128)
        lo, hi = ranges[rank]
        shard.unpack_blocks(R, _oracle_blocks(A, P, Q, lo, hi), P, Q, lo, hi)
        Rt = torch.from_numpy(R)
        shard.allgather_blocks(Rt, P, Q, ranges, rank, pack=shard.host_pack,
                               unpack=shard.host_unpack)
        import oracle
        q.put((rank, "equal" if np.array_equal(Rt.numpy(), oracle.cov_window(A, P, Q))
               else "differs"))
        dist.barrier()
        dist.destroy_process_group()
    except Exception as e:  # noqa: BLE001 - reported to the parent
        q.put((rank, f"error:{type(e).__name__}:{e}"))


@pytest.mark.parametrize("world", [2, 3])
def test_allgather_of_packed_blocks_assembles_R_on_every_rank(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_allgather, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    deadline = time.monotonic() + 120
    while len(res) < world and time.monotonic() < deadline:
        try:
            r, msg = q.get(timeout=1.0)
            res[r] = msg
        except Exception:  # noqa: BLE001 - queue.Empty
            pass
    for p in procs:
        p.join(timeout=30)
        if p.is_alive():
            p.kill()
            p.join()
    assert res == {r: "equal" for r in range(world)}


def test_packed_sizes_match_the_layout():
    lib = __import__("paper_1303_2285_gb300").load()
    import ctypes
    for P, Q in ((4, 5), (16, 16), (1, 7), (9, 1)):
        for lo in range(Q + 1):
            for hi in range(lo, Q + 1):
                n = ctypes.c_size_t(0)
                assert lib.cov_shard_packed_size(0, P, Q, lo, hi, ctypes.byref(n)) == 0
                assert n.value == 8 * shard.packed_elements(P, Q, lo, hi)
    n = ctypes.c_size_t(0)
    assert lib.cov_shard_packed_size(0, 4, 5, 3, 2, ctypes.byref(n)) == 1  # empty-reversed range
    assert lib.cov_shard_packed_size(0, 4, 5, 0, 6, ctypes.byref(n)) == 1  # past Q
