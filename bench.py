#!/usr/bin/env python3
"""Benchmark of the covariance-method hot path on GB300.

Prints ONE JSON line. A step is one call of the combination path
(COV_RECURRENCE) on the bench workload, by default the largest single-GPU
one: the 2048 x 512 SAR-like complex64 input with a 32 x 32 window (R is
1024 x 1024). The step covers the plan, the staging of A, every distinct
product, the seeds, the diagonal walk and the write of R. Inputs are resident
in HBM when the timed region starts; L2 is flushed (256 MiB write) before
every timed step, outside the timed events.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

--impl reference times the CPU oracle (the plain FP64 window loop) on the
host cores, on a bounded sample of the same workload.
Under torchrun each rank computes its own matrix (independent problems, no
data-path collective): weak scaling, value = all ranks' products / max time.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "R elements/s and distinct products/s vs plain FP64 GPU path; % roofline; err vs FP64"
UNIT = "distinct products/s"
DEFAULT_WORKLOAD = "sar_2048x512_w32_f32"
GEMM_WORKLOAD = "cn_1024x1024_w16_f32"
FLUSH_BYTES = 256 << 20
FP32_LANES_PER_SM = 128   # FP32 FMA lanes per SM (4 SMSPs x 32)
FALLBACK_SM_MAX_MHZ = 2070.0
FALLBACK_HBM_GBS = 6800.0

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of
# the production kernel from one ncu capture (profiles/), keyed by (workload,
# kernel, hash of the combination path's kernel sources at capture time):
# null once those sources have changed.
NCU_TRAFFIC = {  # bytes per launch; profiles/launches_*.md, profiles/k_products_inner_*.md
    ("cn_1024x1024_w16_f32", "k_fused", "96da72e2c97e5ecd"): 8561408,
    ("cn_1024x1024_w16_f32", "k_products_inner", "96da72e2c97e5ecd"): 8438016,
    ("sar_2048x512_w32_f32", "k_products_inner", "e46608b38ef1696e"): 8582400,
}
KERNEL_SOURCES = ("cov_device.cuh", "cov_internal.h", "rec_common.cuh", "rec_products.cuh",
                  "rec_products.cu", "rec_fringe.cuh", "rec_fringe.cu", "rec_reduce.cuh",
                  "rec_reduce.cu", "rec_fused.cu", "recurrence.cu", "plan.cpp", "plan.h")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1303_2285_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def parse_knobs(text: str) -> dict:
    """"G,TRB,L,K[,TC]" -> the combination path's tuning knobs."""
    v = [int(x) for x in text.split(",")]
    if len(v) not in (4, 5):
        raise ValueError("--knobs wants G,TRB,L,K or G,TRB,L,K,TC")
    names = ("lag_group", "rows_per_task", "reseed_interval", "kernels", "tile_cols")
    return dict(zip(names, v + [0] * (5 - len(v))))


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


class Cudart:
    """cudaMemsetAsync / cudaMemcpyAsync through ctypes: the timed loops issue
    their L2 flushes and host<->device copies without framework overhead."""
    H2D, D2H = 1, 2

    def __init__(self):
        import ctypes
        import ctypes.util
        cands = ["libcudart.so", "libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so",
                 ctypes.util.find_library("cudart") or ""]
        self.lib = None
        for c in cands:
            if not c:
                continue
            try:
                self.lib = ctypes.CDLL(c)
                break
            except OSError:
                continue
        if self.lib is None:
            raise RuntimeError("libcudart not found")
        vp, sz = ctypes.c_void_p, ctypes.c_size_t
        self.lib.cudaMemsetAsync.argtypes = [vp, ctypes.c_int, sz, vp]
        self.lib.cudaMemsetAsync.restype = ctypes.c_int
        self.lib.cudaMemcpyAsync.argtypes = [vp, vp, sz, ctypes.c_int, vp]
        self.lib.cudaMemcpyAsync.restype = ctypes.c_int

    def memset(self, ptr, value, nbytes, stream) -> int:
        return self.lib.cudaMemsetAsync(ptr, value, nbytes, stream)

    def memcpy(self, dst, src, nbytes, kind, stream) -> int:
        return self.lib.cudaMemcpyAsync(dst, src, nbytes, kind, stream)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, gpu_index: int) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            with open(self.path) as f:
                for line in f:
                    c = [x.strip() for x in line.split(",")]
                    if len(c) < 9 or c[0] != str(gpu_index):
                        continue
                    try:
                        sm.append(float(c[1]))
                        smax.append(float(c[2]))
                    except ValueError:
                        continue
                    for k, nm in enumerate(names):
                        if c[5 + k].lower().startswith("active"):
                            reasons.add(nm)
            os.unlink(self.path)
        except Exception:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# CPU baseline leg: the oracle, as it stands, on the host cores. The only part
# of this file that runs anything under oracle/.
# ---------------------------------------------------------------------------
def cpu_baseline_leg(A_np, P, Q, um_full, K_full, budget_s: float, gpu_check=None,
                     rows=None, single_thread=False, R_gpu_full=None) -> dict:
    """Times the oracle on the first `rows` rows of A (chosen to take about
    budget_s when None) and extrapolates to the full job by window count.
    With R_gpu_full (the GPU's R of the whole input, host), also compares it
    element by element with the oracle's full R (the Gram form of Eq. 2.2,
    FP64; untimed)."""
    import numpy as np

    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    N, M = A_np.shape

    def run(r, nthreads=threads):
        t0 = time.perf_counter()
        R = oracle.cov_window(A_np[:r], P, Q, threads=nthreads)
        return time.perf_counter() - t0, R

    if rows is None:
        rows = calibrate_rows(A_np, P, Q, budget_s, run)
    t, R_s = run(rows)
    k_s = (rows - P + 1) * (M - Q + 1)
    t_full = t * K_full / k_s
    out = {"value": um_full / t_full, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": (f"first {rows} of {N} rows of the same input ({k_s} of {K_full} window "
                      f"positions), full-job time extrapolated by window count"),
           "sample_seconds": round(t, 3), "rows": rows}
    if single_thread and threads > 1:
        # The same oracle on one core (its threaded form splits rows of R with the
        # same per-element order, so both give the same R), sampled for a quarter of the budget.
        def run1(r):
            return run(r, 1)
        rows1 = calibrate_rows(A_np, P, Q, budget_s / 4, run1)
        t1, _ = run1(rows1)
        k1 = (rows1 - P + 1) * (M - Q + 1)
        out["single_thread"] = {
            "value": um_full / (t1 * K_full / k1), "unit": UNIT, "cores": 1,
            "sample": f"first {rows1} of {N} rows ({k1} window positions)",
            "sample_seconds": round(t1, 3)}
    if R_gpu_full is not None:
        from oracle.gram import cov_gram
        t0 = time.perf_counter()
        Ro = cov_gram(A_np, P, Q)
        to = time.perf_counter() - t0
        Rg = np.asarray(R_gpu_full).astype(np.complex128)
        out["gpu_err_vs_oracle_full_R"] = {
            "rel_fro": float(np.linalg.norm(Rg - Ro) / np.linalg.norm(Ro)),
            "max_abs_rel_to_max": float(np.abs(Rg - Ro).max() / np.abs(Ro).max()),
            "elements": int(Ro.size),
            "oracle": "oracle.gram.cov_gram: Eq. 2.2 as X X^H over all window positions, FP64 (BLAS zherk)",
            "oracle_seconds": round(to, 2)}
    if gpu_check is not None:
        G = gpu_check(A_np[:rows])
        err = float(np.linalg.norm(G - R_s) / np.linalg.norm(R_s))
        out["gpu_rel_fro_err_on_sample"] = err
        out["gpu_max_abs_err_rel_to_max_on_sample"] = float(np.abs(G - R_s).max() / np.abs(R_s).max())
    return out


def calibrate_rows(A_np, P, Q, budget_s, run) -> int:
    N, M = A_np.shape
    rows = min(N, P + 7)
    t, _ = run(rows)
    per_window = t / ((rows - P + 1) * (M - Q + 1))
    want_k = max(1, int(budget_s / max(per_window, 1e-9)))
    return int(min(N, max(P, P - 1 + want_k // (M - Q + 1))))


def bench_reference(args, rank, world):
    """The oracle as it stands on the host cores. One step = one oracle call on
    a fixed sample of the workload (its first rows), so that every timed step
    really runs and the whole run takes a minute or two; value = the full
    job's distinct products per second, the sample's time scaled by window
    count (the oracle's cost is proportional to the windows it visits)."""
    import oracle
    import cov_workloads as wl
    if rank != 0:
        return 0
    oracle.build()
    w = wl.WORKLOADS[args.workload]
    A_np = wl.workload_input(w)
    um = _um(w)
    threads = os.cpu_count() or 1
    per_step = min(4.0, 90.0 / max(1, args.steps + args.warmup))

    def run(r, nthreads=threads):
        t0 = time.perf_counter()
        R = oracle.cov_window(A_np[:r], w.P, w.Q, threads=nthreads)
        return time.perf_counter() - t0, R

    rows = calibrate_rows(A_np, w.P, w.Q, per_step, run)
    k_s = (rows - w.P + 1) * (w.M - w.Q + 1)
    times = []
    wall0 = time.perf_counter()
    for k in range(args.warmup + args.steps):
        t, _ = run(rows)
        if k >= args.warmup:
            times.append(t)
    wall = time.perf_counter() - wall0
    t_step = statistics.mean(times)
    value = um * (k_s / w.K) / t_step
    sample = (f"first {rows} of {w.N} rows of the same input ({k_s} of {w.K} window positions) "
              f"per step; value scales the step time to the full job by window count")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(w),
            "step_definition": "one oracle call on the sample below (all steps run; none is extrapolated)",
            "full_job_ms_extrapolated": t_step * (w.K / k_s) * 1e3,
            "wall_s_incl_warmup": wall,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _um(w):
    from oracle import combinations as cb  # counting only
    return cb.um_enumerated(w.N, w.M, w.P, w.Q)


def _config(w):
    return {"workload": w.name, "N": w.N, "M": w.M, "P": w.P, "Q": w.Q, "K": w.K,
            "input": {"cn": "i.i.d. CN(0,1)", "sar": "8 complex exponentials + noise at 10 dB SNR",
                      "int": "integer-valued"}[w.kind] + f", seed {w.seed}",
            "l2": "flushed before every timed step (256 MiB write, outside the timed events)"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def bench_sharded(args, rank, world, local):
    """One matrix split across the ranks by column lag (Section 4.2: the
    combinations of a lag range own whole blocks of R, so no reduction is
    needed). A step: every rank computes its lags' blocks
    (cov_estimate_shard), packs them (cov_shard_pack), one NCCL all-gather of
    the packed blocks, and every rank unpacks the others' (cov_shard_unpack),
    so that each ends with all of R. Strong scaling: the total work is one
    matrix whatever the rank count; value = its distinct products / max over
    ranks of the step time."""
    import datetime
    import socket

    import numpy as np
    import torch
    import torch.distributed as dist

    import cov_workloads as wl
    import paper_1303_2285_gb300 as cov
    from paper_1303_2285_gb300 import shard

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:  # the same NCCL collective with a one-rank group
        with socket.socket() as so:
            so.bind(("127.0.0.1", 0))
            port = so.getsockname()[1]
        store = dist.TCPStore("127.0.0.1", port, 1, True, timeout=datetime.timedelta(seconds=60))
        dist.init_process_group("nccl", store=store, rank=0, world_size=1,
                                device_id=torch.device("cuda", local))
    w = wl.WORKLOADS[args.workload]
    dt = torch.complex64 if w.dtype == "c64" else torch.complex128
    A_np = wl.workload_input(w)  # every rank holds all of A (the same input)
    A = torch.from_numpy(A_np).cuda()
    D = w.P * w.Q
    R = torch.empty((D, D), dtype=dt, device="cuda")
    um = cov.plan_info(w.N, w.M, w.P, w.Q)["distinct_products"]
    if args.knobs:
        cov.tuning_set(w.dtype, w.N, w.M, w.P, w.Q, parse_knobs(args.knobs))
    elif args.autotune:
        cov.autotune(A, w.P, w.Q, reps=5)
    knobs, _ = cov.tuning_get(w.dtype, w.N, w.M, w.P, w.Q)
    ranges, costs = shard.partition_lags(w.N, w.M, w.P, w.Q, world)
    lo, hi = ranges[rank]
    ws = torch.empty(max(256, cov.workspace_size(w.dtype, w.N, w.M, w.P, w.Q, "recurrence")),
                     dtype=torch.uint8, device="cuda")
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    scratch = None

    def step():
        nonlocal scratch
        shard.estimate_shard_into(A, R, w.P, w.Q, lo, hi, workspace=ws)
        scratch = shard.allgather_blocks(R, w.P, w.Q, ranges, rank, scratch=scratch)

    for k in range(args.warmup):
        flush.fill_(k & 0xFF)
        step()
    torch.cuda.synchronize()
    cov.check_device_status(ws)
    K = args.steps
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * K)]
    dist.barrier()
    torch.cuda.synchronize()
    for k in range(K):
        flush.fill_((k + 1) & 0xFF)
        ev[2 * k].record(stream)
        step()
        ev[2 * k + 1].record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    cov.check_device_status(ws)
    total_s = sum(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(K)) / 1e3
    t = torch.tensor([total_s], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_s = float(t.item())
    # the assembled R against the unsharded estimate on the same input
    full = cov.estimate(A, w.P, w.Q, algo="recurrence")
    torch.cuda.synchronize()
    same = bool(torch.equal(torch.view_as_real(full), torch.view_as_real(R)))
    ok = torch.tensor([1 if same else 0], dtype=torch.int32, device="cuda")
    dist.all_reduce(ok, op=dist.ReduceOp.MIN)
    if rank == 0:
        line = {
            "metric": METRIC, "value": um * K / total_s, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": total_s * 1e3 / K, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f64" if w.dtype == "c128" else "f32",
            "data": "synthetic",
            "config": dict(_config(w), tuning=knobs, sharding="column lags per rank",
                           lag_ranges=ranges, rank_costs=costs,
                           collective="NCCL all_gather of the packed blocks (padded to the largest share)"),
            "assembled_R_equals_unsharded": bool(ok.item() == 1),
            "nccl_version": ".".join(str(x) for x in torch.cuda.nccl.version()),
            "process_group_size": dist.get_world_size(),
            # per step: the shard's kernels, one pack, one unpack per other rank
            "gpu_launches": K * ((4 if knobs["kernels"] == 4 else 1) + 1 + (world - 1)),
        }
        print(json.dumps(line))
    dist.barrier()
    dist.destroy_process_group()
    return 0


def bench_ours(args, rank, world, local):
    import numpy as np
    import torch

    import cov_workloads as wl
    import paper_1303_2285_gb300 as cov

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    w = wl.WORKLOADS[args.workload]
    dt = torch.complex64 if w.dtype == "c64" else torch.complex128
    A_np = wl.workload_input(w, index=rank)
    A = torch.from_numpy(A_np).cuda()
    D = w.P * w.Q
    R = torch.empty((D, D), dtype=dt, device="cuda")
    info = cov.plan_info(w.N, w.M, w.P, w.Q)
    um = info["distinct_products"]
    tune_ms, source = None, "defaults"
    if args.knobs:
        cov.tuning_set(w.dtype, w.N, w.M, w.P, w.Q, parse_knobs(args.knobs))
        source = "given"
    elif args.tuning_file and os.path.exists(args.tuning_file):
        cov.tuning_load(args.tuning_file)
        source = "file"
    elif args.autotune:
        # the library's tuner times its candidate knobs on this input and
        # caches the fastest; planning below picks them up (untimed)
        _, tune_ms = cov.autotune(A, w.P, w.Q, reps=5)
        tune_ms, source = round(tune_ms, 5), "autotune"
        if args.tuning_file:
            cov.tuning_save(args.tuning_file)
    knobs, cached = cov.tuning_get(w.dtype, w.N, w.M, w.P, w.Q)
    tuning = dict(knobs, source=source if cached else "defaults", tuned_ms_per_call=tune_ms)
    torch.cuda.synchronize()
    ws = torch.empty(max(256, cov.workspace_size(w.dtype, w.N, w.M, w.P, w.Q, "recurrence")),
                     dtype=torch.uint8, device="cuda")
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    rt = Cudart()
    sp = stream.cuda_stream

    def flush_l2(k):
        return rt.memset(flush.data_ptr(), k & 0xFF, FLUSH_BYTES, sp)

    def call(Ain=A, Rout=R):
        cov.estimate_into(Ain, Rout, w.P, w.Q, algo="recurrence", workspace=ws)

    def mk_events(n):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        for e in evs:
            e.record(stream)
        return evs

    for k in range(args.warmup):
        flush_l2(k)
        call()
    torch.cuda.synchronize()
    cov.check_device_status(ws)

    K = args.steps
    starts, ends = mk_events(K), mk_events(K)
    torch.cuda.synchronize()
    # the timed loop calls the C ABI directly with prepared arguments, so that
    # the host enqueues faster than the GPU runs (no host gaps inside a step)
    lib = cov.load()
    fn = lib.cov_estimate_ex
    cargs = (A.data_ptr(), cov.DTYPES[w.dtype], w.N, w.M, A.stride(0), w.P, w.Q, R.data_ptr(),
             cov.ALGOS["recurrence"], cov.NORMS["mean"], ws.data_ptr(), ws.numel(), stream.cuda_stream)
    sampler = ClockSampler()
    if rank == 0:
        sampler.start()
        time.sleep(0.3)
    barrier()
    codes = 0
    t_enq = time.perf_counter()
    for k in range(K):
        codes |= flush_l2(k + 1)
        starts[k].record(stream)
        codes |= fn(*cargs)
        ends[k].record(stream)
    enqueue_s = time.perf_counter() - t_enq
    barrier()
    if codes != 0:
        raise RuntimeError(f"cov_estimate_ex failed in the timed loop (status bits {codes})")
    clocks = sampler.stop(local) if rank == 0 else None
    cov.check_device_status(ws)
    step_ms = [starts[k].elapsed_time(ends[k]) for k in range(K)]
    fused = knobs["kernels"] == 1

    def stage_pass(n):
        # the library records events on the launching stream around its
        # kernel(s): the fused kernel alone, or each of the four kernels
        # (this serialises them, so the headline step is measured without it)
        flat = mk_events(5 * n)
        torch.cuda.synchronize()
        cov.set_stage_events(flat)
        c = 0
        for k in range(n):
            c |= flush_l2(k)
            c |= fn(*cargs)
        torch.cuda.synchronize()
        cov.set_stage_events(None)
        if c != 0:
            raise RuntimeError("stage-timing pass failed")
        return [[flat[5 * k + i].elapsed_time(flat[5 * k + i + 1]) for k in range(n)] for i in range(4)]

    Ks = min(K, 400)
    stage_ms = stage_pass(Ks)  # production kernels (fused: stage 0 is the kernel)
    # the four-kernel form, for the per-stage split
    cov.tuning_set(w.dtype, w.N, w.M, w.P, w.Q, dict(knobs, kernels=4))
    stage4_ms = stage_pass(min(Ks, 200))
    cov.tuning_set(w.dtype, w.N, w.M, w.P, w.Q, knobs if cached else None)
    total_s = sum(step_ms) / 1e3
    if dist is not None:
        t = torch.tensor([total_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    value = um * K * world / total_s
    ms_per_step = total_s * 1e3 / K

    # ---- end to end through the public API with host buffers -------------
    A_host = torch.from_numpy(A_np).pin_memory()
    R_host = torch.empty((D, D), dtype=dt).pin_memory()
    A_e2e = torch.empty_like(A)
    nbA = A_host.numel() * A_host.element_size()
    nbR = R_host.numel() * R_host.element_size()
    eargs = (A_e2e.data_ptr(),) + cargs[1:]
    Ke = max(3, min(K, 200))
    e_s, e_e = mk_events(Ke), mk_events(Ke)

    def e2e_step():
        c = rt.memcpy(A_e2e.data_ptr(), A_host.data_ptr(), nbA, Cudart.H2D, sp)
        c |= fn(*eargs)
        c |= rt.memcpy(R_host.data_ptr(), R.data_ptr(), nbR, Cudart.D2H, sp)
        return c

    for k in range(3):
        codes |= e2e_step()
    barrier()
    for k in range(Ke):
        codes |= flush_l2(k)
        e_s[k].record(stream)
        codes |= e2e_step()
        e_e[k].record(stream)
    barrier()
    if codes != 0:
        raise RuntimeError("end-to-end loop failed")
    e2e_s = sum(e_s[k].elapsed_time(e_e[k]) for k in range(Ke)) / 1e3
    if dist is not None:
        t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": um * Ke * world / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": nbA, "d2h_bytes_per_step": nbR,
           "ms_per_step": e2e_s * 1e3 / Ke}

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel -----------------------------------
    # fused: the one kernel runs every distinct product (inner and fringe
    # rows); four kernels: the product kernel over the inner rows
    peaks = measured_peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    f_max = float(peaks.get("sm_max_mhz", FALLBACK_SM_MAX_MHZ))
    fp32_peak = sms * FP32_LANES_PER_SM * 2 * f_max * 1e6  # FLOP/s
    fma_rate = measure_fma_rates(cov)
    fp64 = w.dtype == "c128"
    k1_ms = statistics.mean(stage_ms[0])
    k1_flops = 8.0 * (um if fused else info["products_inner"])  # 4 FMA per complex product
    achieved = k1_flops / (k1_ms * 1e-3)
    kname = "k_fused" if fused else "k_products_inner"
    traffic = NCU_TRAFFIC.get((w.name, kname, kernel_source_hash()))
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": fp32_peak / 1e12,
                "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": traffic,
                "kernel": kname, "peak_source": (
                    f"FP32 FMA: {sms} SMs x {FP32_LANES_PER_SM} lanes x 2 FLOP x {f_max:.0f} MHz "
                    f"({'MEASURED_PEAKS.json sm_max_mhz' if 'sm_max_mhz' in peaks else 'recipe max clock'})"
                    + ("; this workload computes in FP64: the FP32 figure is an upper bound" if fp64 else "")),
                "algorithmic_flops_per_launch": k1_flops, "launch_ms": k1_ms,
                "measured_fp32_fma_tflops": 2 * fma_rate["f32"] / 1e12,
                "frac_of_measured_fp32_fma": achieved / (2 * fma_rate["f32"])}
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS)) * 1e9
    bytes_io = w.N * w.M * A.element_size() + D * D * R.element_size()
    t_roof = max(4.0 * um / (fp32_peak / 2), bytes_io / hbm)
    step_roofline = {"t_roof_us": t_roof * 1e6, "t_step_us": ms_per_step * 1e3,
                     "frac": t_roof / (ms_per_step * 1e-3),
                     "definition": "max(4*UM / FP32 FMA peak, (A+R bytes) / HBM)"}

    # ---- plain FP64 GPU path on the same input, and error vs FP64 ----------
    Rd = torch.empty_like(R)
    cov.estimate_into(A, Rd, w.P, w.Q, algo="direct", workspace=ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev0, ev1 = mk_events(2)
    ev0.record(stream)
    cov.estimate_into(A, Rd, w.P, w.Q, algo="direct", workspace=ws)
    ev1.record(stream)
    torch.cuda.synchronize()
    direct_ms = ev0.elapsed_time(ev1)
    call()
    torch.cuda.synchronize()
    Rn, Rdn = R.cpu().numpy().astype(np.complex128), Rd.cpu().numpy().astype(np.complex128)
    err_fro = float(np.linalg.norm(Rn - Rdn) / np.linalg.norm(Rdn))
    err_max = float(np.abs(Rn - Rdn).max() / np.abs(Rdn).max())
    hermitian = bool(np.array_equal(Rn, Rn.conj().T))
    lam_min = float(np.linalg.eigvalsh(Rn).min())
    norm2 = float(np.linalg.norm(Rn, 2))

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if fp64 else "f32",
        "data": "synthetic", "config": dict(_config(w), tuning=tuning),
        "r_elements_per_s": D * D * K * world / total_s,
        "vs_plain_fp64_gpu": {"speedup": direct_ms / ms_per_step, "fp64_direct_ms": direct_ms},
        "err_vs_fp64": {"rel_fro": err_fro, "max_abs_rel_to_max": err_max,
                        "reference": "plain FP64 GPU path (COV_DIRECT) on the same input"},
        "checks": {"hermitian_exact": hermitian, "min_eig_over_norm": lam_min / norm2},
        "kernel_ms": {kname: k1_ms},
        "four_kernel_stages_ms": {n: statistics.mean(s) for n, s in
                                  zip(("products_inner", "fringe_rows", "reduce", "walk_write"),
                                      stage4_ms)},
        "roofline": roofline, "step_roofline": step_roofline, "e2e": e2e,
        "gpu_launches": (1 if fused else 4) * K, "clocks": clocks,
        "host_enqueue_us_per_step": enqueue_s * 1e6 / K,
    }

    if world == 1 and not args.no_cpu_baseline:
        def gpu_check(Asub):
            At = torch.from_numpy(np.ascontiguousarray(Asub)).cuda()
            return cov.estimate(At, w.P, w.Q, algo="recurrence").cpu().numpy().astype(np.complex128)
        line["cpu_baseline"] = cpu_baseline_leg(A_np, w.P, w.Q, um, w.K, args.cpu_seconds, gpu_check,
                                                  single_thread=True, R_gpu_full=Rn)
        line["err_vs_oracle"] = line["cpu_baseline"]["gpu_err_vs_oracle_full_R"]
    if args.extras:
        line["rows"] = extras(args, cov, torch, np, wl, mk_events, stream)
        line["rows"]["batched_4096_uneven_f32"] = bench_batched(cov, torch, np, wl, mk_events, stream,
                                                                fp32_peak)
        line["rows"]["apertures_100x100_of_25x25_w10_f32"] = bench_apertures(
            cov, torch, np, wl, mk_events, stream, fp32_peak, hbm)
        line["rows"]["capon_spectra_of_10000_apertures"] = bench_capon(cov, torch, np, wl, mk_events,
                                                                      stream, fp32_peak)
        line["rows"]["diff_b64_256x256_w12_f32"] = bench_adjoint(cov, torch, np, wl, mk_events, stream,
                                                                 fp32_peak)
        line["rows"]["gemm_tf32x3_" + GEMM_WORKLOAD] = bench_gemm(cov, torch, np, wl, mk_events, stream)
        line["rows"]["gemm_bf16x3_" + GEMM_WORKLOAD] = bench_gemm(cov, torch, np, wl, mk_events, stream,
                                                                  "gemm_bf16x3")
    print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def measure_fma_rates(cov) -> dict:
    """Lane FMAs per second of the FP32 (paired) and FP64 pipes, measured by
    the library's FMA-chain kernel on this GPU (cov_measure_fma_rate)."""
    import torch
    lib = cov.load()
    out = {}
    for name, code in (("f32", 0), ("f64", 1)):
        v = ctypes.c_double(0)
        if lib.cov_measure_fma_rate(code, 5, ctypes.byref(v), torch.cuda.current_stream().cuda_stream):
            raise RuntimeError("cov_measure_fma_rate failed")
        out[name] = v.value
    return out


def bench_batched(cov, torch, np, wl, mk_events, stream, fp32_peak) -> dict:
    """4096 uneven matrices in one persistent, graph-captured launch."""
    shapes = wl.batched_shapes()
    items = []
    for k, (N, M, P, Q) in enumerate(shapes):
        A = torch.from_numpy(wl.complex_normal((N, M), wl.BATCHED_SEED * 100003 + k, "c64")).cuda()
        R = torch.empty((P * Q, P * Q), dtype=torch.complex64, device="cuda")
        items.append((A, R, P, Q))
    um = sum(cov.plan_info(N, M, P, Q)["distinct_products"] for N, M, P, Q in shapes)
    plan = cov.BatchedPlan(items)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.upload(ws)
    tuning = plan.autotune(ws, reps=2)  # untimed: picks form, segment length, task shape
    s = torch.cuda.Stream()
    for _ in range(3):
        plan.run(ws, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.run(ws, stream=s)
    torch.cuda.synchronize()
    n = 10
    ev = mk_events(2 * n)
    for k in range(n):  # inputs (~0.7 GB) exceed L2: no flush needed
        ev[2 * k].record(stream)
        g.replay()
        ev[2 * k + 1].record(stream)
    torch.cuda.synchronize()
    ms = sum(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(n)) / n
    cov.check_device_status(ws)
    # error vs the plain FP64 GPU path on a sample of members
    errs = []
    for k in range(0, len(items), len(items) // 8):
        A, R, P, Q = items[k]
        Rd = cov.estimate(A, P, Q, algo="direct")
        errs.append(float(np.linalg.norm(R.cpu().numpy().astype(np.complex128) - Rd.cpu().numpy())
                          / np.linalg.norm(Rd.cpu().numpy())))
    return {"matrices": len(shapes), "ms_per_launch": ms, "distinct_products": um,
            "distinct_products_per_s": um / (ms * 1e-3), "matrices_per_s": len(shapes) / (ms * 1e-3),
            "fp32_fma_frac": 8.0 * um / (ms * 1e-3) / fp32_peak,
            "input_bytes": sum(N * M * 8 for N, M, _, _ in shapes),
            "err_vs_fp64_direct_rel_fro_max_of_8": max(errs), "graph_captured": True,
            "tuning": tuning}


def bench_apertures(cov, torch, np, wl, mk_events, stream, fp32_peak, hbm) -> dict:
    """Every 25 x 25 aperture at stride 10 of a 1015 x 1015 image (100 x 100
    apertures), 10 x 10 window, read in place: the strip launch
    (cov_estimate_apertures, graph-captured) and, beside it, the batched
    plan over the same apertures."""
    H = W = 1015
    img = torch.from_numpy(wl.complex_normal((H, W), 77, "c64")).cuda()
    s = torch.cuda.Stream()

    def time_graph(fn, n=10):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            fn()
        torch.cuda.synchronize()
        ev = mk_events(2 * n)
        for k in range(n):
            ev[2 * k].record(stream)
            g.replay()
            ev[2 * k + 1].record(stream)
        torch.cuda.synchronize()
        return sum(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(n)) / n

    plan, R = cov.aperture_batch(img, (25, 25), (10, 10), 10, 10)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.upload(ws)
    tuning = plan.autotune(ws, reps=2)  # untimed
    ms_batched = time_graph(lambda: plan.run(ws, stream=s))
    cov.check_device_status(ws)
    ms = time_graph(lambda: cov.apertures(img, (25, 25), (10, 10), 10, 10, out=R, stream=s))
    um = R.shape[0] * cov.plan_info(25, 25, 10, 10)["distinct_products"]
    return {"apertures": R.shape[0], "kernel": "k_apertures (strip launch)", "ms_per_launch": ms,
            "apertures_per_s": R.shape[0] / (ms * 1e-3),
            "distinct_products_per_s": um / (ms * 1e-3), "fp32_fma_frac": 8.0 * um / (ms * 1e-3) / fp32_peak,
            "r_bytes": R.numel() * 8, "r_write_hbm_frac": R.numel() * 8 / (ms * 1e-3) / hbm,
            "graph_captured": True, "batched_plan_ms_per_launch": ms_batched,
            "batched_plan_tuning": tuning}


def bench_capon(cov, torch, np, wl, mk_events, stream, fp32_peak) -> dict:
    """Minimum-variance (Capon) spectra of the 10,000 aperture estimates (the
    downstream use of R named in Section 2.3): an 8 x 8 grid of 2-D steering
    vectors, diagonal loading 0.01 trace(R) / D."""
    H = W = 1015
    img = torch.from_numpy(wl.complex_normal((H, W), 77, "c64")).cuda()
    plan, R = cov.aperture_batch(img, (25, 25), (10, 10), 10, 10)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.upload(ws)
    plan.run(ws)
    g = np.linspace(-np.pi, np.pi, 9)[:-1]
    om, nu = np.repeat(g, 8), np.tile(g, 8)
    i = np.arange(10)
    steer_np = np.array([np.exp(1j * (w * i[:, None] + v * i[None, :])).T.reshape(-1)
                         for w, v in zip(om, nu)]).astype(np.complex64)
    steer = torch.from_numpy(steer_np).cuda()
    out = torch.empty((R.shape[0], steer.shape[0]), dtype=torch.float32, device="cuda")
    for _ in range(2):
        cov.capon_spectrum(R, steer, 0.01, out=out)
    torch.cuda.synchronize()
    n = 5
    ev = mk_events(2 * n)
    for k in range(n):
        ev[2 * k].record(stream)
        cov.capon_spectrum(R, steer, 0.01, out=out)
        ev[2 * k + 1].record(stream)
    torch.cuda.synchronize()
    ms = sorted(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(n))[n // 2]
    D, F, cnt = 100, steer.shape[0], R.shape[0]
    flops = 8.0 * cnt * (D ** 3 / 6 + F * D * D / 2)  # complex MACs of the factorisation and solves
    return {"matrices": cnt, "D": D, "steering_vectors": F, "ms_per_launch": ms,
            "spectra_values_per_s": cnt * F / (ms * 1e-3),
            "fp32_fma_frac": flops / (ms * 1e-3) / fp32_peak,
            "all_finite": bool(torch.isfinite(out).all())}


def bench_adjoint(cov, torch, np, wl, mk_events, stream, fp32_peak) -> dict:
    """Differentiation workload: batch of 64 A (256 x 256, window 12 x 12);
    forward through the batched launch, adjoint dL/dA of every member for
    L = ||R - R_target||_F^2 (G = 2 (R - R_target) formed once, untimed):
    the stencil form over the whole batch in one launch sequence, and the
    dense form member by member (64 calls in one CUDA graph) for comparison."""
    w = wl.WORKLOADS["diff_b64_256x256_w12_f32"]
    P, Q, N, M, B = w.P, w.Q, w.N, w.M, w.batch
    A_all = torch.stack([torch.from_numpy(wl.complex_normal((N, M), w.seed + k, "c64"))
                         for k in range(B)]).cuda()
    R_all = torch.empty((B, P * Q, P * Q), dtype=torch.complex64, device="cuda")
    T = cov.estimate(torch.from_numpy(wl.complex_normal((N, M), 5000, "c64")).cuda(), P, Q)
    plan = cov.BatchedPlan([(A_all[k], R_all[k], P, Q) for k in range(B)])
    wsf = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.upload(wsf)
    plan.run(wsf)
    torch.cuda.synchronize()
    G_all = (2.0 * (R_all - T)).contiguous()
    dA_all = torch.empty_like(A_all)
    lib = cov.load()
    need = ctypes.c_size_t(0)
    lib.cov_backward_strided_workspace_size(B, N, M, P, Q, ctypes.byref(need))
    wss = torch.empty(need.value, dtype=torch.uint8, device="cuda")
    wsd = torch.empty(cov.backward_workspace_size(N, M, P, Q, "dense"), dtype=torch.uint8,
                      device="cuda")
    D = P * Q
    sargs = (A_all.data_ptr(), N * M, G_all.data_ptr(), D * D, dA_all.data_ptr(), N * M, B, N, M,
             P, Q, 0, wss.data_ptr(), wss.numel(), stream.cuda_stream)
    if lib.cov_estimate_backward_strided(*sargs) != 0:
        raise RuntimeError("strided adjoint failed")
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    codes = 0
    with torch.cuda.graph(g, stream=side):
        for k in range(B):
            codes |= lib.cov_estimate_backward_ex(
                A_all[k].data_ptr(), G_all[k].data_ptr(), 0, N, M, P, Q, 0, 1, dA_all[k].data_ptr(),
                wsd.data_ptr(), wsd.numel(), side.cuda_stream)
    if codes != 0:
        raise RuntimeError("dense adjoint failed under capture")
    g.replay()
    torch.cuda.synchronize()
    n = 3
    ev = mk_events(4 * n)
    for k in range(n):
        ev[4 * k].record(stream)
        plan.run(wsf)
        ev[4 * k + 1].record(stream)
        lib.cov_estimate_backward_strided(*sargs)
        ev[4 * k + 2].record(stream)
        g.replay()
        ev[4 * k + 3].record(stream)
    torch.cuda.synchronize()
    cov.check_device_status(wss)
    fwd = sum(ev[4 * k].elapsed_time(ev[4 * k + 1]) for k in range(n)) / n
    bwd = sum(ev[4 * k + 1].elapsed_time(ev[4 * k + 2]) for k in range(n)) / n
    bwd_dense = sum(ev[4 * k + 2].elapsed_time(ev[4 * k + 3]) for k in range(n)) / n
    KW = (N - P + 1) * (M - Q + 1)
    ND = (2 * P - 1) * (2 * Q - 1)
    st_flops = 8.0 * ND * N * M * B     # complex MACs of the stencil (upper bound: full support)
    hx_flops = 8.0 * D * D * KW * B     # complex MACs of Y = H X
    return {"batch": B, "forward_ms": fwd, "backward_ms": bwd,
            "backward_form": "stencil, one strided-batch launch sequence",
            "forward_plus_backward_ms": fwd + bwd,
            "backward_fp32_fma_frac": st_flops / (bwd * 1e-3) / fp32_peak,
            "backward_dense_ms": bwd_dense,
            "backward_dense_fp32_fma_frac": hx_flops / (bwd_dense * 1e-3) / fp32_peak,
            "workspace_bytes_backward": wss.numel()}


TF32_OVER_BF16_NOMINAL = 1.1 / 2.25  # dense tensor rates per GPU (recipe's nominal table)


def bench_gemm(cov, torch, np, wl, mk_events, stream, algo: str = "gemm_tf32x3") -> dict:
    """Dense form R = X X^H on tcgen05 on the bench workload: TF32 x3 (three
    split products, K = 8 MMAs) or BF16 x3 (six split products, K = 16)."""
    w = wl.WORKLOADS[GEMM_WORKLOAD]
    A = torch.from_numpy(wl.workload_input(w)).cuda()
    D = w.P * w.Q
    R = torch.empty((D, D), dtype=torch.complex64, device="cuda")
    ws = torch.empty(cov.workspace_size("c64", w.N, w.M, w.P, w.Q, algo), dtype=torch.uint8,
                     device="cuda")
    for _ in range(2):
        cov.estimate_into(A, R, w.P, w.Q, algo=algo, workspace=ws)
    torch.cuda.synchronize()
    n = 5
    ev = mk_events(2 * n)
    for k in range(n):
        ev[2 * k].record(stream)
        cov.estimate_into(A, R, w.P, w.Q, algo=algo, workspace=ws)
        ev[2 * k + 1].record(stream)
    torch.cuda.synchronize()
    cov.check_device_status(ws)
    ms = sum(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(n)) / n
    Rd = cov.estimate(A, w.P, w.Q, algo="direct")
    Rn, Rdn = R.cpu().numpy().astype(np.complex128), Rd.cpu().numpy().astype(np.complex128)
    nt = (2 * D + 127) // 128
    tiles = nt * (nt + 1) // 2
    bf16 = algo == "gemm_bf16x3"
    products = 6 if bf16 else 3
    flops = products * 2.0 * tiles * 128 * 128 * w.K  # the split products over the upper tiles
    peaks = measured_peaks()
    if bf16:
        peak, src = float(peaks.get("bf16_tflops", 1900.0)), "MEASURED_PEAKS bf16_tflops"
    else:
        peak = float(peaks.get("bf16_tflops", 1900.0)) * TF32_OVER_BF16_NOMINAL
        src = "MEASURED_PEAKS bf16_tflops x 1.1/2.25 (nominal TF32/BF16)"
    info = cov.plan_info(w.N, w.M, w.P, w.Q)
    return {"workload": w.name, "ms_per_call": ms, "tensor_tflops": flops / (ms * 1e-3) / 1e12,
            "peak_tflops": peak, "peak_source": src,
            "frac_of_peak": flops / (ms * 1e-3) / 1e12 / peak,
            "distinct_products_per_s": info["distinct_products"] / (ms * 1e-3),
            "err_vs_fp64_direct_rel_fro": float(np.linalg.norm(Rn - Rdn) / np.linalg.norm(Rdn))}


def extras(args, cov, torch, np, wl, mk_events, stream) -> dict:
    """Timings of the other workloads through the same path (not bench lines).
    Knobs are autotuned first; the calls are timed as replays of a CUDA graph
    of n calls (device time only, no host gaps; inputs stay L2-resident)."""
    out = {}
    lib = cov.load()
    fma_rates = measure_fma_rates(cov)
    out["measured_fma_rates"] = {"fp32_tflops": 2 * fma_rates["f32"] / 1e12,
                                 "fp64_tflops": 2 * fma_rates["f64"] / 1e12,
                                 "how": "cov_measure_fma_rate: independent FMA chains on every SM, "
                                        "best of 5 launches, CUDA events"}
    for name in ("plain_64x64_w8_f64", "cn_1024x1024_w16_f32", "sar_2048x512_w32_f32"):
        if name == args.workload:
            continue
        w = wl.WORKLOADS[name]
        dt = torch.complex64 if w.dtype == "c64" else torch.complex128
        A = torch.from_numpy(wl.workload_input(w)).cuda()
        D = w.P * w.Q
        R = torch.empty((D, D), dtype=dt, device="cuda")
        knobs, _ = cov.autotune(A, w.P, w.Q, reps=3)
        ws = torch.empty(cov.workspace_size(w.dtype, w.N, w.M, w.P, w.Q, "recurrence"),
                         dtype=torch.uint8, device="cuda")
        cargs = (A.data_ptr(), cov.DTYPES[w.dtype], w.N, w.M, A.stride(0), w.P, w.Q, R.data_ptr(),
                 cov.ALGOS["recurrence"], cov.NORMS["mean"], ws.data_ptr(), ws.numel())
        side = torch.cuda.Stream()
        for _ in range(3):
            lib.cov_estimate_ex(*cargs, side.cuda_stream)
        torch.cuda.synchronize()
        n = 20
        g = torch.cuda.CUDAGraph()
        codes = 0
        with torch.cuda.graph(g, stream=side):
            for _ in range(n):
                codes |= lib.cov_estimate_ex(*cargs, side.cuda_stream)
        if codes != 0:
            raise RuntimeError(f"{name}: cov_estimate_ex failed under stream capture")
        g.replay()
        torch.cuda.synchronize()
        reps = 10
        ev = mk_events(2 * reps)
        for k in range(reps):
            ev[2 * k].record(stream)
            g.replay()
            ev[2 * k + 1].record(stream)
        torch.cuda.synchronize()
        ms = sorted(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(reps))[reps // 2] / n
        cov.check_device_status(ws)
        info = cov.plan_info(w.N, w.M, w.P, w.Q)
        Rd = torch.empty_like(R)
        e2 = mk_events(2)
        e2[0].record(stream)
        cov.estimate_into(A, Rd, w.P, w.Q, algo="direct", workspace=ws)
        e2[1].record(stream)
        torch.cuda.synchronize()
        dms = e2[0].elapsed_time(e2[1])
        Rn, Rdn = R.cpu().numpy().astype(np.complex128), Rd.cpu().numpy().astype(np.complex128)
        row_fp64 = w.dtype == "c128"
        rate = fma_rates["f64" if row_fp64 else "f32"]
        out[name] = {"ms_per_call": ms, "timing": f"median of {reps} replays of a {n}-call CUDA graph, L2 warm",
                     "tuning": knobs,
                     "fma_pipe": "FP64" if row_fp64 else "FP32",
                     "measured_fma_tflops": 2 * rate / 1e12,
                     "frac_of_measured_fma_peak": 4.0 * info["distinct_products"] / (ms * 1e-3) / rate,
                     "distinct_products_per_s": info["distinct_products"] / (ms * 1e-3),
                     "r_elements_per_s": D * D / (ms * 1e-3), "fp64_direct_ms": dms,
                     "speedup_vs_fp64_direct": dms / ms,
                     "err_vs_fp64_direct_rel_fro": float(np.linalg.norm(Rn - Rdn) / np.linalg.norm(Rdn))}
    return out


def profile_case(case: str, knobs=None) -> int:  # noqa: C901 - one branch per case
    """A few launches of one kernel family on a small case, for ncu captures:
    the single-matrix combination path on the SAR-like 2048 x 512 input (32 x
    32 window) or on the 1024 x 1024 one (16 x 16), 600 uneven matrices
    through the batched launch (seed 3), the dense TF32x3 form on the
    1024 x 1024 workload, the stencil adjoint of a batch of eight (or, with
    the knob, that many) 256 x 256 inputs with a 12 x 12 window, the 30 x 30 apertures of 25 x 25 (stride
    10, 10 x 10 window) of a 315 x 315 image through the batched launch's
    default form (knob "strip": the strip launch), and the Capon spectra of
    those 900 estimates."""
    import numpy as np
    import torch

    import cov_workloads as wl
    import paper_1303_2285_gb300 as cov
    if case in ("sar", "cn"):
        # the bench's single-matrix step: the combination path on the SAR-like
        # 2048 x 512 input (32 x 32 window) or the 1024 x 1024 one (16 x 16)
        w = wl.WORKLOADS["sar_2048x512_w32_f32" if case == "sar" else "cn_1024x1024_w16_f32"]
        if knobs:
            cov.tuning_set(w.dtype, w.N, w.M, w.P, w.Q, parse_knobs(knobs))
        A = torch.from_numpy(wl.workload_input(w)).cuda()
        R = torch.empty((w.P * w.Q, w.P * w.Q), dtype=torch.complex64, device="cuda")
        ws = torch.empty(cov.workspace_size(w.dtype, w.N, w.M, w.P, w.Q, "recurrence"),
                         dtype=torch.uint8, device="cuda")
        for _ in range(3):
            cov.estimate_into(A, R, w.P, w.Q, algo="recurrence", workspace=ws)
        torch.cuda.synchronize()
        cov.check_device_status(ws)
    elif case == "batched":
        items = []
        for k, (N, M, P, Q) in enumerate(wl.batched_shapes(600, wl.BATCHED_SEED)):
            A = torch.from_numpy(wl.complex_normal((N, M), wl.BATCHED_SEED * 100003 + k, "c64")).cuda()
            items.append((A, torch.empty((P * Q, P * Q), dtype=torch.complex64, device="cuda"), P, Q))
        plan = cov.BatchedPlan(items)
        if knobs:  # the batched plan's form (0 or 3); default: the plan's own
            plan.set_tuning(int(knobs), 0, 4)
        ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
        plan.upload(ws)
        for _ in range(3):
            plan.run(ws)
    elif case == "apertures":
        img = torch.from_numpy(wl.complex_normal((315, 315), 77, "c64")).cuda()
        if knobs == "strip":  # the strip launch
            for _ in range(3):
                cov.apertures(img, (25, 25), (10, 10), 10, 10)
        else:
            plan, R = cov.aperture_batch(img, (25, 25), (10, 10), 10, 10)
            if knobs:  # the batched plan's form (0, 1 or 2); default: the plan's own
                plan.set_tuning(int(knobs), 0, 4)
            ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
            plan.upload(ws)
            for _ in range(3):
                plan.run(ws)
    elif case == "capon":
        img = torch.from_numpy(wl.complex_normal((315, 315), 77, "c64")).cuda()
        plan, R = cov.aperture_batch(img, (25, 25), (10, 10), 10, 10)
        ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
        plan.upload(ws)
        plan.run(ws)
        g = np.linspace(-np.pi, np.pi, 9)[:-1]
        i = np.arange(10)
        steer = torch.from_numpy(np.array(
            [np.exp(1j * (w_ * i[:, None] + v_ * i[None, :])).T.reshape(-1)
             for w_, v_ in zip(np.repeat(g, 8), np.tile(g, 8))]).astype(np.complex64)).cuda()
        for _ in range(3):
            cov.capon_spectrum(R, steer, 0.01)
    elif case == "gemm":
        w = wl.WORKLOADS[GEMM_WORKLOAD]
        A = torch.from_numpy(wl.workload_input(w)).cuda()
        for _ in range(2):
            cov.estimate(A, w.P, w.Q, algo="gemm_tf32x3")
    else:
        N = M = 256
        P = Q = 12
        B = int(knobs) if knobs else 8  # members (the bench row's batch: 64)
        A = torch.stack([torch.from_numpy(wl.complex_normal((N, M), 4 + k, "c64"))
                         for k in range(B)]).cuda()
        G = torch.stack([torch.from_numpy(wl.complex_normal((P * Q, P * Q), 5 + k, "c64"))
                         for k in range(B)]).cuda()
        for _ in range(3):
            cov.estimate_backward_batch(A, G, P, Q)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": case, "ok": True}))
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--sharded", action="store_true",
                    help="split one matrix across the ranks by column lag and gather R with NCCL "
                         "(strong scaling) instead of one matrix per rank")
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--extras", action="store_true", default=True)
    ap.add_argument("--no-extras", dest="extras", action="store_false")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false", default=True)
    ap.add_argument("--tuning-file", default=None,
                    help="load the knobs from this file if it exists, else autotune and save them")
    ap.add_argument("--knobs", default=None,
                    help="G,TRB,L,K[,TC]: use these knobs (lag group, rows per task, re-seed interval, "
                         "kernels 1|4, tile columns 32|64) instead of autotuning")
    ap.add_argument("--profile-case",
                    choices=("sar", "cn", "batched", "gemm", "adjoint", "apertures", "capon"),
                    default=None,
                    help="run a few launches of one secondary kernel on a small case (for ncu) "
                         "and exit")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.profile_case:
        return profile_case(args.profile_case, args.knobs)
    rank, world, local = dist_setup()
    if args.impl == "reference":
        return bench_reference(args, rank, world)
    if args.sharded:
        return bench_sharded(args, rank, world, local)
    return bench_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
