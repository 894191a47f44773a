"""The bench's CPU-only parts: the reference arm (the oracle timed on the host
cores) and the CPU-baseline leg. No GPU is needed for either."""
import json
import os
import subprocess
import sys

import numpy as np

import cov_workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT,
                          capture_output=True, text=True, timeout=600, env=env)


def test_reference_arm_prints_one_json_line():
    p = run_bench(["--impl", "reference", "--steps", "1", "--warmup", "3"])
    assert p.returncode == 0, p.stderr
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "distinct products/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "sar_2048x512_w32_f32"
    # every timed step ran: the steps' time fits inside the run's own wall clock
    assert d["ms_per_step"] * d["steps"] <= d["wall_s_incl_warmup"] * 1e3
    assert d["full_job_ms_extrapolated"] >= d["ms_per_step"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["ms_per_step"] > 0


def test_reference_arm_other_ranks_exit_without_output():
    p = run_bench(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"],
                  {"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def test_cpu_baseline_leg_reports_all_cores_and_one_core():
    import bench
    from oracle import combinations as cb
    N, M, P, Q = 40, 36, 4, 3
    A = wl.complex_normal((N, M), 3)
    K = (N - P + 1) * (M - Q + 1)
    um = cb.um_enumerated(N, M, P, Q)
    out = bench.cpu_baseline_leg(A, P, Q, um, K, 0.2, gpu_check=lambda a: np.zeros((P * Q, P * Q)),
                                 single_thread=True)
    assert out["kind"] == "oracle" and out["value"] > 0 and out["cores"] == (os.cpu_count() or 1)
    assert P <= out["rows"] <= N
    assert out["gpu_rel_fro_err_on_sample"] == 1.0  # the stand-in check returned zeros
    if out["cores"] > 1:
        st = out["single_thread"]
        assert st["cores"] == 1 and st["value"] > 0 and st["unit"] == out["unit"]


def test_cpu_baseline_leg_full_r_error_against_the_oracle():
    import bench
    import oracle
    from oracle import combinations as cb
    N, M, P, Q = 30, 28, 5, 4
    A = wl.complex_normal((N, M), 11)
    K = (N - P + 1) * (M - Q + 1)
    R = oracle.cov_window(A, P, Q)
    out = bench.cpu_baseline_leg(A, P, Q, cb.um_enumerated(N, M, P, Q), K, 0.1,
                                 R_gpu_full=R.astype(np.complex64))
    e = out["gpu_err_vs_oracle_full_R"]
    assert e["elements"] == (P * Q) ** 2
    assert 0 < e["rel_fro"] < 1e-7  # only the complex64 rounding of R
    out = bench.cpu_baseline_leg(A, P, Q, cb.um_enumerated(N, M, P, Q), K, 0.1, R_gpu_full=2 * R)
    assert abs(out["gpu_err_vs_oracle_full_R"]["rel_fro"] - 1.0) < 1e-12
