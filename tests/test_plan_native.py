"""Host-only invariants of the combination path's plan layer (plan.cpp):
compiled with the host C++ compiler together with a small checker
(tests/native/plan_invariants.cpp) and run over a sweep of shapes, element
sizes and tuned knobs. No GPU and no CUDA call."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1303_2285_gb300", "csrc")


def test_plan_invariants(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "plan_invariants")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC,
                    os.path.join(ROOT, "tests", "native", "plan_invariants.cpp"),
                    os.path.join(CSRC, "plan.cpp"), "-o", exe], check=True, timeout=300)
    p = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stdout[-4000:]
    assert p.stdout.strip().endswith("0 violations")
