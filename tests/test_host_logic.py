"""The library's host-side planning logic (trial tiles, the top-k merge's first
level, SPLIT32 counter slots) compiled from its own headers with nvcc and run on
the CPU: tests/host_logic.cu makes no CUDA runtime call."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host_logic.cu")
OUT_DIR = os.path.join(ROOT, "tests", "_build")


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_host_planning_logic():
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    os.makedirs(OUT_DIR, exist_ok=True)
    exe = os.path.join(OUT_DIR, "host_logic")
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                        SRC, "-o", exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
