"""The benchmark's reference arm (the CPU oracle timed on the host cores) runs
without a GPU and prints the contract's JSON line."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1", "--ref-seconds", "2"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["value"] > 0 and line["unit"] == "point-trials/s"
    assert line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_pdot_override_applies_to_pdot_workloads_only(monkeypatch):
    """--pdots resizes the Pdot axis of the workloads that have one (Sec. 3 runs 32,
    128 and 512 values) and is refused for the others."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "5", "--pdots", "128"])
    assert bench.workload_overrides(bench.parse()) == {"n_pdots": 128}
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "1"])
    assert bench.workload_overrides(bench.parse()) == {}
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "1", "--pdots", "8"])
    with pytest.raises(SystemExit):
        bench.workload_overrides(bench.parse())


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 runs the reference arm; the other ranks exit 0
    without work or output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "1", "--ref-seconds", "2"],
                       capture_output=True, text=True, timeout=120, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
