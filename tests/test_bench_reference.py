"""The benchmark's reference arm (the oracle on the host cores) keeps the JSON-line contract, and
under torchrun only rank 0 runs it.  CPU only: one bounded step of the fast workloads."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(args, env_extra=None):
    env = dict(os.environ, **(env_extra or {}))
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                         env=env, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    return [line for line in out.stdout.splitlines() if line.startswith("{")]


@pytest.mark.parametrize("workload", ["nstar", "any", "wrap"])
def test_reference_line(workload):
    lines = run_bench(["--impl", "reference", "--workload", workload, "--steps", "1", "--warmup", "0"])
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "samples/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "L=16" in d["metric"] and d["config"]["L"] == 16 and d["config"]["masks"] == 127


def test_reference_arm_other_ranks_exit_quietly():
    lines = run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"],
                      {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert lines == []
