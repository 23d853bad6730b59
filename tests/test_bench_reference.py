"""The reference arm of bench.py (the oracle timed on the host) for every sweep
form it supports: one JSON line with the contract's keys, on CPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("workload,mode", [("ising32", "plain"), ("ising32", "sw"), ("ising32", "higdon"),
                                           ("ferro3d", "sw")])
def test_reference_arm_prints_one_contract_line(workload, mode):
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", workload, "--mode", mode,
                        "--steps", "1", "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "site-updates/s" and d["value"] > 0
    assert d["config"]["workload"] == workload and d["config"]["mode"] == mode
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
