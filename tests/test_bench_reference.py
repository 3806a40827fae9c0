"""The benchmark's reference arm (`bench.py --impl reference`) runs the oracle on the host
cores, needs no GPU, and prints one JSON line with the contract's keys: the same metric,
unit and direction as the GPU arm, `impl`, a `cpu_baseline` describing the run, and an
`e2e` object with zero host-device traffic.  Run here on a 24^3 grid (the arm takes the
benchmark's --side) so that the CPU suite stays short; every host core runs one
single-threaded oracle process.""" 

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                          "--side", "24"],
                         cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "solves/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["steps"] == 1 and d["n_gpus"] == 1 and d["data"] == "synthetic"
    assert "3d-24^3-7pt" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == (os.cpu_count() or 1) and cb["sample"]
    assert cb["value"] == d["value"] and "single-threaded" in cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
