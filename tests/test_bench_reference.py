"""bench.py's reference arm (the CPU oracle on a bounded sample of the
workload) runs without a GPU and prints one JSON line with the fields the
benchmark contract asks of it."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run(
        [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
         "blobs_small", "--steps", "2", "--warmup", "3"],
        capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference"
    assert j["metric"] == "points/sec for full FAMST build" and j["unit"] == "points/s"
    assert j["value"] > 0 and j["steps"] == 2 and j["warmup"] == 3
    assert j["higher_is_better"] is True and j["n_gpus"] == 1
    assert j["config"]["workload"] == "blobs_small"
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == j["value"]
    e2e = j["e2e"]
    assert e2e["value"] == j["value"] and e2e["unit"] == j["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
