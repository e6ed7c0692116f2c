"""bench.py's output contract, on the host.

* The reference arm (the oracle on the host cores) prints exactly one JSON line with the
  keys of the bench line, its cpu_baseline describing the run and an e2e object with no
  host-device bytes.
* Every stored DRAM-traffic record names a kernel whose sources bench.py hashes, was
  captured from the current sources (its hash matches, so the bench lines report it),
  and carries the ncu command that produced it.
"""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "small",
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_traffic_records_name_hashed_kernels():
    out = subprocess.run([sys.executable, "bench.py", "--source-hash"], cwd=ROOT,
                         capture_output=True, text=True, check=True, timeout=300).stdout
    hashes = dict(line.split() for line in out.strip().splitlines())
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        records = json.load(f)
    names = [k for k in records if "@" in k]
    assert names
    for key in names:
        kernel, workload = key.split("@")
        rec = records[key]
        assert kernel in hashes, key
        assert rec["source_hash"] == hashes[kernel], f"{key}: sources changed since the capture"
        assert rec["command"].startswith("ncu ") and "--clock-control none" in rec["command"]
        assert f"--workload {workload}" in rec["command"]
        assert rec["read_bytes"] > 0 and rec["write_bytes"] > 0
