"""bench.py on the CPU: the reference arm (the oracle, on a bounded sample of the benchmark's
workload) prints one well-formed line on the benchmark's own config, and the committed DRAM
traffic of the dominant kernel belongs to the current kernel source."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference"
    assert d["metric"] == "two-species D2Q9 GLUPS (FP32-deviation batched ensemble)" and d["unit"] == "GLUPS"
    assert d["higher_is_better"] is True and d["value"] > 0
    assert d["config"]["workload"] == bench.C3_WORKLOAD
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_committed_traffic_belongs_to_the_kernel_source():
    """profiles/persistent_kernel_bulk_traffic_c3.json carries the hash of the step kernels'
    sources it was measured on; a kernel change must come with a new capture."""
    with open(os.path.join(ROOT, "profiles", "persistent_kernel_bulk_traffic_c3.json")) as f:
        d = json.load(f)
    assert d["kernel_code_sha256"] == bench.kernel_code_hash()
    e = d["dev32_c3"]
    assert bench.kernel_traffic("dev32_c3") == float(e["bytes_per_step_full_size"])
    # per-site figures consistent with the raw counters
    lu = e["sites"] * e["steps_in_launch"]
    assert abs((e["dram_read_bytes"] + e["dram_write_bytes"]) / lu - e["dram_bytes_per_site"]) < 0.05
    assert e["dram_bytes_per_site"] >= e["algorithmic_bytes_per_site"] * 0.98
