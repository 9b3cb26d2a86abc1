"""The reference arm of bench.py prints the benchmark's one JSON line on the
CPU: the oracle on all host cores on its bounded sample, under the same
metric, unit and workload as the GPU arm."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    r = json.loads(lines[-1])
    sys.path.insert(0, ROOT)
    import bench
    assert r["impl"] == "reference"
    assert r["metric"] == bench.METRIC and r["unit"] == bench.UNIT
    assert r["value"] > 0 and r["ms_per_step"] > 0
    assert r["n_gpus"] == 1 and r["steps"] == 1 and r["warmup"] == 0
    assert r["higher_is_better"] is True and r["scaling"] == "weak" and r["vs_baseline"] is None
    assert r["data"] == "synthetic"
    assert r["config"]["workload"] == bench.WORKLOAD
    assert (r["config"]["P"], r["config"]["T"], r["config"]["period"]) == (bench.LARGE["P"], bench.LARGE["T"],
                                                                         bench.LARGE["period"])
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == r["value"]
    assert cb["cores"] == min(os.cpu_count(), r["config"]["sample_starts"]) and cb["host_cores"] == os.cpu_count()
    e2e = r["e2e"]
    assert e2e["value"] == r["value"] and e2e["unit"] == r["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
