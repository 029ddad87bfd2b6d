"""`bench.py --impl reference` (the FP64 oracle on the host cores, no GPU):
one JSON line with the contract's keys, the same metric, unit and workload
config as the GPU arm, and positive throughput."""
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    t0 = time.perf_counter()
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=900)
    wall = time.perf_counter() - t0
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    from paper_2101_07249_gb300 import inputs
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "inner_loops/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 0 and d["n_gpus"] == 1
    # the steps it reports are the ones it timed: they fit in the run's wall time
    assert d["steps"] * d["ms_per_step"] / 1e3 <= wall
    assert d["config"] == bench.workload_config(inputs.LARGE, "revd")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
