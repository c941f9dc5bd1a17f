"""The bench's reference arm (the FP64 oracle timed on the host cores) keeps
the JSON-line contract: one line with the metric, value, unit, step
counts, the oracle baseline it describes and an end-to-end entry with no
host-device traffic.  Runs on the CPU (no GPU needed)."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["steps"] == 1 and d["warmup"] >= 3 and d["value"] > 0 and d["higher_is_better"] is True
    assert d["unit"] == "grid-pts/s" and d["dtype"] == "f64" and d["data"] == "synthetic"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    # the same config dict as the GPU arm prints (same workload, same keys)
    sys.path.insert(0, ROOT)
    import bench
    assert d["config"] == dict(bench.CONFIG, parallelism="1 GPU")
    assert d["solves_per_s"] * 256 ** 3 == __import__("pytest").approx(d["value"])
