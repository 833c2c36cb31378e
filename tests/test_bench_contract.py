"""bench.py's reference arm on the host (no GPU): the FP64 oracle timed on a bounded slice
of the default workload prints one JSON line with the GPU arm's metric, unit and workload
config, the `impl`, `cpu_baseline` and `e2e` keys, and W untimed warm-up steps."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3",
                          "--ref-rows", "8"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    sys.path.insert(0, ROOT)
    import bench

    assert line["impl"] == "reference"
    assert (line["metric"], line["unit"], line["higher_is_better"]) == ("MLUPS", "MLUPS", True)
    assert line["steps"] == 2 and line["warmup"] == 3 and line["value"] > 0
    assert line["config"]["workload"] == bench.workload_config("fp32")["workload"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
