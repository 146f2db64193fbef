"""The benchmark's reference arm (the CPU oracle timed on the host cores) on
a small mesh, without a GPU: one JSON line with the keys the benchmark
contract fixes, the same metric and unit as the GPU arm, and a CPU baseline
that describes the run."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "12",
                          "--steps", "2", "--warmup", "1"], cwd=ROOT, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["metric"] == "limited-convection face-updates/s (fused SSP-RK3 step)"
    assert line["unit"] == "face-updates/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 2 and line["warmup"] == 1
    # the same workload keys as the GPU arm's line, and whole SSP-RK3 steps
    cfg = line["config"]
    assert cfg["cells"] == 12 ** 3 and cfg["faces"] == 3 * 12 ** 3 and cfg["rk_order"] == 3
    assert "whole SSP-RK3 step" in line["cpu_baseline"]["sample"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
