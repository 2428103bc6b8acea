"""bench.py on the GPU prints one JSON line with every key of the benchmark contract (a short run:
2 timed steps after 3 warm-up steps)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_has_the_contract_keys():
    r = subprocess.run([sys.executable, "bench.py", "--steps", "2", "--warmup", "3", "--equil", "2", "--no-cpu"],
                       cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert k in line, k
    assert line["n_gpus"] == 1 and line["steps"] == 2 and line["warmup"] == 3 and line["value"] > 0
    assert line["gpu_launches"] == 2 * line["steps"]  # queue init + sweep per step
    rf = line["roofline"]
    assert rf["bound"] == "alu" and 0 < rf["frac"] < 1.5 and rf["peak"] > 0
    e2e = line["e2e"]
    assert e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0 and e2e["value"] > 0
    assert line["config"]["workload"] and line["E_per_atom"]["E"] < 0
