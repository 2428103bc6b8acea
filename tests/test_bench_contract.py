"""The reference arm of bench.py (the FP64 oracle on the host cores) prints one JSON line with the
keys of the benchmark contract; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert "workload" in line["config"]


def test_warmup_below_three_is_rejected():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--warmup", "2"],
                       cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert r.returncode != 0


def test_recompute_count_matches_the_sweep_rule():
    """The benchmark line's ln psi drift is averaged over the recomputes of the timed steps; the
    count must match the sweep's rule (a recompute after sweep k when (k + 1) % every == 0)."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    rng = np.random.default_rng(7)
    for every in (1, 5, 50):
        before = rng.integers(0, 400, size=200)
        after = before + rng.integers(0, 300, size=200)
        brute = [sum((k + 1) % every == 0 for k in range(b, a)) for b, a in zip(before, after)]
        assert list(bench.recomputes_between(before, after, every)) == brute
