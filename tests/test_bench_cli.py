"""bench.py's reference arm (the FP64 oracle on the host cores) prints one
JSON line with the keys of the benchmark contract; runs on CPU."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1",
                        "--cpu-rays", "32", "--nsteps", "200"],
                       cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["unit"] == "ray-steps/s" and d["dtype"] == "f64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]


def test_secondary_workload_oracle_samples():
    """The oracle figures attached to the secondary measurements carry the
    cpu_baseline keys and a positive rate; a failure becomes an error field,
    never an exception."""
    sys.path.insert(0, ROOT)
    import bench
    r = bench._with_oracle({}, "luneburg")["cpu_baseline"]
    assert r["kind"] == "oracle" and r["value"] > 0 and r["cores"] >= 1
    assert r["unit"] == "ray-steps/s" and "1024 rays x 2000 RK4 steps, 25 times" in r["sample"]
    bad = bench._with_oracle({}, "no such workload")["cpu_baseline"]
    assert "error" in bad
