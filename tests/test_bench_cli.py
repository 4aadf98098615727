"""bench.py's command line on the CPU: the reference arm (the FP64 oracle on
the host cores) prints one JSON line with the fields the benchmark contract
names, on a bounded sample; the GPU arm's flags parse."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--cpu-rays", "16", "--nsteps", "200"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["cpu_model"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_gpu_arm_flags_parse():
    sys.path.insert(0, ROOT)
    import bench
    argv = sys.argv
    try:
        sys.argv = ["bench.py", "--gpus", "2", "--workload", "adjoint", "--scaling", "strong", "--drawn-order"]
        a = bench.parse()
    finally:
        sys.argv = argv
    assert a.gpus == 2 and a.workload == "adjoint" and a.scaling == "strong" and a.drawn_order
    assert bench.MODEL_GRIN_RAY_STEP == 1292 and bench.MODEL_DOPRI5_ATTEMPT == 1092
