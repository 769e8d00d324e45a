"""bench.py end to end on the GPU (short runs): the JSON line of an HBM-bound FP32
workload and of an FP64-pipe-bound workload carries every field of the contract."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "roofline", "clocks", "gpu_launches")


@pytest.mark.parametrize("workload,bound", [("ch2d-4096-f32-lap5", "hbm"), ("ac2d-256-f64-lap5", "alu"),
                                            ("ch3d-384-f32-lap7", "hbm")])
def test_bench_line(workload, bound):
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--workload", workload, "--steps", "2", "--warmup", "3",
           "--no-served", "--no-cpu-baseline", "--no-e2e"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in KEYS:
        assert k in line, k
    roof = line["roofline"]
    assert roof["bound"] == bound and roof["achieved"] > 0 and 0 < roof["frac"] < 2
    assert line["value"] > 0 and line["gpu_launches"] > 0
    if bound == "alu":
        assert roof["measured_fp64_gops"] > 0
