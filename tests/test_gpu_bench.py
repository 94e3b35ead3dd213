"""The benchmark itself on a reduced case (300 strokes at 256^2): bench.py runs
on the GPU, prints one JSON line with the keys of its contract, and its
pipelined end-to-end path (the upload of step k + 1 on a copy stream while
step k computes, two input buffers) reads back the same gradients, bit for
bit, as a step on device-resident inputs: the overlap reorders no data."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "clocks", "gpu_launches")


def test_bench_line_and_pipelined_e2e():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "3", "--warmup", "3", "--fit-steps", "1",
           "--no-cpu-baseline", "--serve-requests", "0", "--no-memory", "--no-hard", "--no-peaks",
           "--res", "256", "--strokes", "300"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    for k in KEYS:
        assert k in d, k
    e2e = d["e2e"]
    assert e2e["gradients_match_device_step"] is True
    assert e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    assert e2e["value"] > 0 and d["value"] > 0
    assert d["steps"] == 3 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["gpu_launches"] > 0
    assert 0.0 < d["roofline"]["frac"] < 1.5
