"""bench.py prints one JSON line with the fields its callers rely on, for the GPU arm
(reduced lattice) and for the reference arm (the oracle on the host)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BASE_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
             "vs_baseline", "dtype", "data", "config", "e2e"}


def _run(args, timeout=900):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                       timeout=timeout, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_json():
    d = _run(["--impl", "reference", "--small", "--steps", "1", "--warmup", "1"])
    assert d["impl"] == "reference"
    assert BASE_KEYS <= set(d)
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["value"] > 0


@pytest.mark.gpu
def test_gpu_arm_json():
    d = _run(["--small", "--steps", "1", "--warmup", "1", "--no-cpu-baseline", "--no-fp32"])
    assert BASE_KEYS <= set(d)
    assert {"roofline", "clocks", "gpu_launches"} <= set(d)
    r = d["roofline"]
    assert r["bound"] in ("hbm", "alu") and r["peak"] > 0 and 0 < r["frac"] < 1.5
    assert d["gpu_launches"] > 0 and d["value"] > 0 and d["e2e"]["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["d2h_bytes_per_step"] > 0
    # the FP64 workload's moment rows run on pairs of FP32 numbers by default
    assert d["dtype"] in ("f64", "f32x2") and d["scaling"] == "weak"
    assert "arith" in d["config"]
