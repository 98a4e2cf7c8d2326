"""bench.py's reference arm (the CPU oracle as it stands) keeps the JSON contract: one line with
the metric, value, unit, the timing keys, a cpu_baseline describing the run and an e2e entry
with no host-device traffic.  CPU only; the sample is a single RK4IP step per bench step."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--ref-seconds", "0.01"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["unit"] == "mode-steps/s" and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"]
    assert cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_fp32_vs_fp64_error_helper():
    """The helper behind the bench line's FP32-against-FP64 errors: relative L2 of the field
    and of the power spectrum per instance."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    c = [np.array([1.0 + 0j, 2j]), np.array([3.0, 4.0 + 0j])]
    a = [c[0] * (1 + 1e-6), c[1] + np.array([0.0, 1e-3])]
    field, power = bench.fp32_vs_fp64_errors(a, c)
    assert abs(field[0] - 1e-6) < 1e-12 and abs(field[1] - 1e-3 / 5.0) < 1e-12
    assert abs(power[0] - ((1 + 1e-6) ** 2 - 1)) < 1e-12
    assert abs(power[1] - abs(4.001 ** 2 - 16.0) / np.hypot(9.0, 16.0)) < 1e-12
