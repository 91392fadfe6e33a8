"""The benchmark's reference arm (the FP64 oracle on the host cores) prints
one JSON line with the fields of the benchmark contract, on the small
1000 x 1000 workload: no GPU is involved."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "c1",
                        "--steps", "2", "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["unit"] == "TFLOP/s"
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1 and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("c1_1000x1000")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_step_byte_model():
    """The whole-step byte figures the bench reports: at q = 2 the mixed
    path's algorithmic budget is 22 m n bytes (FP32 A read once and written
    as bf16, six bf16 passes, the projection reading FP32 A), and this
    implementation moves 32 m n (A read by both casts, the three bf16 parts
    written and read by the projection); the FP64 path reads A 2q+3 times."""
    sys.path.insert(0, ROOT)
    import bench
    m, n = 1000, 700
    alg, impl = bench.step_bytes(m, n, 2, "bf16", 4)
    assert alg == 22 * m * n and impl == 32 * m * n
    alg, impl = bench.step_bytes(m, n, 2, "f64", 8)
    assert alg == impl == 7 * 8 * m * n
    alg, impl = bench.step_bytes(m, n, 1, "bf16", 4)
    assert alg == 18 * m * n and impl == 28 * m * n
