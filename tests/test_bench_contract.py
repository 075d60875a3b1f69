"""The JSON line of bench.py: every key of the measurement contract, for the oracle
(reference) arm on the host and for the CUDA arm on a small mesh."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BASE_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
             "scaling", "vs_baseline", "dtype", "data", "config", "e2e"}


def run_bench(*args, timeout=900):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                       text=True, timeout=timeout)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-3000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    d = run_bench("--impl", "reference", "--N", "16", "--steps", "3", "--warmup", "3")
    assert BASE_KEYS <= set(d)
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "Mtets/s"
    assert d["steps"] == 3 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("3D P1 stiffness")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert cb["host"]["logical_cpus"] >= 1 and cb["host"]["model"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


@pytest.mark.gpu
def test_gpu_arm_line():
    pytest.importorskip("torch")
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = run_bench("--N", "24", "--steps", "4", "--warmup", "3", "--no-tune", "--no-secondary")
    assert BASE_KEYS <= set(d)
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["scaling"] == "weak" and d["vs_baseline"] is None
    assert "l2" in d["config"] and d["config"]["workload"].startswith("3D P1 stiffness")
    r = d["roofline"]
    assert {"bound", "achieved", "peak", "unit", "frac", "traffic"} <= set(r)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["achieved"] > 0 and r["peak"] > 0
    assert d["roofline_alu"]["bound"] == "alu"  # the FP64 form's FP64-pipe fraction beside it
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] == 2 * d["steps"]  # chunk kernel + fixup per step
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])
    assert {"f64", "f32", "f64x"} <= set(d["forms"])
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] > 0


@pytest.mark.gpu
def test_gpu_workload_line():
    pytest.importorskip("torch")
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = run_bench("--workload", "2d", "--steps", "3", "--warmup", "2")
    assert d["workload"] == "2d" and d["value"] > 0 and d["unit"] == "Mtris/s"
    for form in ("f64", "f32", "f64x"):
        f = d["forms"][form]
        assert f["value"] > 0 and f["ms_per_step"] > 0 and "chunk" in f["kernels_ms"]
