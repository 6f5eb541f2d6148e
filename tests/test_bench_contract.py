"""The JSON line of bench.py: the reference arm (the CPU oracle) on CPU, and
the GPU arm on a small box, each with every key the line must carry."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BASE_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
             "vs_baseline", "dtype", "data", "config", "e2e", "cpu_baseline"}


def run_bench(*args, timeout=900):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                         text=True, timeout=timeout)
    assert out.returncode == 0, out.stderr[-3000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_arm_line():
    d = run_bench("--impl", "reference", "--steps", "1", "--warmup", "1", "--n", "24")
    assert BASE_KEYS <= set(d)
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


@pytest.mark.gpu
def test_gpu_arm_line():
    # 128^3: the coarser twins of the turbulence box reach p < 0 within the
    # steps this run takes (warm-up, timed step, per-operator timing, e2e)
    d = run_bench("--n", "128", "--steps", "1", "--warmup", "3", "--no-batch", "--no-fp64", "--no-cpu-baseline",
                  "--no-same-box")
    assert BASE_KEYS <= set(d) and {"roofline", "gpu_launches", "clocks"} <= set(d)
    r = d["roofline"]
    assert {"bound", "achieved", "peak", "unit", "frac", "traffic"} <= set(r)
    assert r["bound"] == "hbm" and 0 < r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert d["gpu_launches"] > 0 and d["value"] > 0 and d["n_gpus"] == 1
    e = d["e2e"]
    # a full round trip per step: the whole FP32 state up and down
    assert e["value"] > 0 and e["h2d_bytes_per_step"] == 32 * 128 ** 3 and e["d2h_bytes_per_step"] == 32 * 128 ** 3
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])


@pytest.mark.gpu
def test_gpu_decomposed_line():
    """--decomp on one GPU: the z-slab path with the rank exchanging ghost
    planes with itself (periodic), strong scaling."""
    d = run_bench("--decomp", "--n", "128", "--steps", "1", "--warmup", "3")
    assert {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "scaling"} <= set(d)
    assert d["scaling"] == "strong" and d["value"] > 0 and d["gpu_launches"] > 0
    assert d["exchanges_per_step"] == 13


def test_workload_names_follow_the_size():
    """The config of a line names the box it ran and says whether one FP32
    state copy exceeds the 129 MB L2 (1024^3: 34.4 GB; 128^3: 67 MB)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    assert "1024^3" in b.workload_name(1024) and "384^3" in b.workload_name(384)
    assert b.l2_note(1024).startswith("inputs larger than L2") and "34.4 GB" in b.l2_note(1024)
    assert b.l2_note(128).startswith("inputs fit in L2")
