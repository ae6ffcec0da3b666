"""The JSON line bench.py prints: every key the benchmark contract names, with
sane types and values.  The reference arm (the CPU oracle) runs here; the
CUDA arm runs on a GPU on the small plain-method workload."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
COMMON = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
          "vs_baseline", "dtype", "data", "config", "e2e", "cpu_baseline")


def run_bench(*args, timeout=900):
    out = subprocess.run([sys.executable, "bench.py", *args], cwd=ROOT, stdout=subprocess.PIPE,
                         stderr=subprocess.PIPE, text=True, timeout=timeout)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def check_common(d, steps, warmup):
    for k in COMMON:
        assert k in d, k
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == steps and d["warmup"] == warmup
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["data"] == "synthetic" and isinstance(d["config"]["workload"], str)
    e = d["e2e"]
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in e, k
    c = d["cpu_baseline"]
    for k in ("value", "unit", "cores", "kind", "sample"):
        assert k in c, k
    assert c["kind"] == "oracle" and c["cores"] >= 1


def test_reference_arm_line():
    d = run_bench("--impl", "reference", "--steps", "1", "--warmup", "0")
    check_common(d, 1, 0)
    assert d["impl"] == "reference"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["cpu_baseline"]["value"] == d["value"]
    assert d["unit"] == "Gsegments/s"


@pytest.mark.gpu
def test_cuda_arm_line_on_the_tiny_workload():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    d = run_bench("--config", "tiny", "--steps", "3", "--warmup", "3")
    check_common(d, 3, 3)
    assert "impl" not in d or d["impl"] != "reference"
    assert d["unit"] == "Gsegments/s" and d["gpu_launches"] >= 3
    r = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in r, k
    assert r["bound"] == "hbm" and 0 < r["frac"] < 1.5 and r["unit"] == "GB/s"
    assert r["alu"]["bound"] == "alu" and 0 < r["alu"]["frac"] < 1.5
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert d["e2e"]["d2h_bytes_per_step"] == 256 * 256 * (4 + 4)     # float32 map + int32 counts
    assert d["e2e"]["h2d_bytes_per_step"] > 0
    clk = d["clocks"]
    for k in ("sm_mhz", "sm_max_mhz", "reasons"):
        assert k in clk, k
    assert d["fp32_vs_fp64_err"]["column"] <= 1e-5
