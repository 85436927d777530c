"""The JSON line of bench.py on a small workload: one line, the keys and
types of the contract (scalar counts where counts are due, the e2e, roofline
and clocks objects), and a value consistent with the reported step time."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_schema():
    K = 3
    out = subprocess.run([sys.executable, "bench.py", "--workload", "tgv128", "--steps", str(K), "--warmup", "3",
                          "--no-extras", "--no-cpu-baseline"], cwd=ROOT, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert key in d, key
    assert d["n_gpus"] == 1 and d["steps"] == K and d["warmup"] == 3 and d["dtype"] == "f32"
    assert d["config"]["workload"] == "tgv128"
    # whole-job throughput from the step time: N cells per step
    assert d["value"] == pytest.approx(128 ** 3 / (d["ms_per_step"] * 1e-3), rel=1e-9)
    # counts are integers: four launches (CFL + three stages) per timed step
    passes = d["timing"]["passes"]
    assert isinstance(passes, int) and passes >= 1
    assert isinstance(d["gpu_launches"], int) and d["gpu_launches"] == 4 * K * passes
    assert len(d["timing"]["pass_ms"]) == passes
    e2e = d["e2e"]
    assert e2e["unit"] == d["unit"] and e2e["value"] > 0
    assert e2e["h2d_bytes_per_step"] == e2e["d2h_bytes_per_step"] == 5 * 128 ** 3 * 4
    assert len(e2e["pass_ms"]) == 5 and all(isinstance(x, float) for x in e2e["pass_ms"])
    r = d["roofline"]
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-12)
    assert 0 < r["frac"] < 1.5
    assert isinstance(d["clocks"]["reasons"], list)
