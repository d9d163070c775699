"""bench.py on the GPU, short form: one JSON line carrying every key the
benchmark reports (throughput, end to end through host buffers, roofline of
the batch kernel, clocks, kernel launches, the timed CPU oracle), with the
bit-exact gate passed on the timed batch."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--quick",
                        "--steps", "5", "--warmup", "3", "--cpu-budget", "2"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    out = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "e2e", "roofline", "clocks", "gpu_launches", "cpu_baseline"):
        assert key in out, key
    assert out["n_gpus"] == 1 and out["steps"] == 5 and out["warmup"] == 3
    assert out["higher_is_better"] is True and out["scaling"] == "weak"
    assert out["value"] > 0 and out["ms_per_step"] > 0
    assert out["gpu_launches"] >= out["steps"]
    cfg = out["config"]
    assert cfg["workload"] and cfg["exact"] is True and cfg["exact_images_checked"] > 0
    e2e = out["e2e"]
    assert e2e["exact"] is True and e2e["value"] > 0 and e2e["unit"] == out["unit"]
    assert e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    assert e2e["value"] < out["value"]          # the host link is slower than HBM
    roof = out["roofline"]
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert 0 < roof["frac"] < 1.3
    assert abs(roof["frac"] - roof["achieved"] / roof["peak"]) < 1e-3
    clocks = out["clocks"]          # the short run may end before a clock sample
    assert clocks is None or {"sm_mhz", "sm_max_mhz", "reasons"} <= set(clocks)
    cpu = out["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["value"] > 0 and cpu["cores"] >= 1
    assert cpu["unit"] == out["unit"] and cpu["sample"]
