"""The benchmark's JSON line on a GPU: one short run of bench.py (3 warm-up
and 3 timed frequencies of the headline workload, no CPU baseline) and the
keys and invariants its consumers rely on: the metric and its unit, the
device-timed value and the end-to-end value with the bytes copied, the
roofline of the dominant kernel with its peak, the clocks sampled during the
timed region, the launch count, the single-frequency path, and the FP64
residual of the result."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.gpu
def test_bench_line_keeps_its_contract():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "3", "--warmup", "3",
                        "--no-cpu-baseline"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["metric"] and d["unit"] == "matvecs/s" and d["n_gpus"] == 1
    assert d["steps"] == 3 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0
    # every step is one GMRES solve: products per second = products / time
    assert abs(d["value"] * d["ms_per_step"] / 1e3 - d["matvecs_per_solve"]) < 0.02 * d["matvecs_per_solve"]
    assert d["config"]["workload"] == "sphere20480_4k" and d["config"]["n_elements"] == 20480
    e = d["e2e"]
    assert e["value"] > 0 and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] >= 2 * 20480 * 8
    ro = d["roofline"]
    assert ro["bound"] == "hbm" and ro["unit"] == "GB/s" and ro["peak"] > 0
    assert 0.0 < ro["frac"] < 1.5 and abs(ro["frac"] - ro["achieved"] / ro["peak"]) < 1e-3
    c = d["clocks"]
    assert c["sm_mhz"] > 0 and c["sm_max_mhz"] >= c["sm_mhz"] and isinstance(c["reasons"], list)
    assert d["gpu_launches"] > 100 * d["steps"]
    sf = d["single_frequency"]
    assert sf["value"] > 0 and sf["ms_per_step"] > 0 and sf["unit"] == d["unit"]
    assert d["rel_error"]["fp64_residual_sampled_rows"] < 1e-4
    assert "cpu_baseline" not in d
