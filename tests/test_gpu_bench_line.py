"""The benchmark's JSON line on the GPU: a short run with a fixed schedule
prints one line with the metric, the step timing, the HBM roofline of the
dominant kernel and of the whole step, per-kernel medians and quartiles, the
end-to-end figure with its copied bytes, the launch count, the clocks and the
native-FP64 figure of the same schedule, all consistent with each other."""

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SCHED = {"fusion": 1, "staging": 0, "tile_i": 32, "tile_j": 8, "unroll": 1, "k_chunk": 4, "arith": 2}


def test_bench_line_keys_and_consistency():
    r = subprocess.run([sys.executable, "bench.py", "--steps", "20", "--warmup", "3", "--no-cpu-baseline",
                        "--schedule", json.dumps(SCHED)], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks", "kernels",
              "native_f64", "issue_rate", "fp64_equivalent_rate"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 20 and d["warmup"] == 3 and d["higher_is_better"] is True
    n = 128 * 128 * 80
    assert d["value"] == pytest.approx(n / (d["ms_per_step"] * 1e-3), rel=1e-6)
    assert d["config"]["schedule"]["arith"] == 2 and d["config"]["schedule"]["tile_j"] == 8
    rf = d["roofline"]
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and 0 < rf["frac"] < 1
    assert rf["frac"] == pytest.approx(rf["achieved"] / rf["peak"], rel=1e-9)
    assert rf["step"]["algorithmic_bytes"] == 64327680
    assert rf["step"]["achieved"] == pytest.approx(64327680 / (d["ms_per_step"] * 1e-3) / 1e9, rel=1e-6)
    names = [k["name"] for k in d["kernels"]]
    assert names == ["hdiff_fixed_kernel", "hv_thomas_kernel"]
    for k in d["kernels"]:
        assert k["q1"] <= k["median"] <= k["q3"] and k["n"] == 20
    assert d["gpu_launches"] == 2 * 20
    e = d["e2e"]
    assert e["h2d_bytes_per_step"] > 40e6 and e["d2h_bytes_per_step"] == 2 * n * 8
    assert 0 < e["value"] < d["value"]
    assert d["native_f64"]["schedule"]["arith"] == 0
    c = d["clocks"]
    if c.get("samples"):   # nvidia-smi sampled the timed region
        assert c["sm_max_mhz"] >= c["sm_mhz"] > 0
    else:
        assert c["reasons"] == ["unsampled"]
