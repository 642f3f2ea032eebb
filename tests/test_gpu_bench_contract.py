"""The bench's main arm on a small workload (20,000 sets, 100 queries): one JSON
line whose timing, roofline, clock, end-to-end and launch fields are present and
self-consistent."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_main_arm_small_workload_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--workload", "small", "--steps", "2", "--warmup", "3",
                        "--no-extras", "--no-cpu-baseline"], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    B, n_sets = d["config"]["queries"], d["config"]["n_sets"]
    assert (B, n_sets) == (100, 20_000)
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1 and d["unit"] == "doc-sets/s"
    # value = pairs scored per second of the timed steps
    assert abs(d["value"] - B * n_sets / (d["ms_per_step"] * 1e-3)) <= 1e-6 * d["value"]
    st = d["stages"]
    assert 0 < st["maxsim_bf16_ms"] < d["ms_per_step"]
    assert 0 < st["fp32_rerank_ms"] < d["ms_per_step"]
    rf = d["roofline"]
    assert rf["bound"] == "tensor" and rf["unit"] == "TFLOP/s" and rf["peak"] > 0
    assert abs(rf["frac"] - rf["achieved"] / rf["peak"]) <= 1e-9
    assert abs(rf["achieved"] - 2.0 * B * 32 * d["config"]["n_vecs"] * 128 / (st["maxsim_bf16_ms"] * 1e-3) / 1e12) \
        <= 1e-6 * rf["achieved"]
    assert d["gpu_launches_per_step"] >= 5 and d["gpu_launches"] == 2 * d["gpu_launches_per_step"]
    assert "sm_mhz" in d["clocks"] and "reasons" in d["clocks"]
    e2e = d["e2e"]
    assert e2e["value"] > 0 and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == B * 32 * 128 * 4 + (B + 1) * 8
    assert e2e["d2h_bytes_per_step"] == B * d["config"]["k"] * 12
    assert "cpu_baseline" not in d
