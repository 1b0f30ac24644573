"""bench.py's own arm on the GPU prints one JSON line carrying every key of
the benchmark contract, with values that are consistent with each other."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu


def test_bench_line_contract():
    r = subprocess.run([sys.executable, "bench.py", "--steps", "3", "--warmup", "3"], cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e",
              "gpu_launches", "clocks", "roofline", "cpu_baseline"):
        assert k in d, k
    assert d["steps"] == 3 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["unit"] == "s" and d["higher_is_better"] is False and d["value"] > 0
    assert abs(d["ms_per_step"] - 1000 * d["value"]) < 1e-6 * max(1.0, d["ms_per_step"])
    assert d["config"]["workload"] and d["config"]["N"] == 120 and d["config"]["B"] == 5000
    assert d["gpu_launches"] > 0
    e = d["e2e"]
    assert e["value"] > 0 and e["unit"] == "s"
    assert e["h2d_bytes_per_step"] == 120 * 5000  # the int8 MSA
    assert e["d2h_bytes_per_step"] > 0
    roof = d["roofline"]
    assert roof["bound"] in ("tensor", "hbm", "alu") and roof["peak"] > 0
    assert 0 < roof["frac"] <= 1.5 and abs(roof["frac"] - roof["achieved"] / roof["peak"]) < 1e-9
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > d["value"]
    par = cb["parity_of_the_timed_solve"]  # the timed solve against the oracle's rundown
    assert par["fn_within_bound"] and par["top_L_within_bound"], par
    c = d["clocks"]
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(c)
    assert d["fp32_path"]["top_L_identical_to_split_bf16"] is True
    assert e.get("top_N_equal_to_device_run") is True
