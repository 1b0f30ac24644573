"""The roofline arithmetic of bench.py (host only): fractions are achieved
over peak, the reweighting's integer-op count matches a direct count of the
pair tiles, and the algorithmic fraction follows its definition."""
import math

import bench

PK = {"hbm_gbs": 6689.8, "bf16_tflops_sustained": 1744.5, "sm_max_mhz": 2070.0}


def test_hbm_and_tensor_entries():
    kern = {"lbfgs_commit": (4, 2.0, 4 * 1.0e9)}  # 4 launches, 2 ms, 1 GB each
    out = bench.kernel_rooflines(kern, {"tc_logits": 100e-6}, 1000, 50, PK, "measured")
    c = out["lbfgs_commit"]
    assert c["bound"] == "hbm" and math.isclose(c["achieved"], 2000.0)
    assert math.isclose(c["frac"], 2000.0 / 6689.8)
    t = out["tc_logits"]
    flops = 2 * 2 * 1000 * (50 * 21) * (50 * 21 + 1)
    assert t["flops_per_launch"] == flops
    assert math.isclose(t["achieved"], flops / 100e-6 / 1e12)
    assert math.isclose(t["frac"], t["achieved"] / 1744.5)


def test_algorithmic_fraction():
    B, N = 5000, 120
    out = bench.kernel_rooflines({}, {"tc_grad": 122e-6}, B, N, PK, "measured")
    adds_t = B * N * (N - 1) * 21 / (152 * 128 * 2070e6)
    bytes_t = (N * 21 * (N * 21 + 1) * 4 + B * N) / (6689.8e9)
    assert math.isclose(out["tc_grad"]["algorithmic_frac"], max(adds_t, bytes_t) / 122e-6)
    assert adds_t > bytes_t  # the method's adds, not its bytes, bound the family workload


def test_reweight_integer_ops():
    B, N = 300, 70  # 5 tiles of 64 rows (the last ragged), 3 words per row
    out = bench.kernel_rooflines({"reweight": (2, 0.2, 0)}, {}, B, N, PK, "measured")
    tiles = 5
    pairs = sum(1 for a in range(tiles) for b in range(tiles) if a <= b) * 64 * 64
    ops = pairs * 3 * 7
    r = out["reweight"]
    assert r["bound"] == "alu" and r["ops_per_launch"] == ops
    assert math.isclose(r["achieved"], ops / 0.1e-3 / 1e12)
    assert math.isclose(r["peak"], 152 * 128 * 2070e6 / 1e12)
