"""The roofline arithmetic of bench.py (host only): fractions are achieved
over peak, the reweighting's integer-op count matches a direct count of the
pair tiles, and the algorithmic fraction follows its definition."""
import math

import bench

PK = {"hbm_gbs": 6689.8, "bf16_tflops": 1908.3, "bf16_tflops_sustained": 1744.5,
      "sm_max_mhz": 2070.0}


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
    # timed alone on full evaluations: the burst peak is the denominator
    assert math.isclose(t["frac"], t["achieved"] / 1908.3)
    assert math.isclose(t["frac_of_sustained"], t["achieved"] / 1744.5)


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
    assert math.isclose(r["peak"], 152 * 128 * 2070e6 / 1e12)  # derived without measurements
    # with measured lop3 and popc rates the peak is the 6 + 1 mix's rate
    alu = {"lop3_b32": 40e12, "popc_b32": 5e12, "fadd_f32": 39e12}
    r = bench.kernel_rooflines({"reweight": (2, 0.2, 0)}, {}, B, N, PK, "measured", alu)["reweight"]
    assert math.isclose(r["peak"], 7.0 / max(6 / 40e12, 1 / 5e12) / 1e12)


def test_measured_fp32_add_rate_sets_the_algorithmic_fraction():
    B, N = 5000, 120
    alu = {"fadd_f32": 30e12}
    out = bench.kernel_rooflines({}, {"tc_logits": 130e-6, "logits_gather": 1e-3}, B, N, PK,
                                 "measured", alu)
    assert math.isclose(out["tc_logits"]["algorithmic_frac"], B * N * (N - 1) * 21 / 30e12 / 130e-6)
    g = out["logits_gather"]
    assert math.isclose(g["peak"], 30.0) and math.isclose(g["frac"], B * N * N * 21 / 1e-3 / 30e12)


def test_clock_summary_keeps_the_timed_window():
    import datetime
    base = datetime.datetime(2026, 1, 2, 3, 4, 5)

    def line(dt_s, mhz, slow="Not Active", cap="Not Active"):
        ts = (base + datetime.timedelta(seconds=dt_s)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return f"{ts}, 0, {mhz}, 2070, 900.0, 0x0, {slow}, Not Active, Not Active, {cap}"

    t0 = base.timestamp() + 1.0
    lines = [line(0.5, 1200, slow="Active"), line(1.05, 2070), line(1.10, 2040, cap="Active"),
             line(1.15, 2070), line(2.5, 1000)]
    c = bench.summarize_clocks(lines, t0, t0 + 0.2)
    assert c["samples"] == 3 and c["sm_mhz"] == 2070 and c["sm_max_mhz"] == 2070
    assert c["reasons"] == ["sw_power_cap"]  # the slowdown before the window is not counted
    # a window shorter than the sampling period keeps the nearest sample
    c = bench.summarize_clocks(lines, t0 + 0.085, t0 + 0.095)
    assert c["samples"] == 1 and c["sm_mhz"] == 2040
