"""The committed benchmark record (profiles/bench_n4_level7_walks1048576.json)
is one JSON line of bench.py's contract, internally consistent: the
roofline fraction is achieved / peak, the reported DRAM traffic belongs to
the walk-kernel source it was captured on, the clocks saw no throttling, the
end-to-end figure moved bytes each step, and the step's split adds up."""
import json
import os

import bench

RECORD = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles",
                      "bench_n4_level7_walks1048576.json")


def load():
    with open(RECORD) as f:
        lines = [ln for ln in f if ln.strip()]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_record_has_the_contract_keys():
    r = load()
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "clocks",
                "gpu_launches"):
        assert key in r, key
    assert r["metric"] == "walk_steps_per_sec" and r["unit"] == "walk_steps/s" and r["higher_is_better"]
    assert r["warmup"] >= 3 and r["steps"] >= 1 and r["gpu_launches"] > 0
    assert r["config"]["workload"].startswith("n4_t7_level7_walks1048576_L64")
    assert r["config"]["workload"].split("_")[2] == "level7" and r["config"]["dp_bits"] == 12


def test_roofline_and_timing_are_consistent():
    r = load()
    roof = r["roofline"]
    assert roof["bound"] in ("alu", "tensor") and roof["peak"] > 0
    assert abs(roof["frac"] - roof["achieved"] / roof["peak"]) < 1e-9
    if roof["bound"] == "tensor":
        # the tensor-core shape: f16 flops against the measured dense peak, and
        # the same multiply-adds against the mma.sync rate it issues on
        assert roof["kernel"] == "k_walks<4,3>" and roof["unit"] == "TFLOP/s"
        ms = roof["mma_sync"]
        assert abs(ms["achieved_mac_per_s"] / 2 - roof["achieved"] * 1e12 / 4) / ms["achieved_mac_per_s"] < 1e-9
        assert abs(ms["frac"] - ms["achieved_mac_per_s"] / ms["peak_mac_per_s"]) < 1e-9
    # steps per bench step / seconds per bench step = the headline value
    steps_per_step = r["config"]["walks"] * r["config"]["steps_per_walk_per_step"]
    assert abs(r["value"] - steps_per_step / (r["ms_per_step"] / 1e3)) / r["value"] < 0.02
    rec = bench.WALK_NCU.get(roof["kernel"])
    if roof["traffic"] is not None and rec and rec["dram_bytes_per_launch"] is not None:
        assert roof["traffic"] == rec["dram_bytes_per_launch"]


def test_clocks_and_e2e():
    r = load()
    clk = r["clocks"]
    assert not {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"} & set(clk["reasons"])
    assert clk["sm_mhz"] >= 0.9 * clk["sm_max_mhz"]
    e2e = r["e2e"]
    assert e2e["unit"] == r["unit"] and e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    cpu = r["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] > 0


def test_step_split_and_extras():
    r = load()
    sp = r["step_split_ms"]
    assert abs(sp["walk_ms"] + sp["rewalk_ms"] + sp["collect_ms"] - r["ms_per_step"]) / r["ms_per_step"] < 0.02
    for key in ("tto_walk_cfg1", "tto_walk_cfg2", "tto_walk_cfg3"):
        t = r[key]
        assert t["mode"] == "walk" and t["status"] == "found" and t["exhaustive_points"] == 0
    s = r["serving"]
    assert 0 <= s["miss_rate"] < 1 and s["p99_all_s"] >= s["p50_all_s"]
    assert sum(s["status_counts"].values()) == 2000


def test_tensor_roofline_arithmetic():
    """bench.walk_roofline for the tensor-core shape on made-up inputs: the
    achieved flops are 4 per 16-bit-weight multiply-add (two f16 byte-plane
    multiply-adds), against the measured dense bf16 peak; the mma.sync
    fraction counts the same multiply-adds twice against the given rate; the
    dp4a shapes stay ALU-bound against twice the dp4a rate."""
    n, w_steps, steps, walk_s = 4, 1_000_000, 2_000_000, 0.5
    d = 4 ** n - 1
    macs = w_steps * 2 * d * d / walk_s
    r = bench.walk_roofline("k_walks<4,3>", n, w_steps, steps, walk_s, 1, 1e13, 2070.0, 152, hmma_per_s=3e14)
    peak, _ = bench.measured_tensor_tflops(sustained=True)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - 4 * macs / 1e12) < 1e-9 and r["peak"] == peak
    assert abs(r["frac"] - r["achieved"] / peak) < 1e-12
    assert abs(r["mma_sync"]["frac"] - 2 * macs / 3e14) < 1e-12
    assert abs(r["dp4a_equivalent"]["frac"] - macs / 2e13) < 1e-12
    r0 = bench.walk_roofline("k_walks<4,0>", n, w_steps, steps, walk_s, 1, 1e13, 2070.0, 152)
    assert r0["bound"] == "alu" and abs(r0["frac"] - macs / 2e13) < 1e-12
