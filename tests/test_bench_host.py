"""Host-side helpers of bench.py (no GPU): the DRAM traffic the roofline line
takes from the committed ncu summaries is that of the section whose kernel
hash matches, never a neighbouring kernel's."""
import glob
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def sections(path):
    out, cur = [], None
    for line in open(path):
        key, _, val = line.partition("=")
        key, val = key.strip(), val.strip()
        if key == "kernel_hash":
            cur = val
        elif key == "dram_bytes_per_launch":
            out.append((cur, float(val)))
    return out


def test_profiled_traffic_matches_its_own_section():
    found = 0
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        for h, b in sections(path):
            if h != "n/a":
                assert bench.profiled_traffic(h) == b
                found += 1
    assert found >= 2  # the fused kernel and the toy segment kernel
    assert bench.profiled_traffic("n/a") is None
    assert bench.profiled_traffic("0" * 16) is None


def test_roofline_of_the_op_list():
    """t_roof = max(n B / BW, n sum N_op / R_op): the Crystal Ball + ARGUS step
    (1.01e8 FP32 events, 4 bytes each) with 2 exp, 2 log, 1 sqrt, 1 rcp and 8
    FMA per event at the given rates is compute bound at 123.8 us, so a
    217.2 us step reaches 0.57 of it."""
    import bench
    rates = {"ex2_approx_f32": 9.67e12, "lg2_approx_f32": 4.94e12, "sqrt_approx_f32": 4.97e12,
             "rcp_approx_f32": 4.97e12, "fp32_fma": 3.78e13}
    r = bench.roofline_8d("c5", "fp32", 101_000_000, 4, 0.2172, rates, 6790.7)
    assert r["bound"] == "alu"
    assert abs(r["t_compute_us"] - 123.8) < 0.1
    assert abs(r["t_hbm_us"] - 59.5) < 0.1
    assert abs(r["frac"] - 0.57) < 0.005
    assert abs(r["achieved"] * r["t_roof_us"] * 1e-6 / 101_000_000 - r["frac"]) < 1e-12
    # an HBM-bound case: one FMA per event and 8 bytes
    r = bench.roofline_8d("c1", "fp64", 10_000, 8, 0.01, {"fp64_fma": 1e18}, 8000.0)
    assert r["bound"] == "hbm" and abs(r["t_roof_us"] - 0.01) < 1e-9
