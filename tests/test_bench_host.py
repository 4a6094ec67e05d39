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
