"""Host-side pieces of bench.py that need no GPU: the committed ncu summary
parses, and the kernel-source hash that gates its traffic figure is stable."""
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_column_pass_summary_has_the_keys_bench_reads():
    vals = {}
    for line in open(os.path.join(ROOT, "profiles", "k_col_tc_geno_int8.md")):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    assert len(vals["kernel_source_sha256"]) == 16
    assert float(vals["dram_bytes_per_launch"]) > 5.05e8  # at least the algorithmic bytes
    # the traffic is reported only for the kernel sources it was measured on
    expect = float(vals["dram_bytes_per_launch"]) if vals["kernel_source_sha256"] == bench.kernel_hash() else None
    assert bench.ncu_traffic(bench.kernel_hash()) == expect
    assert bench.ncu_traffic("0" * 16) is None


def test_kernel_hash_is_deterministic():
    assert bench.kernel_hash() == bench.kernel_hash()
    assert len(bench.kernel_hash()) == 16


def test_measured_peak_is_read():
    peak, kind = bench.measured_peaks()
    assert peak > 1000.0 and kind in ("measured", "fallback")
