"""The benchmark's roofline arithmetic on the host (no GPU): per kernel family, the binding
roof is the larger of the two time floors (algorithmic bytes over the measured HBM copy
bandwidth, algorithmic flops over the family's compute peak), `frac` is measured against
that roof, and `alu_frac` gives the compute side whichever roof binds."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
bench = pytest.importorskip("bench")


def fam(name, ms, flops, nbytes, launches=10):
    return {"name": name, "launches": launches, "ms": ms, "flops": flops, "bytes": nbytes}


def test_fp64_family_alu_bound():
    # 1 TFLOP in 1 s on a 1.26 TFLOP/s FP64 roof, a few bytes: ALU-bound
    r = bench.roofline_entry(fam("spmm_A", 1000.0, 1e12, 1e6), n=1024, s=8, fp64_probe=1.05)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(bench.FP64_NOMINAL_TFLOPS)
    assert r["frac"] == pytest.approx(1.0 / bench.FP64_NOMINAL_TFLOPS)
    assert r["alu_frac"] == pytest.approx(r["frac"])
    assert "1.050 TFLOP/s" in r["peak_source"]


def test_fp32_unit_override_and_alu_frac_when_hbm_binds():
    hbm = bench._peaks()[0]
    # bytes that take 1 ms at the copy bandwidth, flops that take 0.1 ms on the FP32 roof,
    # measured over 10 ms: HBM binds at 0.1, the ALU side sits at 0.01
    nbytes = hbm * 1e9 * 1e-3
    flops = bench.FP32_NOMINAL_TFLOPS * 1e12 * 1e-4
    r = bench.roofline_entry(fam("spai_columns", 10.0, flops, nbytes), n=1024, s=8, fp32_probe=74.6, unit="fp32")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["frac"] == pytest.approx(0.1)
    assert r["alu_frac"] == pytest.approx(0.01)
    # the same family as FP64 work: the FP64 roof binds instead
    r64 = bench.roofline_entry(fam("spai_columns", 10.0, flops, nbytes), n=1024, s=8)
    assert r64["bound"] == "alu" and r64["peak"] == pytest.approx(bench.FP64_NOMINAL_TFLOPS)


def test_latency_family_has_no_roof():
    r = bench.roofline_entry(fam("arnoldi_ls", 1.0, 10.0, 0.0), n=1024, s=8)
    assert r["bound"] == "latency" and r["frac"] is None and r["achieved"] is None


def test_tensor_family_traffic_scales_with_blocks():
    # the Gram product's DRAM traffic model: (8 B per entry per block + fitted constant) n s
    n, s = 262144, 8
    per_launch = 8.0 * n * s * 17  # 16 basis blocks + W
    r = bench.roofline_entry(fam("block_dot_tc", 1.0, 2.0 * n * s * s * 16, per_launch, launches=1), n=n, s=s)
    a, b = bench.NCU_TRAFFIC["block_dot_tc"]
    assert r["traffic"] == pytest.approx((a * 17 + b) * n * s)
    assert r["bound"] == "hbm"
