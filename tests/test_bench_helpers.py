"""Host arithmetic of the benchmark's roofline objects (no GPU): the learned
tail's bound from its MUFU operations per pair and its network flops, the
choice of the binding pipe, and which lines carry the committed ncu DRAM
figure."""
import math

import bench


def test_learned_tail_bound_from_unit_counts():
    # n0 = 4: 9 near-image rsqrt, 4 rsqrt + 2 rcp of the base, 1 rsqrt of dR = 16 MUFU ops per pair
    r = bench.surrogate_roofline(152, 2070.0, 4, pairs=1.0e11, kernel_s=1.0)
    mufu_peak = 152 * 2070e6 * bench.MUFU_RSQRT_PER_SM_CLK / 16
    assert r["bound"] == "alu" and math.isclose(r["peak"], mufu_peak, rel_tol=1e-12)
    assert math.isclose(r["achieved"], 1.0e11) and math.isclose(r["frac"], 1.0e11 / mufu_peak)
    # the network alone: 2 (3 x 32 + 32 x 32 + 32 x 2) = 2368 flops per pair at the tensor rate
    assert "2368 network flops" in r["peak_basis"]


def test_bound_scales_with_the_near_range():
    # MUFU ops per pair: 2 n0 + 1 near images + 4 rsqrt and 2 rcp of the base + 1 rsqrt of dR
    r0 = bench.surrogate_roofline(152, 2070.0, 0, 1.0, 1.0)    # 8 ops: still under the tensor bound
    r50 = bench.surrogate_roofline(152, 2070.0, 50, 1.0, 1.0)  # 108 ops
    assert r0["bound"] == "alu" and r50["bound"] == "alu"
    assert math.isclose(r0["peak"] / r50["peak"], 108 / 8, rel_tol=1e-12)


def test_only_the_headline_carries_the_dram_figure():
    head = bench.surrogate_roofline(152, 2070.0, 4, 1.0, 1.0)
    other = bench.surrogate_roofline(152, 2070.0, 4, 1.0, 1.0, headline=False)
    assert other["traffic"] is None
    assert head["traffic"] == bench.recorded_traffic("surrogate")
    t = bench.recorded_traffic("surrogate")
    assert t is None or t > 0
    assert len(bench.kernel_source_hash("surrogate")) == 16
