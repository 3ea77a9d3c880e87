"""Host arithmetic of bench.py's secondary ceilings (FP32 pipe, instruction issue)."""
import pytest

import bench


def test_other_ceilings_arithmetic():
    nodes, kt = 1000, [1e-6, 1e-6, 1e-6]
    peak = 78.5e12  # a measured FP32 fused multiply-add rate in flop/s
    ctr = {"current": True, "fp32_flop_per_node": (300.0, 310.0, 320.0), "warp_instr_per_node": (15.0, 16.0, 17.0)}
    oc = bench.other_ceilings(nodes, kt, {"sm_mhz": 1000.0}, peak, ctr)
    flops = nodes * 930.0 / 3e-6
    assert oc["fp32"]["achieved"] == pytest.approx(flops / 1e12)
    assert oc["fp32"]["peak"] == pytest.approx(78.5)
    assert oc["fp32"]["frac"] == pytest.approx(flops / peak)
    issue = nodes * 48.0 / 3e-6
    assert oc["issue"]["frac"] == pytest.approx(issue / (152 * 4 * 1e9))
    assert bench.other_ceilings(nodes, kt, {}, peak, ctr) is None        # no clock sample
    assert bench.other_ceilings(nodes, [0.0, 1e-6, 1e-6], {"sm_mhz": 1.0}, peak, ctr) is None
    # counters of a kernel that changed since their capture are not used
    assert bench.other_ceilings(nodes, kt, {"sm_mhz": 1000.0}, peak, dict(ctr, current=False)) is None
    # no FP32 flop count (paired instructions): the issue fraction alone
    oc = bench.other_ceilings(nodes, kt, {"sm_mhz": 1000.0}, peak, dict(ctr, fp32_flop_per_node=None))
    assert "fp32" not in oc and oc["issue"]["frac"] == pytest.approx(issue / (152 * 4 * 1e9))


def test_stage_counters_name_both_kernels():
    for fam in ("node", "line"):
        c = bench.STAGE_COUNTERS[fam]
        assert {"kernel", "current", "dram_bytes_per_node", "fp32_flop_per_node", "warp_instr_per_node"} <= set(c)
        assert "TX" in c["kernel"] and "TY" in c["kernel"]


def test_workload_label_follows_the_element_count():
    assert bench.workload_label(1024) == bench.WORKLOAD
    assert "768x768" in bench.workload_label(768) and "9.4M nodes" in bench.workload_label(768)
