"""Host arithmetic of bench.py's secondary ceilings (FP32 pipe, instruction issue)."""
import pytest

import bench


def test_other_ceilings_arithmetic():
    nodes, kt = 1000, [1e-6, 1e-6, 1e-6]
    peak = 78.5e12  # a measured FP32 fused multiply-add rate in flop/s
    oc = bench.other_ceilings(nodes, kt, {"sm_mhz": 1000.0}, peak)
    flops = nodes * sum(bench.STAGE_FP32_FLOP_PER_NODE) / 3e-6
    assert oc["fp32"]["achieved"] == pytest.approx(flops / 1e12)
    assert oc["fp32"]["peak"] == pytest.approx(78.5)
    assert oc["fp32"]["frac"] == pytest.approx(flops / peak)
    issue = nodes * sum(bench.STAGE_WARP_INSTR_PER_NODE) / 3e-6
    assert oc["issue"]["frac"] == pytest.approx(issue / (152 * 4 * 1e9))
    assert bench.other_ceilings(nodes, kt, {}, peak) is None        # no clock sample
    assert bench.other_ceilings(nodes, [0.0, 1e-6, 1e-6], {"sm_mhz": 1.0}, peak) is None


def test_workload_label_follows_the_element_count():
    assert bench.workload_label(1024) == bench.WORKLOAD
    assert "768x768" in bench.workload_label(768) and "9.4M nodes" in bench.workload_label(768)
