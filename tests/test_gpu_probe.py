"""Throughput probes (instrumentation): the sustained pipe rates stay within
GB300's unit counts (128 FP32 lanes, 32 MUFU ex2 and 2 FP64 FMA lanes per
clock per SM, the figures the derived rooflines use) and well above a
fraction of them; the FP64 exponential rate (the FP64 grid pass's measured
roofline) is below the FP64 FMA rate."""
import pytest

from paper_1607_05816_gb300 import uot as U

pytestmark = pytest.mark.gpu


def test_probe_pipes_within_unit_counts():
    r = U.probe_pipes()
    assert 0.5 * 128 <= r["ffma_per_clk_per_sm"] <= 128 * 1.02
    assert 0.5 * 32 <= r["mufu_ex2_per_clk_per_sm"] <= 32 * 1.02
    assert 0.25 <= r["dfma_per_clk_per_sm"] <= 64 * 1.02
    # an FP64 exponential takes several FP64 pipe operations
    assert 0.0 < r["dexp_per_clk_per_sm"] < r["dfma_per_clk_per_sm"]
