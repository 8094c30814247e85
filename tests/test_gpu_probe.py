"""The issue-rate probe behind the roofline denominator, through the C ABI.

An SM has 4 sub-partitions of 32 lanes, each issuing at most one warp
instruction per clock, and an instruction does at most two FP32 operations
per lane (paired FP32 forms) or two integer adds (three-input add).  So no
probe can exceed 2 x 128 lane-operations per SM per clock per operation it
counts in one instruction; the count-pass step (6 operations, at least 5
instructions: subtract, two compares, two adds) stays under 6/5 x 2 x 128.
A probe that miscounted its operations or its clock, or whose chains the
assembler had folded, would land outside these bounds.
"""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rates():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_10459_gb300 as m
    from paper_1807_10459_gb300 import build
    build.build()
    return m.probe_issue_rates(0)


def test_sm_count_and_clock(rates):
    assert rates["n_sms"] == torch.cuda.get_device_properties(0).multi_processor_count
    assert 300.0 < rates["sm_clock_mhz"] < 3500.0


def test_rates_within_the_issue_bound(rates):
    bound = 2 * 128 * 1.03
    assert 0 < rates["fadd_per_sm_clk"] <= bound
    assert 0 < rates["fmnmx_per_sm_clk"] <= bound
    assert 0 < rates["iadd_per_sm_clk"] <= bound
    assert 0 < rates["fsetp_add_per_sm_clk"] <= 3 / 2 * bound
    assert 0 < rates["count_mix_per_sm_clk"] <= 6 / 5 * bound


def test_per_second_rates_imply_a_plausible_clock(rates):
    """Per second over per SM and clock is the clock each probe ran at (the
    clock may ramp between probes, so each is checked on its own)."""
    for name in ("fadd", "fmnmx", "fsetp_add", "iadd", "count_mix"):
        mhz = rates[f"{name}_per_s"] / (rates[f"{name}_per_sm_clk"] * rates["n_sms"]) / 1e6
        assert 300.0 < mhz < 3500.0, (name, mhz)
