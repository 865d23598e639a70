"""The unit-rate microbenchmark behind the ALU roofline's peak: measured
results per SM per clock of the SFU's ex2 and the FP32 FMA pipe."""
import pytest

pytestmark = pytest.mark.gpu


def test_unit_rates_are_measured_and_plausible(cuda_device):
    import paper_2012_13257_b300 as g
    r = g.measure_unit_rates()
    # an SM has 4 sub-partitions of 32 FP32 lanes (128 FMA results per clock);
    # B300's SFU returns 32 exponentials per SM per clock (twice the 16 of
    # earlier parts).  Packed FFMA2 halves the issue slots but not the FMA
    # pipe's time, so it reaches the same FMA rate.
    assert 28.0 <= r["ex2"] <= 33.0, r
    assert 110.0 <= r["ffma"] <= 129.0, r
    assert 110.0 <= r["ffma2"] <= 129.0, r
