"""fram_measure_alu, the probe whose lane rates are the roofline denominators of the synthesis and
the adjoint: every kind runs, its time grows with the iteration count, and the measured lane
operations per SM per clock are plausible for a Blackwell SM (the FP32 pipe has 128 lanes per SM;
the MUFU pipe a small fraction of that)."""
import pytest

from paper_2304_08052_gb300 import api

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,lo,hi", [(0, 64.0, 130.0), (1, 64.0, 130.0), (2, 4.0, 66.0)])
def test_probe_rates_are_plausible(kind, lo, hi):
    short = api.measure_alu(kind, 100)
    long = api.measure_alu(kind, 800)
    assert long["ms"] > 4.0 * short["ms"]            # the loop runs: time follows the iterations
    assert lo <= long["per_sm_per_clock"] <= hi, long
    assert 500.0 <= long["clock_mhz"] <= 2200.0, long
