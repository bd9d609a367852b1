"""The integer-pipe microbenchmark returns plausible rates: a 32-bit multiply
rate near 16 lanes per clock per sub-partition (the FMA-heavy pipe's width),
widening products slower than single ones, and an SM clock within the
GPU's range."""
import pytest

from paper_2309_04909_gb300 import measure_int_peaks
from tests._util import cuda_ok

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]


def test_int_peaks_plausible():
    p = measure_int_peaks(0)
    assert p["sm_count"] > 0 and 100.0 < p["sm_mhz"] < 5000.0
    per_clock = lambda r: r / (p["sm_count"] * 4 * p["sm_mhz"] * 1e6)
    assert 8.0 < per_clock(p["imad_per_s"]) < 33.0
    assert 0.0 < p["imad_wide_per_s"] < p["imad_per_s"]
    assert 0.0 < p["imad_hi_per_s"] <= 1.05 * p["imad_per_s"]
    assert p["alu_per_s"] > 0.0
