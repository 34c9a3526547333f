"""The arithmetic-throughput microbenchmark used as the measured roofline
denominator returns plausible rates (positive, below twice the nominal
unit-count peak at the nominal clock)."""
import pytest

from paper_2410_08267_gb300 import nuprof as nu

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_plausible():
    require_gpu()
    p = nu.nu_measure_peaks()
    nominal = 2 * 128 * p["sm_count"] * p["clock_mhz_nominal"] * 1e6 / 1e12
    for k in ("ffma_tflops", "ffma2_tflops"):
        assert 0.2 * nominal < p[k] < 2.5 * nominal, (k, p[k], nominal)
    assert p["rsqrt_gops"] > 0 and p["lg2_gops"] > 0
    assert 0 < p["dfma_tflops"] < p["ffma_tflops"]
