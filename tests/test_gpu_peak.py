"""dg_peak_fma: the measured FMA throughput used as the FP64 path's roofline
denominator (a diagnostic entry point)."""
import pytest

from paper_1305_5536_gb300 import dg

pytestmark = pytest.mark.gpu


def test_peak_fma_is_measured_and_ordered():
    f64 = dg.peak_fma("fp64")
    f32 = dg.peak_fma("fp32")
    # a GB300 has ~1.2 TFLOP/s FP64 and ~75 TFLOP/s FP32 FMA (non-tensor) nominal
    assert 1e11 < f64 < 1e14, f64
    assert 1e12 < f32 < 1e15, f32
    assert f32 > 8 * f64, (f32, f64)


def test_peak_fma_rejects_bad_precision():
    import ctypes
    L = dg.load()
    out = ctypes.c_double(0.0)
    assert L.dg_peak_fma(7, ctypes.byref(out)) == dg.DG_EINVAL
    assert b"precision" in L.dg_last_error(None)
