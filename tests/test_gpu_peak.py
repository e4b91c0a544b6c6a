"""The measured FMA rates that the benchmark's rooflines divide by
(qr_fma_peak): plausible for a B300, consistent between the FP32 forms, and
the SM count read from the device."""
import pytest

pytestmark = pytest.mark.gpu


def test_fma_peaks_are_plausible():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_21084_b300 import _lib as L
    from paper_2407_21084_b300 import build

    build.build()
    st = torch.cuda.Stream()
    f32 = L.fma_peak(L.QR_PEAK_FP32, 40.0, st.cuda_stream)
    f2 = L.fma_peak(L.QR_PEAK_FP32X2, 40.0, st.cuda_stream)
    mix = L.fma_peak(L.QR_PEAK_FP32MIX, 40.0, st.cuda_stream)
    f64 = L.fma_peak(L.QR_PEAK_FP64, 40.0, st.cuda_stream)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert f32["sm_count"] == sms
    # 128 FP32 lanes per SM at 1-2.1 GHz: the measured rate cannot exceed it
    assert 0.2 * sms * 256 * 1.0e9 / 1e12 < f32["tflops"] < sms * 256 * 2.1e9 / 1e12
    assert 0.5 < f2["tflops"] / f32["tflops"] < 1.1
    assert 0.3 < mix["tflops"] / f32["tflops"] < 1.1
    assert 0.0 < f64["tflops"] < f32["tflops"]
    with pytest.raises(Exception):
        L.fma_peak(7, 40.0, st.cuda_stream)
