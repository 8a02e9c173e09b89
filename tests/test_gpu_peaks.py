"""dock_measure_peaks, the roofline denominators of the scoring kernels: the
measured FP32 FMA and MUFU rates must be positive and not above what the
SMs' lanes can issue at a clock above the device's highest."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_measured_peaks_are_plausible():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2509_12232_gb300 import build
    build.build()
    from paper_2509_12232_gb300 import dock
    f, m = dock.dock_measure_peaks(torch.cuda.current_stream())
    props = torch.cuda.get_device_properties(0)
    clock_ghz = 2.2  # above GB300's 2,070 MHz maximum: an upper bound
    f_max = props.multi_processor_count * 128 * 2 * clock_ghz / 1e3
    # the special-function unit: 16 ex2 per SM and clock on earlier Blackwell parts; GB300
    # doubles it (measured about 9.96 Tops/s): bound by 32
    m_max = props.multi_processor_count * 32 * clock_ghz / 1e3
    assert 0.5 * f_max / 1.1 < f <= f_max, (f, f_max)
    assert 0.15 * m_max / 1.1 < m <= m_max, (m, m_max)
