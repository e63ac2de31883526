"""The FMA-throughput diagnostic (hydro_fma_rate), the FP32 roofline's measured denominator."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_fma_rates_are_physical():
    from paper_1204_4779_gb300 import hydro
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    f32 = hydro.fma_rate(torch.float32)
    f64 = hydro.fma_rate(torch.float64)
    # 128 FP32 lanes per SM per clock; SM clocks between 0.5 and 2.2 GHz
    assert 0.5 * 128 * sms * 0.5e9 < f32 < 1.02 * 128 * sms * 2.2e9, f32
    assert 0 < f64 < f32, (f64, f32)
    print(f"FMA rates: FP32 {f32 / 1e12:.2f} T/s, FP64 {f64 / 1e12:.3f} T/s ({sms} SMs)")


def test_fma_rate_rejects_bad_arguments():
    import ctypes
    from paper_1204_4779_gb300 import hydro
    lib = hydro.load_library()
    out = ctypes.c_double()
    assert lib.hydro_fma_rate(7, None, ctypes.byref(out)) == hydro.HYDRO_EINVAL
    assert lib.hydro_fma_rate(hydro.HYDRO_F32, None, None) == hydro.HYDRO_EINVAL
