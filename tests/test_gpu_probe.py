"""mgsa_fp64_probe, the measured FP64 FMA rate bench.py reports beside the
derived peak: a positive rate of the right magnitude for the GPU's SM count
and clock, and argument errors refused on the host."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1703_10440_gb300 import mgsa  # noqa: E402


def test_probe_rate_is_near_the_derived_peak():
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    tf, ms = mgsa.mgsa_fp64_probe(0, 20000)
    assert ms > 0
    # 2 FP64 FMAs per clock per SM at any clock between 1 and 2.2 GHz
    assert sms * 2 * 2 * 1.0e9 * 0.5 / 1e12 < tf < sms * 2 * 2 * 2.2e9 * 1.05 / 1e12, (tf, sms)


def test_probe_argument_errors():
    import ctypes

    lib = mgsa.lib()
    tf, ms = ctypes.c_double(0), ctypes.c_double(0)
    assert lib.mgsa_fp64_probe(0, 0, ctypes.byref(tf), ctypes.byref(ms)) == mgsa.MGSA_ERR_INVALID
    assert lib.mgsa_fp64_probe(0, 10, None, ctypes.byref(ms)) == mgsa.MGSA_ERR_INVALID
    assert lib.mgsa_fp64_probe(10**6, 10, ctypes.byref(tf), ctypes.byref(ms)) == mgsa.MGSA_ERR_INVALID
