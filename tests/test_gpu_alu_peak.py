"""The FMA microbenchmark behind the sweep kernels' roofline: the measured packed FP32 rate must
sit near the issue limit derived from the device (SMs x 128 FP32 lanes x 2 flops x clock), and the
FP64 rate below it."""
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1712_01132_gb300 import dvm

pytestmark = pytest.mark.gpu


def test_fma_peaks_are_plausible():
    props = torch.cuda.get_device_properties(0)
    derived = props.multi_processor_count * 128 * 2 * 2.07e9 / 1e12      # at the maximum SM clock
    f32 = dvm.alu_peak("fp32")
    f64 = dvm.alu_peak("fp64")
    print("FMA peaks: FP32 %.1f TFLOP/s (derived %.1f), FP64 %.2f TFLOP/s" % (f32, derived, f64))
    assert 0.5 * derived < f32 < 1.1 * derived
    assert 0.0 < f64 < f32
