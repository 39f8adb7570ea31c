"""The FP32 FMA throughput microbenchmark (fpo_fma_peak): its flop count is
the launch's work and its rate lies below the FP32 lanes' nominal rate at the
GPU's maximum SM clock (128 FP32 lanes per SM, 2 flop per FMA)."""

import ctypes as C

import pytest

from paper_2202_08614_gb300 import fpo

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def test_fma_peak_counts_its_work_and_stays_below_the_lanes_rate():
    sink = torch.empty(3 * 64, device="cuda")
    flops = C.c_double(0.0)
    fpo.check(fpo.lib().fpo_fma_peak(3, 64, 10, C.c_void_p(sink.data_ptr()), C.byref(flops), None))
    torch.cuda.synchronize()
    assert flops.value == 2 * 16 * 10 * 3 * 64
    assert torch.isfinite(sink).all()
    with pytest.raises(fpo.FPOError):
        fpo.check(fpo.lib().fpo_fma_peak(1, 48, 10, C.c_void_p(sink.data_ptr()), None, None))
    props = torch.cuda.get_device_properties(0)
    nominal = props.multi_processor_count * 128 * 2 * 2.07e9 / 1e12  # TFLOP/s at the 2070 MHz maximum
    tf = fpo.fma_peak_tflops()
    print(f"FP32 FMA: {tf:.1f} TFLOP/s (lanes at 2070 MHz: {nominal:.1f})")
    assert 0.3 * nominal < tf <= 1.02 * nominal
