"""The peak-rate probes return rates in the range a GB300 can reach (nominal: FP32 FMA about 80
TFLOP/s, TF32 dense about 1.1 PFLOP/s, FP64 far below FP32), and the MMA probe's bounded wait
completes."""
import pytest
import torch

from paper_1904_02603_gb300 import vest as V

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_02603_gb300 import build as B
    B.build()
    V.load()


def test_probe_rates_are_plausible():
    buf = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
    fp32 = V.vest_probe_peak(V.PROBE_FP32_FMA)
    fp64 = V.vest_probe_peak(V.PROBE_FP64_FMA)
    tf32 = V.vest_probe_peak(V.PROBE_TF32_MMA)
    l2 = V.vest_probe_peak(V.PROBE_L2_GATHER, buf)
    print(f"\nFP32 FMA {fp32:.1f} TFLOP/s, FP64 FMA {fp64:.2f} TFLOP/s, TF32 MMA {tf32:.0f} TFLOP/s, L2 gather {l2:.2f} TB/s")
    assert 20 < fp32 < 200
    assert 0.1 < fp64 < fp32
    assert 100 < tf32 < 5000
    assert 0.5 < l2 < 200
    assert V.vest_device_status() == 0


def test_probe_rejects_unknown_kind_and_small_buffer():
    with pytest.raises(V.VestError):
        V.vest_probe_peak(9)
    with pytest.raises(V.VestError):
        V.vest_probe_peak(V.PROBE_L2_GATHER, torch.empty(1024, dtype=torch.uint8, device="cuda"))
