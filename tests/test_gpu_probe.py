"""The issue-rate probe behind the render's roofline denominator: the FP32
FMA rate must land near the unit-count peak (152 SMs x 128 lanes x clock)
and the ex2 rate well below it (a quarter-rate unit or slower)."""
import pytest

pytestmark = pytest.mark.gpu


def test_peak_probe_rates():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_00435_gb300 import gs
    import bench
    fma, ex2 = bench.peak_probe(torch, gs, iters=4000, reps=3)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = sms * 128 * 2.07e9 / 1e12          # T lane-ops/s at the maximum clock
    assert 0.5 * nominal < fma < 1.05 * nominal, (fma, nominal)
    assert 0.0 < ex2 < 0.5 * fma, (ex2, fma)
    with pytest.raises(gs.GsError):
        gs.gs_peak_probe(2, 10, torch.zeros(1, device="cuda"))
