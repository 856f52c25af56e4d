"""The CUDA-core FMA peak measurement (ads_measure_fma_peak) runs through the
C ABI and returns plausible figures: positive, and below what the device's
SM count and clock allow for its FMA lanes (128 FP32 FMA lanes per SM, two
FMAs per lane for the packed FFMA2 form; FP64 at most the FP32 rate)."""
import pytest

pytestmark = pytest.mark.gpu


def test_fma_peaks_plausible():
    import torch
    import paper_1911_08158_gb300 as ads
    props = torch.cuda.get_device_properties(0)
    ghz = 2.2   # above the part's maximum SM clock
    bound32 = props.multi_processor_count * 128 * 2 * ghz / 1e3   # TFLOP/s
    got = {k: ads.ads.measure_fma_peak(k, 0, 1 << 14)[0] for k in ("ffma", "ffma2", "dfma")}
    assert 0 < got["ffma"] <= 1.05 * bound32, got
    assert 0 < got["ffma2"] <= 2.1 * bound32, got
    assert 0 < got["dfma"] <= 1.05 * bound32, got
    with pytest.raises(ads.AdsError):
        ads.ads.measure_fma_peak("ffma", 0, 0)
