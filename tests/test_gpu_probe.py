"""The measured FMA peaks of crk_fma_peak: positive, the FP32 rate near the
FP32 pipe's count (SMs x 128 lanes x 2 flop x clock), and FP64 far below it
on this part."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def crk():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2510_03557_gb300 import crk as c

    return c


def test_fma_peaks_are_measured(crk):
    import torch

    props = torch.cuda.get_device_properties(0)
    f32 = crk.crk_fma_peak(crk.CRK_MIXED)
    f64 = crk.crk_fma_peak(crk.CRK_FP64)
    bound = props.multi_processor_count * 128 * 2 * 2.2e9 / 1e12   # above any boost clock of the part
    assert 0.3 * bound < f32 < bound
    assert 0 < f64 < f32
    with pytest.raises(crk.CrkError) as e:
        crk.crk_fma_peak(7)
    assert e.value.code == crk.CRK_EINVAL
