"""The measurement probes behind the benchmark's roofline: the integer-pipe
ceilings of the butterfly and the Shoup product, and the rates of the 32-bit
multiply instructions they are made of.  Sanity only: positive rates, and the
order the hardware fixes (a low product occupies the multiply pipe half as
long as a high or widening one)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2503_22227_gb300 import api  # noqa: E402


def test_int_peaks_and_multiply_rates():
    modmul, bfly, bfly_wide = api.measure_int_peak()
    assert modmul > 1e11 and bfly > 1e11 and bfly_wide > 1e11
    assert bfly_wide > bfly            # the wide form skips a conditional subtraction
    lo, hi, wide = api.measure_imad_rates()
    assert lo > 1.5 * hi > 0 and wide > 0
    # a butterfly issues several multiplies: it cannot beat the low-product rate
    assert bfly_wide < lo
