"""Peak probes (lbm_probe_peak): measured sustained rates of the arithmetic pipes that the
step kernels' roofline denominators use."""
import pytest

from paper_1703_04594_gb300 import lbm
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def test_rates_are_plausible_and_ordered():
    r = {k: lbm.probe_peak(k) for k in (lbm.PROBE_DFMA, lbm.PROBE_FFMA, lbm.PROBE_IMAD, lbm.PROBE_MULHI64,
                                        lbm.PROBE_UMULHI64)}
    print({k: f"{v / 1e12:.3f} Tops/s" for k, v in r.items()})
    # float64 FMA: at most 2 per clock per SM on 152 SMs at 2.07 GHz (0.63 Tops/s)
    assert 0.1e12 < r[lbm.PROBE_DFMA] <= 0.66e12
    # float32 FMA runs at tens of times the float64 rate on this part
    assert r[lbm.PROBE_FFMA] > 20 * r[lbm.PROBE_DFMA]
    # a 64-bit high product takes several integer instructions, yet beats a float64 FMA
    assert r[lbm.PROBE_UMULHI64] > r[lbm.PROBE_DFMA]
    assert r[lbm.PROBE_IMAD] > r[lbm.PROBE_UMULHI64]


def test_unknown_kind_is_rejected():
    with pytest.raises(lbm.LbmError):
        lbm.probe_peak(9)
