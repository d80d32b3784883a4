"""AoS and clustered-SoA layouts of the fused FP64 step (the paper's layout comparison,
Sec. 4) give the SoA step's results: the same arithmetic on the same gathered values, with
different addresses.  The compiler may contract multiply-adds differently in each kernel,
so the bar is 1e-13 relative after 3 steps (the single-collide bar), not bit equality;
the layout conversions themselves are exact."""
import pytest
import torch

from paper_1703_04594_gb300 import lbm
from tests.gpu_util import device_init, require_gpu, rt_fields

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


@pytest.mark.parametrize("layout", [lbm.LAYOUT_AOS, lbm.LAYOUT_CSOA])
@pytest.mark.parametrize("lx,ly", [(64, 128), (37, 45), (8, 200)])
def test_layout_step_equals_soa(layout, lx, ly):
    p = lbm.Params(lx, ly, gx=1e-4)
    f = device_init(p, rt_fields(p, seed=21))
    want = lbm.run(p, f.clone(), lbm.empty_state(p), 3)
    a = lbm.convert_layout(p, f, lbm.LAYOUT_SOA, torch.zeros_like(f), layout)
    b = torch.zeros_like(f)
    for _ in range(3):
        lbm.step_layout(p, layout, a, b)
        a, b = b, a
    back = lbm.convert_layout(p, a, layout, torch.zeros_like(f), lbm.LAYOUT_SOA)
    g, w = back[:, :, :ly], want[:, :, :ly]
    assert float(((g - w).abs() / w.abs()).max()) <= 1e-13


@pytest.mark.parametrize("layout", [lbm.LAYOUT_AOS, lbm.LAYOUT_CSOA])
def test_layout_round_trip(layout):
    p = lbm.Params(37, 45)
    f = device_init(p, rt_fields(p, seed=22))
    a = lbm.convert_layout(p, f, lbm.LAYOUT_SOA, torch.zeros_like(f), layout)
    back = lbm.convert_layout(p, a, layout, torch.zeros_like(f), lbm.LAYOUT_SOA)
    assert torch.equal(back[:, :, :45], f[:, :, :45])
