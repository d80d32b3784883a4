"""AoS, partitioned-SoA and CAoSoA layouts of the fused FP64 step (the paper's layout
comparison, Sec. 4; thermal walls only).  Each layout's step is checked against the oracle
(populations within 1e-12 relative after 3 steps, the float64 parity bar).  It
also gives the SoA step's results: the same arithmetic on the same gathered values, with
different addresses.  The compiler may contract multiply-adds differently in each kernel,
so that bar is 1e-13 relative after 3 steps (the single-collide bar), not bit equality;
the layout conversions themselves are exact."""
import pytest
import torch

from oracle import lbm as OL
from paper_1703_04594_gb300 import lbm
from tests.gpu_util import device_init, oracle_params, rel_err, require_gpu, rt_fields, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


@pytest.mark.parametrize("layout", [lbm.LAYOUT_AOS, lbm.LAYOUT_PSOA, lbm.LAYOUT_CAOSOA])
@pytest.mark.parametrize("lx,ly", [(64, 128), (37, 45), (8, 200), (6, 33), (4, 64)])
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


def layout_run(p, f, layout, steps):
    a = lbm.convert_layout(p, f, lbm.LAYOUT_SOA, torch.zeros_like(f), layout)
    b = torch.zeros_like(f)
    for _ in range(steps):
        lbm.step_layout(p, layout, a, b)
        a, b = b, a
    return lbm.convert_layout(p, a, layout, torch.zeros_like(f), lbm.LAYOUT_SOA)


@pytest.mark.parametrize("layout", [lbm.LAYOUT_AOS, lbm.LAYOUT_PSOA, lbm.LAYOUT_CAOSOA])
@pytest.mark.parametrize("lx,ly", [(37, 45), (64, 128), (6, 33)])
def test_layout_step_matches_oracle(layout, lx, ly):
    p = lbm.Params(lx, ly, tau=0.7, gx=1e-4)
    fields = rt_fields(p, seed=23)
    fields = (fields[0], fields[1] + 0.01, fields[2] - 0.005, fields[3])   # moving fluid
    got = layout_run(p, device_init(p, fields), layout, 3)
    want = OL.run(OL.init_equilibrium(*fields), oracle_params(p), 3)
    assert rel_err(to_host(p, got), want) <= 1e-12


@pytest.mark.parametrize("layout", [lbm.LAYOUT_AOS, lbm.LAYOUT_PSOA, lbm.LAYOUT_CAOSOA])
def test_layout_round_trip(layout):
    p = lbm.Params(37, 45)
    f = device_init(p, rt_fields(p, seed=22))
    a = lbm.convert_layout(p, f, lbm.LAYOUT_SOA, torch.zeros_like(f), layout)
    back = lbm.convert_layout(p, a, layout, torch.zeros_like(f), lbm.LAYOUT_SOA)
    assert torch.equal(back[:, :, :45], f[:, :, :45])


def test_caosoa_addresses():
    """CAoSoA puts the 37 clusters of one (x, j) next to each other: element (i, x, y) at
    ((x * P + j) * 37 + i) * 32 + k with y = k * P + j (checked on a 4 x 64 lattice, P = 2)."""
    p = lbm.Params(4, 64)
    P = lbm.pitch(p) // 32
    f = lbm.empty_state(p)
    i, x, y = torch.meshgrid(torch.arange(37), torch.arange(4), torch.arange(lbm.pitch(p)), indexing="ij")
    f.copy_((i * 1_000_000 + x * 1000 + y).to(torch.float64))
    a = lbm.convert_layout(p, f, lbm.LAYOUT_SOA, torch.zeros_like(f), lbm.LAYOUT_CAOSOA).flatten().cpu()
    for (ii, xx, yy) in [(0, 0, 0), (5, 1, 33), (36, 3, 63), (17, 0, 1), (20, 2, 32)]:
        k, j = yy // P, yy % P
        assert float(a[((xx * P + j) * 37 + ii) * 32 + k]) == ii * 1_000_000 + xx * 1000 + yy
