"""Dense states on every float64 entry point, against the oracle.

The float64 paths sum the moments (eq. "macro") in signed 64-bit fixed point with 2^-52
resolution, which holds magnitudes below 2^11.  A state whose populations reach 8 or more
in magnitude (densities above ~30) would wrap those sums, so such sites sum in plain
float64.  These tests run states of mean density 1600 and 5000 (where the sums of
sum_i |v_i|^2 f_i reach 2233 and 6980, beyond 2^11), and a density ramp that crosses the
bound inside one warp, through every float64 entry point, and hold them to the same bars as
the ordinary states: populations within 1e-12 relative of the oracle after 3 steps.

The FP32 forms store g_i = f_i - w_i rho0 and state their own range, |g_i| < 8 * 2^k with
2^k <= rho0 < 2^(k+1): with rho0 at the state's density they meet their per-field bar;
with rho0 = 1 every site of a density-1600 state is outside the range and comes out NaN.
"""
import pytest
import torch

from oracle import lbm as OL
from paper_1703_04594_gb300 import lbm
from tests.gpu_util import device_init, field_errors, oracle_params, rel_err, require_gpu, rt_fields, to_host

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-12
STEPS = 3
LX, LY = 20, 40          # two warps per column, the second one ragged


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def dense_fields(p, kind):
    """(rho, ux, uy, T) of a dense state.  'rt1600' / 'rt5000': the Rayleigh-Taylor state with
    its density scaled to a mean of 1600 / 5000; 'rest1600': uniform rest state at rho = 1600,
    T = 1; 'ramp': a Rayleigh-Taylor state whose density runs from 30 to 40 along y, so the rest
    population 0.233 rho crosses 8 (at rho ~ 34.3) inside the first warp of every column."""
    rho, ux, uy, T = rt_fields(p, seed=31)
    if kind == "rt1600":
        return rho * 1600.0, ux, uy, T
    if kind == "rt5000":
        return rho * 5000.0, ux, uy, T
    if kind == "rest1600":
        return torch.full_like(rho, 1600.0), ux, uy, torch.ones_like(T)
    if kind == "ramp":
        y = torch.arange(p.ly, dtype=torch.float64)
        return rho * (30.0 + 10.0 * y / (p.ly - 1))[None, :], ux + 0.01, uy - 0.005, T
    raise ValueError(kind)


KINDS = ["rt1600", "rt5000", "rest1600", "ramp"]
BCS = [lbm.BC_WALLS, lbm.BC_PERIODIC_Y]


def params(bc, precision=lbm.FP64, **kw):
    return lbm.Params(LX, LY, tau=kw.pop("tau", 0.8), gx=kw.pop("gx", 1e-4), precision=precision, bc=bc, **kw)


def oracle_run(p, fields, steps=STEPS):
    return OL.run(OL.init_equilibrium(*fields), oracle_params(p), steps)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP64_FIXED])
def test_run_matches_oracle(kind, bc, precision):
    p = params(bc, precision)
    fields = dense_fields(p, kind)
    f = device_init(p, fields)
    res = lbm.run(p, f, lbm.empty_state(p), STEPS)
    assert rel_err(to_host(p, res), oracle_run(p, fields)) <= STEP_TOL


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("bc", BCS)
def test_separate_kernels_match_oracle(kind, bc):
    p = params(bc)
    fields = dense_fields(p, kind)
    f = device_init(p, fields)
    tmp, out = lbm.empty_state(p), lbm.empty_state(p)
    for _ in range(STEPS):
        lbm.propagate(p, f, tmp)
        lbm.bc(p, f, tmp)
        lbm.collide(p, tmp, out)
        f, out = out, f
    assert rel_err(to_host(p, f), oracle_run(p, fields)) <= STEP_TOL


@pytest.mark.parametrize("kind", ["rt5000", "ramp"])
@pytest.mark.parametrize("layout", [lbm.LAYOUT_AOS, lbm.LAYOUT_PSOA, lbm.LAYOUT_CAOSOA])
def test_layout_steps_match_oracle(kind, layout):
    p = params(lbm.BC_WALLS)
    fields = dense_fields(p, kind)
    f = device_init(p, fields)
    a = lbm.convert_layout(p, f, lbm.LAYOUT_SOA, torch.zeros_like(f), layout)
    b = torch.zeros_like(f)
    for _ in range(STEPS):
        lbm.step_layout(p, layout, a, b)
        a, b = b, a
    back = lbm.convert_layout(p, a, layout, torch.zeros_like(f), lbm.LAYOUT_SOA)
    assert rel_err(to_host(p, back), oracle_run(p, fields)) <= STEP_TOL


@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP64_FIXED])
@pytest.mark.parametrize("mode", [lbm.BATCH_PER_STEP, lbm.BATCH_PERSISTENT])
def test_batch_matches_oracle(precision, mode):
    ps, fa, fb, want = [], [], [], []
    for kind in KINDS:
        p = params(lbm.BC_WALLS, precision)
        fields = dense_fields(p, kind)
        ps.append(p)
        fa.append(device_init(p, fields))
        fb.append(lbm.empty_state(p))
        want.append(oracle_run(p, fields))
    b = lbm.Batch(ps, fa, fb)
    b.configure(mode, 4)
    b.run(STEPS)
    torch.cuda.synchronize()
    assert b.status() == lbm.OK
    for p, got, w in zip(ps, b.states(), want):
        assert rel_err(to_host(p, got), w) <= STEP_TOL
    b.close()


@pytest.mark.parametrize("kind", KINDS)
def test_moments_and_kinetic_energy_match_oracle(kind):
    p = params(lbm.BC_WALLS)
    fields = dense_fields(p, kind)
    f = device_init(p, fields)
    res = lbm.run(p, f, lbm.empty_state(p), STEPS)
    got = [t.cpu() for t in lbm.moments(p, res)]
    fo = oracle_run(p, fields)
    want = OL.fields(fo)
    for k in (0, 3):                                   # rho, T
        assert rel_err(got[k], want[k]) <= STEP_TOL
    umax = float(torch.sqrt(want[1] ** 2 + want[2] ** 2).max())
    for k in (1, 2):
        assert float((got[k] - want[k]).abs().max()) <= STEP_TOL * umax + 1e-15
    ke, ke_o = float(lbm.kinetic_energy(p, res)), float(OL.kinetic_energy(fo))
    assert abs(ke - ke_o) <= 1e-10 * ke_o


@pytest.mark.parametrize("kind", ["rt1600", "ramp"])
@pytest.mark.parametrize("bc", BCS)
def test_adjoint_step_matches_oracle_vjp(kind, bc):
    """lam_n = (d step / d f)^T lam_next and d(lam_next . step)/d tau against torch autograd
    through the oracle's step."""
    p = params(bc, tau=0.7)
    fields = dense_fields(p, kind)
    f = device_init(p, fields)
    f = lbm.run(p, f, lbm.empty_state(p), 2).clone()
    g = torch.Generator().manual_seed(5)
    lam = torch.randn(37, p.lx, p.ly, dtype=torch.float64, generator=g)
    lam_dev = lbm.empty_state(p)
    lam_dev.zero_()
    lam_dev[:, :, : p.ly] = lam.cuda()
    lam_n = lbm.empty_state(p)
    dtau = torch.zeros((), dtype=torch.float64, device="cuda")
    lbm.adjoint_step(p, f, lam_dev, lam_n, dtau, lbm.adjoint_work(p))
    fo = to_host(p, f).requires_grad_(True)
    tau_t = torch.tensor(p.tau, dtype=torch.float64, requires_grad=True)
    op = oracle_params(p)
    op = OL.Params(op.lx, op.ly, tau=tau_t, gx=op.gx, gy=op.gy, t_bottom=op.t_bottom, t_top=op.t_top, bc=op.bc)
    (OL.step(fo, op) * lam).sum().backward()
    want = fo.grad
    got = to_host(p, lam_n)
    assert float((got - want).abs().max()) <= STEP_TOL * float(want.abs().max())
    assert abs(float(dtau) - float(tau_t.grad)) <= 1e-10 * abs(float(tau_t.grad))


def fp32(p, rho0, precision=lbm.FP32_SHIFTED):
    return lbm.Params(p.lx, p.ly, tau=p.tau, gx=p.gx, gy=p.gy, t_bottom=p.t_bottom, t_top=p.t_top,
                      rho0=rho0, precision=precision, bc=p.bc)


@pytest.mark.parametrize("precision", [lbm.FP32_SHIFTED, lbm.FP32_CONSERVED])
@pytest.mark.parametrize("kind,rho0", [("rt1600", 1600.0), ("rest1600", 1600.0), ("rt5000", 5000.0)])
def test_fp32_with_matching_reference_density(kind, rho0, precision):
    p = fp32(params(lbm.BC_WALLS), rho0, precision)
    fields = dense_fields(p, kind)
    f = device_init(p, fields)
    res = lbm.run(p, f, lbm.empty_state(p), STEPS)
    got = [t.cpu() for t in lbm.moments(p, res)]
    want = OL.fields(oracle_run(p, fields))
    err = field_errors(got, want)
    assert max(err[k] for k in ("rho_max", "rho_rms", "T_max", "T_rms", "u_max_cs")) <= 1e-5, err


def test_fp32_outside_its_range_gives_nan():
    """rho0 = 1 with a density-1600 state: every site stores a rest deviation of ~373, far
    outside |g| < 8, so its moments and every population it produces are NaN."""
    p = fp32(params(lbm.BC_WALLS), 1.0)
    f = device_init(p, dense_fields(p, "rt1600"))
    rho = lbm.moments(p, f)[0]
    assert bool(torch.isnan(rho).all())
    res = lbm.run(p, f, lbm.empty_state(p), 1)
    assert bool(torch.isnan(res[:, :, : p.ly]).all())
