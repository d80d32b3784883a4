"""FP64 storage with the fixed-point relaxation (LBM_FP64_FIXED) against the CPU oracle.

The equilibrium polynomial and the BGK relaxation of every population run in 64-bit fixed
point, scaled per shell so that each output carries a few units of 2^-58 relative to its
size, below float64's 2^-53 rounding unit.  So the bars are those of the float64 path:
populations within 1e-12 relative after 10 steps, and never less accurate than the float64
relaxation on the same input.  Sites outside the
fixed-point range (fast or hot fluid) take the float64 relaxation; the tests cover both
sides of the range and its edge.
"""
import pytest
import torch

from oracle import lbm as OL
from paper_1703_04594_gb300 import lbm
from tests.gpu_util import device_init, oracle_params, rel_err, require_gpu, rt_fields, to_host

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-12


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def run_fixed(p, fields, steps):
    fa = device_init(p, fields)
    fb = lbm.empty_state(p)
    return lbm.run(p, fa, fb, steps)


def oracle_run(p, fields, steps):
    return OL.run(OL.init_equilibrium(*fields), oracle_params(p), steps)


def test_ten_steps_rayleigh_taylor_64x128():
    p = lbm.Params(64, 128, precision=lbm.FP64_FIXED)
    fields = rt_fields(p, seed=1)
    assert rel_err(to_host(p, run_fixed(p, fields, 10)), oracle_run(p, fields, 10)) <= STEP_TOL


@pytest.mark.parametrize("lx,ly,bc,gx", [(37, 45, lbm.BC_WALLS, 3e-4), (4, 6, lbm.BC_WALLS, 0.0),
                                         (33, 70, lbm.BC_PERIODIC_Y, 1e-4), (64, 200, lbm.BC_WALLS, 0.0)])
def test_one_step_ragged(lx, ly, bc, gx):
    """One step of a moving fluid: the fixed-point relaxation is as accurate as the float64 one.
    The error against the oracle is set by the float64 stages the two share (moment sums,
    1/rho, the Hermite coefficients) and by cancellation in (1 - omega) f + omega f^eq where
    the state is far from equilibrium (the periodic-y seam of the RT state reaches 1.3e-12
    in both); the fixed-point products add nothing visible on top."""
    errs = {}
    for prec in (lbm.FP64_FIXED, lbm.FP64):
        p = lbm.Params(lx, ly, tau=0.7, gx=gx, gy=-2e-4, bc=bc, precision=prec)
        fields = rt_fields(p, seed=11)
        fields = (fields[0], fields[1] + 0.02, fields[2] - 0.03, fields[3])
        errs[prec] = rel_err(to_host(p, run_fixed(p, fields, 1)), oracle_run(p, fields, 1))
    print(f"one step {lx}x{ly}: fixed {errs[lbm.FP64_FIXED]:.3g}, float64 {errs[lbm.FP64]:.3g}")
    assert errs[lbm.FP64_FIXED] <= 1.05 * errs[lbm.FP64] + 1e-15
    assert errs[lbm.FP64_FIXED] <= STEP_TOL * 2


def moving_fields(p, ux, uy, temp):
    rho = torch.full((p.lx, p.ly), 1.0, dtype=torch.float64)
    x = torch.arange(p.lx, dtype=torch.float64)[:, None]
    y = torch.arange(p.ly, dtype=torch.float64)[None, :]
    wave = torch.sin(6.283185307179586 * (x / p.lx + 2 * y / p.ly))
    return (rho * (1 + 0.05 * wave), (ux * (1 + 0.1 * wave)).expand(p.lx, p.ly).contiguous(),
            (uy * (1 - 0.1 * wave)).expand(p.lx, p.ly).contiguous(),
            (temp * (1 + 0.02 * wave)).contiguous())


@pytest.mark.parametrize("ux,uy,temp", [
    (0.11, -0.10, 1.2),    # inside the range, near its edge: |c u_x| up to 0.145, T_s - 1 up to 0.22
    (0.30, 0.05, 1.0),     # too fast: every site takes the float64 relaxation
    (0.02, 0.01, 1.45),    # too hot: float64 relaxation
    (0.125, 0.0, 1.0),     # |c u_x| from 0.135 to 0.165 straddles the edge 0.15: mixed warps
])
def test_range_edges_and_fallback(ux, uy, temp):
    p = lbm.Params(48, 64, tau=0.9, gy=-1e-4, bc=lbm.BC_PERIODIC_Y, precision=lbm.FP64_FIXED)
    fields = moving_fields(p, ux, uy, torch.full((p.lx, p.ly), temp, dtype=torch.float64))
    assert rel_err(to_host(p, run_fixed(p, fields, 5)), oracle_run(p, fields, 5)) <= STEP_TOL


def test_tiny_and_zero_populations_take_the_float64_relaxation():
    """A population outside [2^-7, 8) times its shell scale 2^-e_s (here 0 and 1e-12 in two
    shells) puts its site outside the fixed-point range: that site takes the float64
    relaxation, so its outputs agree with the float64 step's to rounding (the same
    arithmetic), and every output stays within the parity bar of the oracle."""
    fx = lbm.Params(40, 64, tau=0.8, gy=-1e-4, precision=lbm.FP64_FIXED)
    fd = lbm.Params(40, 64, tau=0.8, gy=-1e-4)
    _, _, vx, vy = lbm.model()
    f = device_init(fx, rt_fields(fx, seed=21))
    hit = torch.zeros(fx.lx, fx.ly, dtype=torch.bool)
    for i, val, xs, ys in ((36, 0.0, slice(0, None, 3), slice(5, 60, 7)),
                           (30, 1e-12, slice(1, None, 3), slice(4, 60, 5))):
        f[i, xs, ys] = val
        src = torch.zeros(fx.lx, fx.ly, dtype=torch.bool)
        src[xs, ys] = True
        hit |= torch.roll(src, shifts=(vx[i], vy[i]), dims=(0, 1))    # where it is pulled to
    host = to_host(fx, f)
    a = to_host(fx, lbm.step(fx, f, lbm.empty_state(fx)))
    b = to_host(fd, lbm.step(fd, f, lbm.empty_state(fd)))
    assert int(hit.sum()) > 50
    assert rel_err(a[:, hit], b[:, hit]) <= 1e-15
    assert rel_err(a, OL.step(host, oracle_params(fx))) <= STEP_TOL


def test_fixed_and_float64_relaxations_agree_on_a_long_run():
    """256 x 512 RT lattice, 50 steps: the fixed-point and float64 relaxations differ only by
    rounding (both well below the parity bar)."""
    fx = lbm.Params(256, 512, precision=lbm.FP64_FIXED)
    fd = lbm.Params(256, 512, precision=lbm.FP64)
    fields = rt_fields(fx, seed=12)
    a = run_fixed(fx, fields, 50)
    b = lbm.run(fd, device_init(fd, fields), lbm.empty_state(fd), 50)
    assert rel_err(to_host(fx, a), to_host(fd, b)) <= 1e-13


@pytest.mark.parametrize("tau", [0.8, 1.3])      # 1 - omega negative and positive
def test_no_mass_drift(tau):
    """Periodic box without gravity, 400 steps: collision conserves mass, so the total may
    move only by rounding.  The truncations of the fixed-point products are re-centred, so
    the fixed-point relaxation drifts no more than the float64 one (whose own drift comes
    from the float64 weights and rounding) and stays within 1e-14 of the initial mass (an
    unre-centred truncation of 2^-54 per population and step would show as ~1e-14)."""
    drift = {}
    for prec in (lbm.FP64_FIXED, lbm.FP64):
        p = lbm.Params(64, 64, tau=tau, gy=0.0, bc=lbm.BC_PERIODIC_Y, precision=prec)
        fields = moving_fields(p, 0.05, -0.03, torch.full((p.lx, p.ly), 1.05, dtype=torch.float64))
        f0 = device_init(p, fields)
        m0 = float(f0[:, :, : p.ly].sum())
        f = lbm.run(p, f0.clone(), lbm.empty_state(p), 400)
        drift[prec] = abs(float(f[:, :, : p.ly].sum()) - m0) / m0
    print(f"mass drift after 400 steps: fixed {drift[lbm.FP64_FIXED]:.3g}, float64 {drift[lbm.FP64]:.3g}")
    assert drift[lbm.FP64_FIXED] <= max(drift[lbm.FP64], 1e-14)


def test_state_buffers_interchange_with_fp64():
    """LBM_FP64_FIXED uses the float64 buffers: moments of a fixed-path state read as FP64."""
    p = lbm.Params(32, 64, precision=lbm.FP64_FIXED)
    assert lbm.buffer_bytes(p) == lbm.buffer_bytes(lbm.Params(32, 64))
    fields = rt_fields(p, seed=13)
    f = device_init(p, fields)
    rho, ux, uy, T = lbm.moments(p, f)
    assert rel_err(rho.cpu(), fields[0]) <= 1e-13 and rel_err(T.cpu(), fields[3]) <= 1e-13


def test_full_size_sampled_columns():
    """4096 x 8192 (the throughput lattice, seed 2) in the launch configuration the bench
    times: two fixed-point steps on the GPU; the oracle recomputes sampled columns from
    crops of +-6 columns (two steps reach 6 columns) built from the same seeded fields."""
    p = lbm.Params(4096, 8192, precision=lbm.FP64_FIXED)
    fields = rt_fields(p, seed=2)
    res = run_fixed(p, fields, 2)
    got = res[:, :, : p.ly]
    for x in [0, 2047, 4095]:
        cols = [(x + d) % p.lx for d in range(-6, 7)]
        crop = [t[cols] for t in fields]
        op = OL.Params(13, p.ly, tau=p.tau, gx=p.gx, gy=p.gy, t_bottom=p.t_bottom, t_top=p.t_top)
        want = OL.run(OL.init_equilibrium(*crop), op, 2)[:, 6]
        assert rel_err(got[:, x].double().cpu(), want) <= STEP_TOL, x
    del res, got
    torch.cuda.empty_cache()



@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP64_FIXED])
def test_injected_nan_reaches_exactly_its_destination_site(precision):
    """Fault made on the host: one population of one site is set to NaN.  After one step
    the site it is pulled to, and only that site, holds NaN in every population (its
    moments are NaN, so lbm_moments flags it); every other site is unchanged with respect
    to a clean run.  Both the float64 and the fixed-point forms (whose range check sends
    the site to the float64 collision) behave the same way."""
    p = lbm.Params(24, 48, precision=precision)
    _, _, vx, vy = lbm.model()
    fields = rt_fields(p, seed=23)
    clean = device_init(p, fields)
    bad = clean.clone()
    i, xs, ys = 30, 5, 20
    bad[i, xs, ys] = float("nan")
    a = to_host(p, lbm.step(p, clean, lbm.empty_state(p)))
    b = to_host(p, lbm.step(p, bad, lbm.empty_state(p)))
    xd, yd = (xs + vx[i]) % p.lx, ys + vy[i]
    nan_sites = torch.isnan(b).any(dim=0)
    assert nan_sites.sum() == 1 and bool(nan_sites[xd, yd])
    assert bool(torch.isnan(b[:, xd, yd]).all())
    keep = ~nan_sites
    assert torch.equal(a[:, keep], b[:, keep])
    rho = lbm.moments(p, lbm.step(p, bad, lbm.empty_state(p)))[0].cpu()
    assert torch.isnan(rho).sum() == 1 and bool(torch.isnan(rho[xd, yd]))
