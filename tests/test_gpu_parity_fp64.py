"""FP64 CUDA path vs the CPU oracle, through the C-ABI.

Bar: propagate bit-exact; populations within 1e-12 relative (max over elements of
|gpu - oracle| / |oracle|) after 10 steps.  Single kernels: init and bc within 1e-14 (a
few ulp of the float64 results); collide within 1e-13, because its moment sums carry up
to 37 * 2^-53 absolute rounding (fixed-point or float64 summation alike), which moves
s = xi . u and so every equilibrium population by up to ~1e-14..1e-13 relative.
"""
import math

import pytest
import torch

from oracle import d2q37 as OM
from oracle import lbm as OL
from paper_1703_04594_gb300 import lbm
from tests.gpu_util import device_init, oracle_params, rel_err, require_gpu, rt_fields, to_host

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-12
KERNEL_TOL = 1e-14
COLLIDE_TOL = 1e-13


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def oracle_state(p, seed):
    return OL.init_equilibrium(*rt_fields(p, seed))


def test_init_matches_oracle():
    p = lbm.Params(64, 128)
    fields = rt_fields(p, seed=1)
    f = device_init(p, fields)
    assert rel_err(to_host(p, f), OL.init_equilibrium(*fields)) <= KERNEL_TOL


@pytest.mark.parametrize("form", ["pull", "push"])
@pytest.mark.parametrize("bc", [lbm.BC_WALLS, lbm.BC_PERIODIC_Y])
@pytest.mark.parametrize("lx,ly", [(37, 45), (5, 7), (130, 70)])
def test_propagate_bit_exact(form, bc, lx, ly):
    """Pull (gather) and push (scatter) forms of propagate, Sec. 4: the same copy."""
    p = lbm.Params(lx, ly, bc=bc)
    f = device_init(p, rt_fields(p, seed=3))
    tmp = lbm.empty_state(p)
    tmp.fill_(float("nan"))
    (lbm.propagate if form == "pull" else lbm.propagate_push)(p, f, tmp)
    got = to_host(p, tmp)
    want = OL.propagate(to_host(p, f), oracle_params(p))
    # entries with a source inside the fluid are pure copies: bit-exact
    valid = torch.zeros_like(want, dtype=torch.bool)
    for i, (vx, vy) in enumerate(OM.VELOCITIES):
        ys = torch.arange(p.ly) - vy
        ok = (ys >= 0) & (ys < p.ly) if bc == lbm.BC_WALLS else torch.ones(p.ly, dtype=torch.bool)
        valid[i] = ok[None, :].expand(p.lx, p.ly)
    assert torch.equal(got[valid], want[valid])
    # entries whose source is outside are left for bc
    assert torch.isnan(got[~valid]).all()


def test_bc_matches_oracle():
    p = lbm.Params(37, 45)
    f = device_init(p, rt_fields(p, seed=4))
    tmp = lbm.empty_state(p)
    lbm.propagate(p, f, tmp)
    lbm.bc(p, f, tmp)
    fh = to_host(p, f)
    want = OL.bc(OL.propagate(fh, oracle_params(p)), fh, oracle_params(p))
    assert rel_err(to_host(p, tmp), want) <= KERNEL_TOL


def test_collide_matches_oracle():
    p = lbm.Params(37, 45, gx=2e-4, gy=-3e-4)
    fields = rt_fields(p, seed=5)
    fields = (fields[0], fields[1] + 0.01, fields[2] - 0.02, fields[3])   # moving fluid
    f = device_init(p, fields)
    out = lbm.empty_state(p)
    lbm.collide(p, f, out)
    assert rel_err(to_host(p, out), OL.collide(to_host(p, f), oracle_params(p))) <= COLLIDE_TOL


def test_separate_kernels_equal_fused_step():
    p = lbm.Params(64, 96)
    f = device_init(p, rt_fields(p, seed=6))
    tmp, a, b = lbm.empty_state(p), lbm.empty_state(p), lbm.empty_state(p)
    lbm.propagate(p, f, tmp)
    lbm.bc(p, f, tmp)
    lbm.collide(p, tmp, a)
    lbm.step(p, f, b)
    assert rel_err(to_host(p, a), to_host(p, b)) <= COLLIDE_TOL


def test_push_propagate_step_equals_fused_step():
    p = lbm.Params(64, 96, gx=1e-4)
    f = device_init(p, rt_fields(p, seed=7))
    tmp, a, b = lbm.empty_state(p), lbm.empty_state(p), lbm.empty_state(p)
    lbm.propagate_push(p, f, tmp)
    lbm.bc(p, f, tmp)
    lbm.collide(p, tmp, a)
    lbm.step(p, f, b)
    assert rel_err(to_host(p, a), to_host(p, b)) <= COLLIDE_TOL


def test_ten_steps_rayleigh_taylor_64x128():
    """The small parity run: 64 x 128, walls at T = 1.15 / 0.85, tau = 0.8,
    g = 1e-4 in -y, RT initial state seed 1, 10 fused steps."""
    p = lbm.Params(64, 128)
    fields = rt_fields(p, seed=1)
    fa = device_init(p, fields)
    fb = lbm.empty_state(p)
    res = lbm.run(p, fa, fb, 10)
    want = OL.run(OL.init_equilibrium(*fields), oracle_params(p), 10)
    assert rel_err(to_host(p, res), want) <= STEP_TOL


@pytest.mark.parametrize("lx,ly,bc,gx", [(37, 45, lbm.BC_WALLS, 3e-4), (4, 6, lbm.BC_WALLS, 0.0),
                                         (5, 7, lbm.BC_PERIODIC_Y, 1e-3), (33, 70, lbm.BC_PERIODIC_Y, 0.0),
                                         (130, 33, lbm.BC_WALLS, -2e-4)])
def test_ragged_and_minimum_lattices(lx, ly, bc, gx):
    p = lbm.Params(lx, ly, tau=0.7, gx=gx, gy=-2e-4, bc=bc)
    fields = rt_fields(p, seed=7)
    fa = device_init(p, fields)
    fb = lbm.empty_state(p)
    res = lbm.run(p, fa, fb, 5)
    want = OL.run(OL.init_equilibrium(*fields), oracle_params(p), 5)
    assert rel_err(to_host(p, res), want) <= STEP_TOL


def test_padding_is_never_read():
    p = lbm.Params(16, 40)            # pitch 64: 24 padding rows per column
    fields = rt_fields(p, seed=8)
    fa = device_init(p, fields)
    fa[:, :, p.ly:] = float("nan")
    fb = lbm.empty_state(p)
    res = lbm.run(p, fa, fb, 3)
    assert torch.isfinite(res[:, :, : p.ly]).all()


def test_moments_and_kinetic_energy_match_oracle():
    p = lbm.Params(64, 128)
    fields = rt_fields(p, seed=9)
    fa = device_init(p, fields)
    fb = lbm.empty_state(p)
    res = lbm.run(p, fa, fb, 4)
    want_f = OL.run(OL.init_equilibrium(*fields), oracle_params(p), 4)
    rho, ux, uy, T = [t.cpu() for t in lbm.moments(p, res)]
    orho, oux, ouy, oT = OL.fields(want_f)
    assert rel_err(rho, orho) <= STEP_TOL and rel_err(T, oT) <= STEP_TOL
    scale = float(torch.sqrt((oux ** 2 + ouy ** 2).mean()))
    assert float((ux - oux).abs().max()) <= STEP_TOL * max(scale, 1e-12) * 10
    assert float((uy - ouy).abs().max()) <= STEP_TOL * max(scale, 1e-12) * 10
    ke = float(lbm.kinetic_energy(p, res))
    oke = float(OL.kinetic_energy(want_f))
    assert abs(ke - oke) <= 1e-10 * oke


def test_kinetic_energy_of_a_drifting_state_matches_oracle():
    """The kinetic energy against the oracle at the population bar, 1e-12: on a state with a
    drift (u ~ 0.02) its relative error is that of the moments, not that of velocities near
    zero (the test above, 4 steps from rest, where 1e-10 is the bound)."""
    p = lbm.Params(64, 128)
    rho, ux, uy, T = rt_fields(p, seed=9)
    fields = (rho, ux + 0.02, uy - 0.01, T)
    res = lbm.run(p, device_init(p, fields), lbm.empty_state(p), 4)
    want_f = OL.run(OL.init_equilibrium(*fields), oracle_params(p), 4)
    ke = float(lbm.kinetic_energy(p, res))
    oke = float(OL.kinetic_energy(want_f))
    assert abs(ke - oke) <= 1e-12 * oke, (ke, oke)


def test_simulate_host_end_to_end():
    p = lbm.Params(32, 64)
    fields = rt_fields(p, seed=10)
    fin = [t.contiguous().pin_memory() for t in fields]
    fout = [torch.empty(p.lx, p.ly, dtype=torch.float64).pin_memory() for _ in range(4)]
    fa, fb = lbm.empty_state(p), lbm.empty_state(p)
    fdev = torch.empty(4 * p.lx * p.ly, dtype=torch.float64, device="cuda")
    lbm.simulate_host(p, fin, 3, fout, fa, fb, fdev)
    want = OL.fields(OL.run(OL.init_equilibrium(*fields), oracle_params(p), 3))
    assert rel_err(fout[0], want[0]) <= STEP_TOL and rel_err(fout[3], want[3]) <= STEP_TOL


def test_invalid_device_arguments():
    p = lbm.Params(16, 16)
    f = lbm.empty_state(p)
    with pytest.raises(lbm.LbmError):
        lbm.step(p, f, f)                                   # aliasing
    with pytest.raises(lbm.LbmError):
        lbm.step(lbm.Params(16, 16, tau=0.4), f, lbm.empty_state(p))


def test_full_size_sampled_columns():
    """4096 x 8192 (the throughput lattice, seed 2) in the launch configuration the bench
    times: two fused steps on the GPU; the oracle recomputes sampled columns from crops
    of +-6 columns (two steps reach 6 columns), built from the same seeded fields."""
    p = lbm.Params(4096, 8192)
    fields = rt_fields(p, seed=2)
    fa = device_init(p, fields)
    fb = lbm.empty_state(p)
    res = lbm.run(p, fa, fb, 2)
    got = res[:, :, : p.ly]
    for x in [0, 1234, 4095]:
        cols = [(x + d) % p.lx for d in range(-6, 7)]
        crop = [t[cols] for t in fields]
        op = OL.Params(13, p.ly, tau=p.tau, gx=p.gx, gy=p.gy, t_bottom=p.t_bottom, t_top=p.t_top)
        want = OL.run(OL.init_equilibrium(*crop), op, 2)[:, 6]
        assert rel_err(got[:, x].double().cpu(), want) <= STEP_TOL, x
    del fa, fb, res, got
    torch.cuda.empty_cache()


def test_fixed_point_moment_sums_within_float64_summation_error():
    """The FP64 path sums the populations in 64-bit fixed point (2^-52 resolution, rounded):
    the density differs from the exactly rounded sum by at most 37 * 2^-53 + 1 ulp."""
    import math
    p = lbm.Params(24, 40, gx=2e-4)
    f = lbm.run(p, device_init(p, rt_fields(p, seed=6)), lbm.empty_state(p), 3)
    rho = lbm.moments(p, f)[0].cpu()
    g = f[:, :, : p.ly].cpu()
    worst = 0.0
    for x in range(p.lx):
        for y in range(p.ly):
            exact = math.fsum(g[:, x, y].tolist())
            worst = max(worst, abs(float(rho[x, y]) - exact))
    assert worst <= 37 * 2.0 ** -53 + 2.3e-16, worst


@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP64_FIXED])
def test_stored_oracle_fixture(precision):
    """The GPU steps against the stored oracle fixture tests/golden/rt_16x32_3steps.txt
    (16 x 32, seed 9, 3 steps): per-population sums and three sampled sites."""
    from tests.test_golden_fixture import load_golden, maker
    SITES = maker().SITES
    p = lbm.Params(16, 32, precision=precision)
    res = to_host(p, lbm.run(p, device_init(p, rt_fields(p, seed=9)), lbm.empty_state(p), 3))
    want = load_golden()
    for i in range(37):
        got = [float(res[i].sum())] + [float(res[i, x, y]) for x, y in SITES]
        for a, b in zip(got, want[i]):
            assert abs(a - b) <= STEP_TOL * abs(b), (i, a, b)
