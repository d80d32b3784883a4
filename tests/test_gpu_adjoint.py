"""Hand-written adjoint of the FP64 step (C-ABI lbm_adjoint_step and friends) and the
checkpointed reverse mode built on it.

Checks: (1) dot-product test of one adjoint step against central differences of the
forward step; (2) the full gradient of the kinetic energy after 20 steps on 32 x 64 with
respect to the 8 interface amplitudes and tau against the oracle's reverse-mode gradient;
(3) the same gradient on 512 x 1024 after 500 steps with checkpoints every 22 steps
against central finite differences (h = 1e-6) of GPU forward runs.
"""
import time

import pytest
import torch

from oracle import lbm as OL
from paper_1703_04594_gb300 import adjoint as A
from paper_1703_04594_gb300 import inputs as I
from paper_1703_04594_gb300 import lbm
from tests.gpu_util import device_init, oracle_params, require_gpu, rt_fields, to_host

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-6


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def gpu_energy_and_grad(lx, ly, seed, tau, steps, every=None, gx=0.0, gy=-1e-4, precision=lbm.FP64,
                        recompute_precision=None):
    m = I.rt_modes(lx, ly, seed)
    a = m.a.clone().requires_grad_(True)
    fields = I.rt_fields(lx, ly, I.RTModes(a=a, phi=m.phi), g=abs(gy))
    dev = [t.cuda() for t in fields]
    tau_t = torch.tensor(tau, dtype=torch.float64, requires_grad=True)
    p = lbm.Params(lx, ly, tau=tau, gx=gx, gy=gy, precision=precision)
    e = A.kinetic_energy_after(*dev, tau_t, p, steps, every, recompute_precision=recompute_precision)
    e.backward()
    return float(e), a.grad.clone(), float(tau_t.grad)


def gpu_energy(lx, ly, a, phi, tau, steps, gx=0.0, gy=-1e-4):
    fields = I.rt_fields(lx, ly, I.RTModes(a=a, phi=phi), g=abs(gy))
    p = lbm.Params(lx, ly, tau=tau, gx=gx, gy=gy)
    f = lbm.empty_state(p)
    lbm.init(p, *[t.contiguous().cuda() for t in fields], f)
    res = lbm.run(p, f, lbm.empty_state(p), steps)
    return float(lbm.kinetic_energy(p, res))


@pytest.mark.parametrize("bc", [lbm.BC_WALLS, lbm.BC_PERIODIC_Y])
def test_adjoint_step_dot_product(bc):
    p = lbm.Params(24, 40, tau=0.7, gx=3e-4, gy=-2e-4, bc=bc)
    fields = I.rt_state(p.lx, p.ly, 7)
    fields = (fields[0], fields[1] + 0.01, fields[2] - 0.005, fields[3])
    f = lbm.empty_state(p)
    lbm.init(p, *[t.contiguous().cuda() for t in fields], f)
    f = lbm.run(p, f, lbm.empty_state(p), 2).clone()
    g = torch.Generator(device="cuda").manual_seed(0)
    lam = torch.randn(f.shape, dtype=torch.float64, device="cuda", generator=g)
    v = torch.randn(f.shape, dtype=torch.float64, device="cuda", generator=g) * f.abs()
    lam[:, :, p.ly:] = 0
    v[:, :, p.ly:] = 0
    h = 1e-6
    sp, sm = lbm.empty_state(p), lbm.empty_state(p)
    lbm.step(p, f + h * v, sp)
    lbm.step(p, f - h * v, sm)
    jv = ((sp - sm) / (2 * h))[:, :, : p.ly]
    lhs = float((lam[:, :, : p.ly] * jv).sum())
    lam_n = lbm.empty_state(p)
    dtau = torch.zeros((), dtype=torch.float64, device="cuda")
    lbm.adjoint_step(p, f, lam, lam_n, dtau, lbm.adjoint_work(p))
    rhs = float((lam_n[:, :, : p.ly] * v[:, :, : p.ly]).sum())
    assert abs(lhs - rhs) <= 1e-7 * abs(rhs), (lhs, rhs)
    # dL/dtau of one step against central differences in tau
    ht = 1e-6
    pp = lbm.Params(p.lx, p.ly, tau=p.tau + ht, gx=p.gx, gy=p.gy, bc=bc)
    pm = lbm.Params(p.lx, p.ly, tau=p.tau - ht, gx=p.gx, gy=p.gy, bc=bc)
    lbm.step(pp, f, sp)
    lbm.step(pm, f, sm)
    fd = float((lam[:, :, : p.ly] * ((sp - sm) / (2 * ht))[:, :, : p.ly]).sum())
    assert abs(fd - float(dtau)) <= 1e-6 * abs(fd), (fd, float(dtau))


def oracle_vjp(p, f_host, lam):
    """(d step / d f)^T lam and d(lam . step)/d tau by torch autograd through the oracle."""
    fo = f_host.clone().requires_grad_(True)
    tau_t = torch.tensor(p.tau, dtype=torch.float64, requires_grad=True)
    op = oracle_params(p)
    op = OL.Params(op.lx, op.ly, tau=tau_t, gx=op.gx, gy=op.gy, t_bottom=op.t_bottom, t_top=op.t_top, bc=op.bc)
    (OL.step(fo, op) * lam).sum().backward()
    return fo.grad, float(tau_t.grad)


def reach_max(m, bc):
    """max of m over the sites within 3 lattice steps (x periodic; y periodic or clamped)."""
    pad_y = 3
    if bc == lbm.BC_PERIODIC_Y:
        mm = torch.cat([m[:, -pad_y:], m, m[:, :pad_y]], dim=1)
    else:
        mm = torch.cat([m[:, :1].expand(-1, pad_y), m, m[:, -1:].expand(-1, pad_y)], dim=1)
    mm = torch.cat([mm[-3:], mm, mm[:3]], dim=0)
    return torch.nn.functional.max_pool2d(mm[None, None], 7, stride=1)[0, 0]


@pytest.mark.parametrize("bc", [lbm.BC_WALLS, lbm.BC_PERIODIC_Y])
@pytest.mark.parametrize("kind", ["rt", "hot_fast", "wide_lambda"])
def test_adjoint_step_matches_oracle_vjp(kind, bc):
    """One adjoint step against autograd through the oracle's step, per element.
    'rt': a Rayleigh-Taylor state; 'hot_fast': temperatures up to 1.38 and a drift of
    c u ~ 0.2, so that sites leave the fixed-point range of the VJP (t > 0.25,
    |c u_s| > 0.15) and take the float64 path, mixed with in-range sites within a warp;
    'wide_lambda': lambda scaled per site by 10^U(-6, 3), so that the outputs of a small
    site next to large ones (its VJP in block fixed point) are checked against the largest
    lambda within its reach, not against the lattice maximum."""
    p = lbm.Params(20, 40, tau=0.7, gx=1e-4, gy=-2e-4, bc=bc)
    rho, ux, uy, T = rt_fields(p, seed=11)
    if kind == "hot_fast":
        T = T * 1.2
        ux = ux + 0.17
    f = device_init(p, (rho, ux, uy, T))
    f = lbm.run(p, f, lbm.empty_state(p), 2).clone()
    g = torch.Generator().manual_seed(13)
    lam = torch.randn(37, p.lx, p.ly, dtype=torch.float64, generator=g)
    if kind == "wide_lambda":
        lam = lam * 10.0 ** (torch.rand(1, p.lx, p.ly, dtype=torch.float64, generator=g) * 9.0 - 6.0)
    lam_dev = lbm.empty_state(p)
    lam_dev.zero_()
    lam_dev[:, :, : p.ly] = lam.cuda()
    lam_n = lbm.empty_state(p)
    dtau = torch.zeros((), dtype=torch.float64, device="cuda")
    lbm.adjoint_step(p, f, lam_dev, lam_n, dtau, lbm.adjoint_work(p))
    want, want_tau = oracle_vjp(p, to_host(p, f), lam)
    got = to_host(p, lam_n)
    scale = reach_max(lam.abs().amax(0), bc)[None]
    err = float(((got - want).abs() / scale).max())
    assert err <= 1e-13, err
    assert abs(float(dtau) - want_tau) <= 1e-10 * abs(want_tau), (float(dtau), want_tau)


def test_gradient_matches_oracle_reverse_mode_32x64_20_steps():
    lx, ly, seed, tau, steps = 32, 64, 3, 0.8, 20
    e, ga, gt = gpu_energy_and_grad(lx, ly, seed, tau, steps, every=5, gx=1e-4, gy=-1e-4)
    m = I.rt_modes(lx, ly, seed)
    a = m.a.clone().requires_grad_(True)
    tau_t = torch.tensor(tau, dtype=torch.float64, requires_grad=True)
    fields = I.rt_fields(lx, ly, I.RTModes(a=a, phi=m.phi), g=1e-4)
    f = OL.init_equilibrium(*fields)
    op = OL.Params(lx, ly, tau=tau_t, gx=1e-4, gy=-1e-4)
    eo = OL.kinetic_energy(OL.run(f, op, steps))
    eo.backward()
    assert abs(e - float(eo)) <= 1e-10 * float(eo)
    scale = float(a.grad.abs().max())
    assert float((ga - a.grad).abs().max()) <= GRAD_TOL * scale, (ga, a.grad)
    assert abs(gt - float(tau_t.grad)) <= GRAD_TOL * abs(float(tau_t.grad)), (gt, float(tau_t.grad))


def test_fixed_point_forward_gives_the_same_gradient():
    """Forward steps with the fixed-point relaxation (LBM_FP64_FIXED) reach the same states
    within rounding, so the checkpointed gradient is the same within 1e-9."""
    args = (64, 128, 4, 0.8, 40)
    e0, ga0, gt0 = gpu_energy_and_grad(*args, every=7)
    e1, ga1, gt1 = gpu_energy_and_grad(*args, every=7, precision=lbm.FP64_FIXED)
    assert abs(e1 - e0) <= 1e-12 * abs(e0)
    assert float((ga1 - ga0).abs().max()) <= 1e-9 * float(ga0.abs().max())
    assert abs(gt1 - gt0) <= 1e-9 * abs(gt0)


def test_gradient_matches_finite_differences_512x1024_500_steps():
    """The differentiation workload: 512 x 1024, 500 steps, checkpoints every 22 steps;
    dE/da_k (k = 1..8) and dE/dtau against central differences of GPU forward runs.

    Two step sizes.  With h = 1e-6 the difference E(a+h) - E(a-h) of the weakly coupled
    amplitudes is only ~1e-9 of E, so the forward runs' own float64 rounding limits that
    difference quotient to ~1e-4 relative; the adjoint must agree within 3e-4 there.  With
    h = 1e-3 (truncation error (h / interface width)^2 ~ 2.5e-7) the quotient is accurate and
    the adjoint must agree within 1e-6.
    """
    lx, ly, seed, tau, steps = 512, 1024, 5, 0.8, 500
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e, ga, gt = gpu_energy_and_grad(lx, ly, seed, tau, steps, every=22)
    torch.cuda.synchronize()
    t_grad = time.perf_counter() - t0
    m = I.rt_modes(lx, ly, seed)
    t0 = time.perf_counter()
    gpu_energy(lx, ly, m.a, m.phi, tau, steps)
    t_fwd = time.perf_counter() - t0
    print(f"forward {t_fwd:.3f} s, forward + checkpointed adjoint {t_grad:.3f} s")
    errs = {}
    for h in (1e-6, 1e-3):
        err = []
        for k in range(8):
            ap, am = m.a.clone(), m.a.clone()
            ap[k] += h
            am[k] -= h
            fd = (gpu_energy(lx, ly, ap, m.phi, tau, steps) - gpu_energy(lx, ly, am, m.phi, tau, steps)) / (2 * h)
            err.append(abs(fd - float(ga[k])) / abs(fd))
        ht = h * tau
        fd_tau = (gpu_energy(lx, ly, m.a, m.phi, tau + ht, steps)
                  - gpu_energy(lx, ly, m.a, m.phi, tau - ht, steps)) / (2 * ht)
        err.append(abs(fd_tau - gt) / abs(fd_tau))
        errs[h] = err
        print(f"h={h:g}: relative gradient errors (a_1..a_8, tau):", [f"{x:.2e}" for x in err])
    assert max(errs[1e-3]) <= GRAD_TOL, errs
    assert max(errs[1e-6]) <= 3e-4, errs


def test_fixed_point_recomputation_gives_the_same_gradient():
    """FP64 forward steps with the backward pass's segments recomputed by the fixed-point
    relaxation (the default) against the float64 recomputation: the same energy (the
    forward pass is the FP64 one) and the same gradient within 1e-9."""
    args = (64, 128, 4, 0.8, 40)
    e0, ga0, gt0 = gpu_energy_and_grad(*args, every=7, recompute_precision=lbm.FP64)
    e1, ga1, gt1 = gpu_energy_and_grad(*args, every=7)
    assert e1 == e0
    assert float((ga1 - ga0).abs().max()) <= 1e-9 * float(ga0.abs().max())
    assert abs(gt1 - gt0) <= 1e-9 * abs(gt0)


def test_every_state_kept_gives_the_same_gradient():
    """every = 1 keeps every state and recomputes none: the adjoint steps see the same
    states in the same order, so the gradient is bit for bit that of every = 7 with the
    float64 recomputation."""
    args = (64, 128, 4, 0.8, 40)
    e0, ga0, gt0 = gpu_energy_and_grad(*args, every=7, recompute_precision=lbm.FP64)
    e1, ga1, gt1 = gpu_energy_and_grad(*args, every=1)
    assert e1 == e0
    assert torch.equal(ga1, ga0)
    assert gt1 == gt0
