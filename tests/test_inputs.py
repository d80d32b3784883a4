"""Seeded Rayleigh-Taylor input fields: determinism, amplitude rule, hydrostatics."""
import math

import torch

from paper_1703_04594_gb300 import inputs as I


def test_seeded_and_deterministic():
    a = I.rt_state(32, 64, seed=1)
    b = I.rt_state(32, 64, seed=1)
    c = I.rt_state(32, 64, seed=2)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    assert not torch.equal(a[3], c[3])


def test_interface_amplitude_is_one_percent_of_height():
    lx, ly = 64, 128
    m = I.rt_modes(lx, ly, seed=3)
    dev = I.interface(lx, ly, m) - ly / 2
    assert abs(float(dev.abs().max()) - 0.01 * ly) < 1e-12


def test_unperturbed_column_matches_continuous_hydrostatics():
    """With a = 0 the column is the tanh profile; the trapezoid pressure must match
    p(y) = exp(-g int_{Ly/2}^{y} dy/T) with the closed-form primitive
    int dy / (A + B tanh z) = w [A z - B ln(A cosh z + B sinh z)] / (A^2 - B^2),
    z = (y - Ly/2)/w, A = (Tb+Tt)/2, B = (Tt-Tb)/2."""
    lx, ly, g = 4, 256, 1e-4
    modes = I.RTModes(a=torch.zeros(8, dtype=torch.float64), phi=torch.zeros(8, dtype=torch.float64))
    tb, tt = 1.15, 0.85
    rho, ux, uy, T = I.rt_fields(lx, ly, modes, t_bottom=tb, t_top=tt, g=g)
    A, B, w = (tb + tt) / 2, (tt - tb) / 2, I.INTERFACE_WIDTH

    def prim(y):
        z = (y - ly / 2) / w
        return w * (A * z - B * math.log(A * math.cosh(z) + B * math.sinh(z))) / (A * A - B * B)

    for y in range(0, ly, 7):
        p_exact = math.exp(-g * (prim(y) - prim(ly // 2)))
        p_num = float(rho[0, y] * T[0, y])
        assert abs(p_num - p_exact) < 2e-6 * p_exact, y
    assert torch.all(ux == 0) and torch.all(uy == 0)
    # hot below, cold above; dense cold layer on top (Rayleigh-Taylor unstable)
    assert float(T[0, 0]) > 1.14 and float(T[0, -1]) < 0.86
    assert float(rho[0, -1]) > float(rho[0, 0])


def test_fields_differentiable_in_amplitudes():
    lx, ly = 16, 32
    m = I.rt_modes(lx, ly, seed=4)
    m.a.requires_grad_(True)
    rho, _, _, T = I.rt_fields(lx, ly, m)
    (rho.sum() + T.sum()).backward()
    assert m.a.grad is not None and torch.isfinite(m.a.grad).all()


def test_batch_workload_follows_its_recipe():
    """The batched workload: 256 lattices, Lx from {128, 192, ..., 1024}, Ly = 2 Lx,
    tau in [0.6, 1.0], distinct interface seeds, deterministic for its seed, and the
    234.0 M sites the batched bench line reports for seed 4."""
    w = I.batch_workload()
    assert w == I.batch_workload() and len(w) == 256
    assert all(lx in range(128, 1025, 64) and ly == 2 * lx for lx, ly, _, _ in w)
    assert all(0.6 <= tau <= 1.0 for _, _, tau, _ in w)
    assert len({s for *_, s in w}) == 256
    assert len({lx for lx, *_ in w}) >= 12            # uneven sizes: most of the 15 values occur
    assert round(sum(lx * ly for lx, ly, _, _ in w) / 1e6, 1) == 234.0
    assert I.batch_workload(seed=5) != w
