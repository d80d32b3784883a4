"""Pins for the oracle's propagate, bc, collide and step.

Expected values come from invariants of the method (conservation, permutation,
round trips, fixed points), from hand-written index arithmetic on tiny lattices, and
from the closed form of the rest-state equilibrium.
"""
import math

import pytest
import torch

from oracle import d2q37 as M
from oracle import lbm as L


def near_equilibrium(lx, ly, seed=0, noise=0.01):
    g = torch.Generator().manual_seed(seed)
    rho = 0.8 + 0.4 * torch.rand(lx, ly, generator=g, dtype=torch.float64)
    u = 0.05 * (torch.rand(lx, ly, 2, generator=g, dtype=torch.float64) - 0.5)
    T = 0.9 + 0.2 * torch.rand(lx, ly, generator=g, dtype=torch.float64)
    f = M.equilibrium(rho, u, T)
    return f * (1 + noise * (torch.rand(f.shape, generator=g, dtype=torch.float64) - 0.5))


def conserved(f):
    rho = f.sum(0)
    jx = (M.XI[:, 0, None, None] * f).sum(0)
    jy = (M.XI[:, 1, None, None] * f).sum(0)
    e = ((M.XI * M.XI).sum(1)[:, None, None] * f).sum(0)
    return rho, jx, jy, e


# ----------------------------------------------------------------------------- collide
def test_collide_conserves_mass_momentum_energy_without_gravity():
    p = L.Params(4, 6, tau=0.8, gx=0.0, gy=0.0)
    f = near_equilibrium(4, 6)
    a, b = conserved(f), conserved(L.collide(f, p))
    for x, y in zip(a, b):
        torch.testing.assert_close(y, x, rtol=2e-15, atol=1e-15)


def test_collide_gravity_kick_and_unchanged_temperature():
    p = L.Params(4, 6, tau=0.7, gx=3e-3, gy=-1e-3)
    f = near_equilibrium(4, 6, seed=1)
    rho0, u0, T0 = L.moments(f)
    rho1, u1, T1 = L.moments(L.collide(f, p))
    torch.testing.assert_close(rho1, rho0, rtol=2e-15, atol=0)
    torch.testing.assert_close(u1[..., 0] - u0[..., 0], torch.full_like(rho0, 3e-3), rtol=0, atol=1e-15)
    torch.testing.assert_close(u1[..., 1] - u0[..., 1], torch.full_like(rho0, -1e-3), rtol=0, atol=1e-15)
    torch.testing.assert_close(T1, T0, rtol=2e-15, atol=0)


def test_collide_fixed_point_at_equilibrium():
    p = L.Params(4, 6, tau=0.9, gx=0.0, gy=0.0)
    f = near_equilibrium(4, 6, seed=2, noise=0.0)
    torch.testing.assert_close(L.collide(f, p), f, rtol=1e-14, atol=1e-17)


def test_collide_tau_one_gives_equilibrium_of_moments():
    p = L.Params(4, 6, tau=1.0, gx=0.0, gy=0.0)
    f = near_equilibrium(4, 6, seed=3)
    rho, u, T = L.moments(f)
    torch.testing.assert_close(L.collide(f, p), M.equilibrium(rho, u, T), rtol=1e-14, atol=1e-17)


def test_collide_relaxation_is_linear_blend():
    # f' = (1 - 1/tau) f + (1/tau) f^eq(moments): check against tau = 1 result
    f = near_equilibrium(4, 6, seed=4)
    feq = L.collide(f, L.Params(4, 6, tau=1.0, gx=0.0, gy=0.0))
    tau = 0.65
    ref = (1 - 1 / tau) * f + feq / tau
    torch.testing.assert_close(L.collide(f, L.Params(4, 6, tau=tau, gx=0.0, gy=0.0)), ref, rtol=1e-13, atol=1e-16)


def test_moments_recover_equilibrium_fields():
    g = torch.Generator().manual_seed(5)
    rho = 0.8 + 0.4 * torch.rand(3, 5, generator=g, dtype=torch.float64)
    u = 0.1 * (torch.rand(3, 5, 2, generator=g, dtype=torch.float64) - 0.5)
    T = 0.85 + 0.3 * torch.rand(3, 5, generator=g, dtype=torch.float64)
    r2, u2, T2 = L.moments(M.equilibrium(rho, u, T))
    torch.testing.assert_close(r2, rho, rtol=1e-15, atol=0)
    torch.testing.assert_close(u2, u, rtol=0, atol=1e-15)
    torch.testing.assert_close(T2, T, rtol=1e-14, atol=0)


# --------------------------------------------------------------------------- propagate
def encoded(lx, ly):
    i = torch.arange(37, dtype=torch.float64)[:, None, None]
    x = torch.arange(lx, dtype=torch.float64)[None, :, None]
    y = torch.arange(ly, dtype=torch.float64)[None, None, :]
    return i * 10000 + x * 100 + y


@pytest.mark.parametrize("bc", ["walls", "periodic_y"])
def test_propagate_brute_force_indices(bc):
    lx, ly = 4, 8
    p = L.Params(lx, ly, bc=bc)
    out = L.propagate(encoded(lx, ly), p)
    for i in range(37):
        vx, vy = M.VELOCITIES[i]
        for x in range(lx):
            for y in range(ly):
                ys = y - vy
                if bc == "walls" and not (0 <= ys < ly):
                    continue
                want = i * 10000 + ((x - vx) % lx) * 100 + (ys % ly)
                assert float(out[i, x, y]) == want


def test_propagate_is_permutation_and_round_trips():
    lx, ly = 5, 7
    p = L.Params(lx, ly, bc="periodic_y")
    f = torch.rand(37, lx, ly, dtype=torch.float64, generator=torch.Generator().manual_seed(0))
    g = L.propagate(f, p)
    assert torch.equal(torch.sort(g.flatten()).values, torch.sort(f.flatten()).values)
    opp = [0] + list(range(19, 37)) + list(range(1, 19))
    back = L.propagate(g[opp], p)[opp]
    assert torch.equal(back, f)


# --------------------------------------------------------------------------------- bc
def rest_weight_polynomial(q, theta):
    """f^eq(rho, 0, T) / (w rho) = 1 + theta(q - D)/2 + theta^2 (q^2 - 2(D+2) q + D(D+2))/8."""
    D = 2
    return 1 + 0.5 * theta * (q - D) + theta * theta * (q * q - 2 * (D + 2) * q + D * (D + 2)) / 8


def test_bc_ghost_values_hand_computed():
    lx, ly = 4, 8
    p = L.Params(lx, ly, t_bottom=1.15, t_top=0.85)
    f = near_equilibrium(lx, ly, seed=7)
    out = L.bc(L.propagate(f, p), f, p)
    for i in range(37):
        vx, vy = M.VELOCITIES[i]
        q = M.C_SCALE ** 2 * (vx * vx + vy * vy)
        for x in range(lx):
            xs = (x - vx) % lx
            for y in range(ly):
                ys = y - vy
                if 0 <= ys < ly:
                    want = f[i, xs, ys]
                elif ys < 0:
                    want = M.W_SHELL[M.SHELL_INDEX[i]] * float(f[:, xs, 0].sum()) * rest_weight_polynomial(q, 0.15)
                else:
                    want = M.W_SHELL[M.SHELL_INDEX[i]] * float(f[:, xs, ly - 1].sum()) * rest_weight_polynomial(q, -0.15)
                assert abs(float(out[i, x, y]) - float(want)) <= 4e-15 * abs(float(want)), (i, x, y)


def test_bc_rows_affected_are_the_three_outermost():
    lx, ly = 4, 10
    p = L.Params(lx, ly)
    f = near_equilibrium(lx, ly, seed=8)
    g = L.propagate(f, p)
    changed = (L.bc(g, f, p) != g).any(dim=0).any(dim=0)
    assert changed.tolist() == [True] * 3 + [False] * 4 + [True] * 3


def test_bc_is_linear_in_f():
    lx, ly = 4, 8
    p = L.Params(lx, ly)
    f1, f2 = near_equilibrium(lx, ly, seed=9), near_equilibrium(lx, ly, seed=10)
    lhs = L.bc(L.propagate(0.3 * f1 + 0.7 * f2, p), 0.3 * f1 + 0.7 * f2, p)
    rhs = 0.3 * L.bc(L.propagate(f1, p), f1, p) + 0.7 * L.bc(L.propagate(f2, p), f2, p)
    torch.testing.assert_close(lhs, rhs, rtol=1e-14, atol=1e-17)


def test_rest_state_at_wall_temperature_is_fixed_point_of_step():
    lx, ly = 4, 8
    p = L.Params(lx, ly, gx=0.0, gy=0.0, t_bottom=1.1, t_top=1.1)
    rho = torch.full((lx, ly), 1.3, dtype=torch.float64)
    T = torch.full((lx, ly), 1.1, dtype=torch.float64)
    f = L.init_equilibrium(rho, torch.zeros_like(rho), torch.zeros_like(rho), T)
    torch.testing.assert_close(L.step(f, p), f, rtol=1e-14, atol=1e-17)


# ------------------------------------------------------------------------------ step
def test_periodic_step_global_conservation_with_gravity():
    lx, ly = 6, 8
    p = L.Params(lx, ly, tau=0.8, gx=0.0, gy=-1e-3, bc="periodic_y")
    f = near_equilibrium(lx, ly, seed=11)
    m0 = f.sum()
    jy0 = (M.XI[:, 1, None, None] * f).sum()
    n = 3
    fn = L.run(f, p, n)
    torch.testing.assert_close(fn.sum(), m0, rtol=1e-14, atol=0)
    jyn = (M.XI[:, 1, None, None] * fn).sum()
    assert abs(float(jyn - jy0) - n * float(m0) * -1e-3) < 1e-13


def test_kinetic_energy_definition():
    lx, ly = 3, 4
    g = torch.Generator().manual_seed(12)
    rho = 1 + 0.1 * torch.rand(lx, ly, generator=g, dtype=torch.float64)
    u = 0.05 * torch.rand(lx, ly, 2, generator=g, dtype=torch.float64)
    T = torch.ones(lx, ly, dtype=torch.float64)
    f = M.equilibrium(rho, u, T)
    want = 0.5 * float((rho * (u * u).sum(-1)).sum())
    assert abs(float(L.kinetic_energy(f)) - want) < 1e-15 * want
