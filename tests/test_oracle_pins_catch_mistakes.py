"""The pins are not vacuous: plant plausible mistakes in the oracle (on the CPU, by
monkeypatching) and check that at least one pin fails for each."""
import pytest
import torch

import oracle.d2q37 as M
import oracle.lbm as L
from tests import test_oracle_model as TM
from tests import test_oracle_step as TS


def _fails(fn, *args):
    try:
        fn(*args)
    except AssertionError:
        return True
    return False


def _all_moment_pins_pass():
    return all(not _fails(TM.test_equilibrium_moments_match_maxwellian_to_order_four, p, q)
               for p in range(5) for q in range(5) if p + q <= 4)


def test_unmodified_oracle_passes():
    assert _all_moment_pins_pass()


@pytest.mark.parametrize("mutation", ["drop_theta2", "sign_h3", "half_a2", "drop_a4_pairs"])
def test_equilibrium_mutations_are_caught(monkeypatch, mutation):
    orig_coef, orig_herm = M.maxwell_coefficient, M.hermite

    def coef(n, u, theta, idx):
        if mutation == "drop_theta2" and n == 4:
            return orig_coef(n, u, theta, idx) - theta * theta * sum(
                [1.0 if (idx[0] == idx[1] and idx[2] == idx[3]) else 0.0,
                 1.0 if (idx[0] == idx[2] and idx[1] == idx[3]) else 0.0,
                 1.0 if (idx[0] == idx[3] and idx[1] == idx[2]) else 0.0])
        if mutation == "half_a2" and n == 2:
            return 0.5 * orig_coef(n, u, theta, idx)
        if mutation == "drop_a4_pairs" and n == 4:
            uu = [u[..., k] for k in range(2)]
            a, b, c, d = idx
            return uu[a] * uu[b] * uu[c] * uu[d] + theta * theta * (
                M._delta(a, b) * M._delta(c, d) + M._delta(a, c) * M._delta(b, d) + M._delta(a, d) * M._delta(b, c))
        return orig_coef(n, u, theta, idx)

    def herm(n, xi, idx):
        if mutation == "sign_h3" and n == 3:
            x = [xi[..., k] for k in range(2)]
            a, b, c = idx
            return x[a] * x[b] * x[c] + (x[a] * M._delta(b, c) + x[b] * M._delta(a, c) + x[c] * M._delta(a, b))
        return orig_herm(n, xi, idx)

    monkeypatch.setattr(M, "maxwell_coefficient", coef)
    monkeypatch.setattr(M, "hermite", herm)
    assert not _all_moment_pins_pass()


def test_wrong_gravity_shift_is_caught(monkeypatch):
    def bad_shift(u, T, p):
        g = torch.tensor([p.gx, p.gy], dtype=torch.float64)
        return u + p.tau * g, T          # temperature correction dropped
    monkeypatch.setattr(L, "gravity_shift", bad_shift)
    assert _fails(TS.test_collide_gravity_kick_and_unchanged_temperature)


def test_push_instead_of_pull_is_caught(monkeypatch):
    orig = L.propagate

    def push(f, p):
        opp = [0] + list(range(19, 37)) + list(range(1, 19))
        return orig(f[opp], p)[opp]      # moves every population the wrong way
    monkeypatch.setattr(L, "propagate", push)
    assert _fails(TS.test_propagate_brute_force_indices, "walls")


def test_wrong_wall_density_row_is_caught(monkeypatch):
    orig = L.bc

    def bad_bc(f_tilde, f_prev, p):
        return orig(f_tilde, torch.roll(f_prev, 1, dims=2), p)   # density from the wrong row
    monkeypatch.setattr(L, "bc", bad_bc)
    assert _fails(TS.test_bc_ghost_values_hand_computed)


def test_relaxation_with_tau_instead_of_its_inverse_is_caught(monkeypatch):
    def bad_collide(f_tilde, p):
        rho, u, T = L.moments(f_tilde)
        u_s, T_s = L.gravity_shift(u, T, p)
        return f_tilde - (f_tilde - M.equilibrium(rho, u_s, T_s)) * p.tau
    monkeypatch.setattr(L, "collide", bad_collide)
    assert _fails(TS.test_collide_relaxation_is_linear_blend)


def test_temperature_without_the_dimension_factor_is_caught(monkeypatch):
    orig = L.moments

    def bad_moments(f):
        rho, u, T = orig(f)
        return rho, u, T * M.D
    monkeypatch.setattr(L, "moments", bad_moments)
    assert _fails(TS.test_moments_recover_equilibrium_fields)


def test_swapped_wall_temperatures_are_caught(monkeypatch):
    orig = L.bc

    def bad_bc(f_tilde, f_prev, p):
        q = L.Params(p.lx, p.ly, tau=p.tau, gx=p.gx, gy=p.gy, t_bottom=p.t_top, t_top=p.t_bottom, bc=p.bc)
        return orig(f_tilde, f_prev, q)
    monkeypatch.setattr(L, "bc", bad_bc)
    assert _fails(TS.test_bc_ghost_values_hand_computed)


def test_gravity_with_the_wrong_sign_is_caught(monkeypatch):
    orig = L.gravity_shift

    def bad_shift(u, T, p):
        q = L.Params(p.lx, p.ly, tau=p.tau, gx=-p.gx, gy=-p.gy, t_bottom=p.t_bottom, t_top=p.t_top, bc=p.bc)
        return orig(u, T, q)
    monkeypatch.setattr(L, "gravity_shift", bad_shift)
    assert _fails(TS.test_collide_gravity_kick_and_unchanged_temperature)


def test_missing_periodic_wrap_in_x_is_caught(monkeypatch):
    def clamped(f, p):
        q, lx, ly = f.shape
        out = torch.empty_like(f)
        for i in range(q):
            vx, vy = M.VELOCITIES[i]
            xs = (torch.arange(lx) - vx).clamp(0, lx - 1)
            ys = torch.arange(ly) - vy
            ys = ys % ly if p.bc == "periodic_y" else ys.clamp(0, ly - 1)
            out[i] = f[i][xs][:, ys]
        return out
    monkeypatch.setattr(L, "propagate", clamped)
    assert _fails(TS.test_propagate_brute_force_indices, "walls")


@pytest.mark.parametrize("mutation", ["swap_shell_weights", "scale_off_by_1e-3"])
def test_wrong_weights_or_lattice_scale_are_caught(monkeypatch, mutation):
    if mutation == "swap_shell_weights":
        w = M.W_SHELL[:]
        w[6], w[7] = w[7], w[6]
        monkeypatch.setattr(M, "WEIGHTS", torch.tensor([w[s] for s in M.SHELL_INDEX], dtype=torch.float64))
    else:
        monkeypatch.setattr(M, "XI", M.XI * 1.001)
    pq = [(p, q) for p in range(9) for q in range(9) if p + q <= 9]
    assert any(_fails(TM.test_lattice_isotropy_all_moments_to_order_eight, p, q) for p, q in pq)
