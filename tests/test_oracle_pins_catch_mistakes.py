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
