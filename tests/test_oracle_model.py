"""Pins for the oracle's D2Q37 model: velocity set, weights, scale and equilibrium.

Every expected value here comes from mathematics independent of the oracle's code:
Gaussian moments (n-1)!!, binomial expansions of the Maxwellian's moments, and the
scalar (non-tensor) form of the fourth-order Hermite expansion.
"""
import itertools
import math

import pytest
import torch

from oracle import d2q37 as M


def gauss(n):
    return 0 if n % 2 else math.prod(range(n - 1, 0, -2))


def test_velocity_set():
    v = M.VELOCITIES
    assert len(v) == 37 and len(set(v)) == 37
    assert max(max(abs(a), abs(b)) for a, b in v) == 3          # hops up to three sites
    assert v[0] == (0, 0)
    for k in range(1, 19):
        assert v[k + 18] == (-v[k][0], -v[k][1])
    counts = [M.SHELL_INDEX.count(s) for s in range(8)]
    assert counts == [1, 4, 4, 4, 8, 4, 4, 8]


def test_weights_positive_normalised():
    assert all(w > 0 for w in M.W_SHELL)
    assert abs(float(M.WEIGHTS.sum()) - 1.0) < 1e-15
    assert 1.19 < M.C_SCALE < 1.20


@pytest.mark.parametrize("p,q", [(p, q) for p in range(9) for q in range(9) if p + q <= 9])
def test_lattice_isotropy_all_moments_to_order_eight(p, q):
    """sum_i w_i xi_x^p xi_y^q equals the Gaussian moment <Zx^p><Zy^q> for every
    p + q <= 8 (odd ones vanish by symmetry); order 9 is odd and also vanishes."""
    lhs = float((M.WEIGHTS * M.XI[:, 0] ** p * M.XI[:, 1] ** q).sum())
    rhs = gauss(p) * gauss(q)
    assert abs(lhs - rhs) <= 2e-14 * max(1.0, abs(rhs))


def test_isotropy_fails_at_order_ten():
    # Sanity that the pin is not vacuous: a 37-velocity set cannot match order 10.
    lhs = float((M.WEIGHTS * M.XI[:, 0] ** 10).sum())
    assert abs(lhs - gauss(10)) > 1e-3


def maxwell_moment_1d(u, T, n):
    """E[(u + sqrt(T) Z)^n] by the binomial expansion."""
    s = math.sqrt(T)
    return sum(math.comb(n, j) * u ** (n - j) * s ** j * gauss(j) for j in range(n + 1))


def random_states(n=6, seed=0):
    g = torch.Generator().manual_seed(seed)
    rho = 0.5 + 1.5 * torch.rand(n, generator=g, dtype=torch.float64)
    u = 0.2 * (torch.rand(n, 2, generator=g, dtype=torch.float64) - 0.5)
    T = 0.7 + 0.6 * torch.rand(n, generator=g, dtype=torch.float64)
    return rho, u, T


@pytest.mark.parametrize("p,q", [(p, q) for p in range(5) for q in range(5) if p + q <= 4])
def test_equilibrium_moments_match_maxwellian_to_order_four(p, q):
    rho, u, T = random_states()
    feq = M.equilibrium(rho, u, T)                                  # [37, n]
    lhs = (feq * (M.XI[:, 0] ** p * M.XI[:, 1] ** q)[:, None]).sum(dim=0)
    for j in range(rho.numel()):
        r, ux, uy, t = float(rho[j]), float(u[j, 0]), float(u[j, 1]), float(T[j])
        rhs = r * maxwell_moment_1d(ux, t, p) * maxwell_moment_1d(uy, t, q)
        assert abs(float(lhs[j]) - rhs) <= 1e-13 * max(1.0, abs(rhs)), (p, q, j)


def test_equilibrium_scalar_closed_form():
    """The tensor contraction equals the scalar fourth-order Hermite form
    w rho {1 + s + [s^2 - U + t(q-D)]/2 + s[s^2 - 3U + 3t(q-D-2)]/6
           + [s^4 - 6 s^2 U + 3U^2 + 6t(s^2(q-D-4) + U(D+2-q)) + 3t^2(q^2 - 2(D+2)q + D(D+2))]/24}
    with s = xi.u, U = |u|^2, q = |xi|^2, t = T - 1."""
    rho, u, T = random_states(8, seed=3)
    feq = M.equilibrium(rho, u, T)
    D = 2
    for i in range(37):
        xi = M.XI[i]
        q = float((xi * xi).sum())
        s = u[:, 0] * xi[0] + u[:, 1] * xi[1]
        U = (u * u).sum(dim=1)
        t = T - 1
        poly = (1 + s + 0.5 * (s * s - U + t * (q - D))
                + s / 6 * (s * s - 3 * U + 3 * t * (q - D - 2))
                + (s ** 4 - 6 * s * s * U + 3 * U * U + 6 * t * (s * s * (q - D - 4) + U * (D + 2 - q))
                   + 3 * t * t * (q * q - 2 * (D + 2) * q + D * (D + 2))) / 24)
        ref = M.WEIGHTS[i] * rho * poly
        torch.testing.assert_close(feq[i], ref, rtol=1e-13, atol=1e-16)


def test_equilibrium_rest_state_is_weights():
    feq = M.equilibrium(torch.tensor([1.0], dtype=torch.float64), torch.zeros(1, 2, dtype=torch.float64),
                        torch.tensor([1.0], dtype=torch.float64))
    torch.testing.assert_close(feq[:, 0], M.WEIGHTS, rtol=0, atol=1e-17)
