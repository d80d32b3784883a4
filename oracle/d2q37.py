"""D2Q37 model constants and the Hermite equilibrium, written from first principles.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper (Sec. 3, around eq. ``macro`` and Fig. ``streamscheme``) states that the
model has 37 populations in D = 2 dimensions that hop up to three lattice sites and
that the equilibrium is a function of density, velocity and temperature; it defers
the velocity table, the weights and the equilibrium to the literature it cites.  The
readings used here:

* Velocity set: the 37 integer vectors of the eight shells
  (0,0), (1,0), (1,1), (2,0), (2,1), (2,2), (3,0), (3,1) under all sign changes and
  the x<->y swap (1+4+4+4+8+4+4+8 = 37; longest hop 3, as Fig. ``streamscheme``).
* Weights and scale: the molecular velocity of population i is xi_i = c * v_i.  The
  eight shell weights and ``c`` are the unique positive solution of the nine even
  isotropy conditions  sum_i w_i xi_ix^p xi_iy^q = <Z_x^p Z_y^q>  (Z a standard
  normal pair, reference temperature T0 = 1) for (p, q) in
  (0,0),(2,0),(4,0),(2,2),(6,0),(4,2),(8,0),(6,2),(4,4).  They are solved below.
* Equilibrium: the Hermite expansion of the Maxwellian truncated at fourth order,
  f_i^eq = w_i rho sum_{n<=4} a^(n)(u, T) : H^(n)(xi_i) / n!, with a^(n) the Hermite
  coefficients of the Maxwellian of velocity u and temperature T, written below as
  explicit index sums (no factoring).

Population order (a free labelling, Fig. ``streamscheme`` calls the labels
arbitrary): index 0 is the rest population; 1..18 are the representatives listed in
``_REPS``; index 18+k is the opposite of index k.
"""
from __future__ import annotations

import itertools
import math

import mpmath as mp
import torch

D = 2
Q = 37

# Representatives with vx > 0, or vx == 0 and vy > 0; their negatives follow.
_REPS = [(1, 0), (0, 1), (1, 1), (1, -1), (2, 0), (0, 2), (2, 1), (1, 2), (2, -1),
         (1, -2), (2, 2), (2, -2), (3, 0), (0, 3), (3, 1), (1, 3), (3, -1), (1, -3)]
VELOCITIES = [(0, 0)] + _REPS + [(-a, -b) for (a, b) in _REPS]

# Shell of a vector = the sorted absolute components; eight shells.
SHELLS = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2), (3, 0), (3, 1)]


def shell_of(v):
    a, b = sorted((abs(v[0]), abs(v[1])), reverse=True)
    return SHELLS.index((a, b))


SHELL_INDEX = [shell_of(v) for v in VELOCITIES]

# Isotropy conditions: (p, q) exponents and the Gaussian moments <Z^n> = (n-1)!!.
ISOTROPY_PQ = [(0, 0), (2, 0), (4, 0), (2, 2), (6, 0), (4, 2), (8, 0), (6, 2), (4, 4)]


def gaussian_moment(n: int) -> int:
    """<Z^n> for a standard normal Z: 0 for odd n, (n-1)!! for even n."""
    if n % 2:
        return 0
    return math.prod(range(n - 1, 0, -2)) if n > 0 else 1


def _shell_sums(p, q):
    """S_s(p, q) = sum over the vectors v of shell s of vx^p vy^q (integers)."""
    out = [0] * len(SHELLS)
    for v in VELOCITIES:
        out[shell_of(v)] += v[0] ** p * v[1] ** q
    return out


def _residuals(w, c):
    """Isotropy residuals r_(p,q) = sum_s w_s c^(p+q) S_s(p,q) - <Z^p><Z^q>."""
    res = []
    for p, q in ISOTROPY_PQ:
        s = _shell_sums(p, q)
        lhs = sum(w[k] * c ** (p + q) * s[k] for k in range(len(SHELLS)))
        res.append(lhs - gaussian_moment(p) * gaussian_moment(q))
    return res


def solve_weights(dps: int = 40):
    """Solve the nine isotropy conditions for the eight shell weights and ``c``.

    For fixed c the conditions are linear in the eight weights, so the nine of them
    have a solution only where the augmented 9x9 matrix [A(c) | m] is singular.  We
    scan c for sign changes of its determinant (a polynomial in c), bisect each,
    keep the root whose least-squares weights are all positive, and polish it with
    multidimensional Newton at ``dps`` digits.
    Returns (c, [w_0..w_7]) as mpmath numbers.
    """
    mp.mp.dps = dps

    def rows_for(c):
        rows, rhs = [], []
        for p, q in ISOTROPY_PQ:
            s = _shell_sums(p, q)
            rows.append([c ** (p + q) * s[k] for k in range(len(SHELLS))])
            rhs.append(gaussian_moment(p) * gaussian_moment(q))
        return rows, rhs

    def weights_for(c):
        # least squares over all nine equations; exact where they are compatible
        rows, rhs = rows_for(c)
        return list(mp.qr_solve(mp.matrix(rows), mp.matrix(rhs))[0])

    def compat(c):
        # The nine equations in eight weights are solvable iff the augmented 9x9
        # matrix [A(c) | m] is singular; its determinant is a polynomial in c.
        rows, rhs = rows_for(c)
        return mp.det(mp.matrix([r + [m] for r, m in zip(rows, rhs)]))

    def bisect(lo, hi, g_lo):
        for _ in range(4 * dps):
            mid = (lo + hi) / 2
            g_mid = compat(mid)
            if g_mid * g_lo > 0:
                lo, g_lo = mid, g_mid
            else:
                hi = mid
        return (lo + hi) / 2

    grid = [mp.mpf(0.8) + mp.mpf(k) / 200 for k in range(241)]  # c in 0.8 .. 2.0
    roots = []
    prev_c, prev_g = None, None
    for c in grid:
        g = compat(c)
        if prev_g is not None and prev_g * g < 0:
            root_c = bisect(prev_c, c, prev_g)
            if all(wk > 0 for wk in weights_for(root_c)):
                roots.append(root_c)
        prev_c, prev_g = c, g
    if len(roots) != 1:
        raise RuntimeError(f"expected one positive isotropic solution, found {len(roots)}")
    c0 = roots[0]
    w0 = weights_for(c0)
    sol = mp.findroot(lambda *z: _residuals(z[:8], z[8]), list(w0) + [c0])
    return sol[8], [sol[k] for k in range(8)]


_C_MP, _W_SHELL_MP = solve_weights()
C_SCALE = float(_C_MP)
W_SHELL = [float(w) for w in _W_SHELL_MP]
WEIGHTS = torch.tensor([W_SHELL[s] for s in SHELL_INDEX], dtype=torch.float64)
V_INT = torch.tensor(VELOCITIES, dtype=torch.int64)            # [37, 2] integer hops
XI = V_INT.to(torch.float64) * C_SCALE                          # [37, 2] xi_i = c v_i


# ---------------------------------------------------------------------------
# Hermite tensors and Maxwellian coefficients, written as explicit index sums.
# ---------------------------------------------------------------------------
def _delta(a, b):
    return 1.0 if a == b else 0.0


def hermite(n, xi, idx):
    """Tensor Hermite polynomial H^(n)_{idx}(xi) (probabilists', unit variance).

    xi: [..., D] tensor; idx: tuple of n axis indices.
    H0 = 1; H1_a = x_a; H2_ab = x_a x_b - d_ab;
    H3_abc = x_a x_b x_c - (x_a d_bc + x_b d_ac + x_c d_ab);
    H4_abcd = x_a x_b x_c x_d - (x_a x_b d_cd + x_a x_c d_bd + x_a x_d d_bc
              + x_b x_c d_ad + x_b x_d d_ac + x_c x_d d_ab)
              + (d_ab d_cd + d_ac d_bd + d_ad d_bc).
    """
    x = [xi[..., k] for k in range(D)]
    if n == 0:
        return torch.ones_like(x[0])
    if n == 1:
        (a,) = idx
        return x[a]
    if n == 2:
        a, b = idx
        return x[a] * x[b] - _delta(a, b)
    if n == 3:
        a, b, c = idx
        return x[a] * x[b] * x[c] - (x[a] * _delta(b, c) + x[b] * _delta(a, c) + x[c] * _delta(a, b))
    if n == 4:
        a, b, c, d = idx
        quad = x[a] * x[b] * x[c] * x[d]
        pairs = (x[a] * x[b] * _delta(c, d) + x[a] * x[c] * _delta(b, d) + x[a] * x[d] * _delta(b, c)
                 + x[b] * x[c] * _delta(a, d) + x[b] * x[d] * _delta(a, c) + x[c] * x[d] * _delta(a, b))
        dd = _delta(a, b) * _delta(c, d) + _delta(a, c) * _delta(b, d) + _delta(a, d) * _delta(b, c)
        return quad - pairs + dd
    raise ValueError(n)


def maxwell_coefficient(n, u, theta, idx):
    """Hermite coefficient a^(n)_{idx} of the Maxwellian with velocity u, temperature
    1 + theta (per unit density):
    a0 = 1; a1_a = u_a; a2_ab = u_a u_b + th d_ab;
    a3_abc = u_a u_b u_c + th (u_a d_bc + u_b d_ac + u_c d_ab);
    a4_abcd = u_a u_b u_c u_d + th (u_a u_b d_cd + u_a u_c d_bd + u_a u_d d_bc
              + u_b u_c d_ad + u_b u_d d_ac + u_c u_d d_ab)
              + th^2 (d_ab d_cd + d_ac d_bd + d_ad d_bc).
    u: [..., D]; theta: [...].
    """
    uu = [u[..., k] for k in range(D)]
    if n == 0:
        return torch.ones_like(theta)
    if n == 1:
        (a,) = idx
        return uu[a]
    if n == 2:
        a, b = idx
        return uu[a] * uu[b] + theta * _delta(a, b)
    if n == 3:
        a, b, c = idx
        return uu[a] * uu[b] * uu[c] + theta * (uu[a] * _delta(b, c) + uu[b] * _delta(a, c) + uu[c] * _delta(a, b))
    if n == 4:
        a, b, c, d = idx
        quad = uu[a] * uu[b] * uu[c] * uu[d]
        pairs = (uu[a] * uu[b] * _delta(c, d) + uu[a] * uu[c] * _delta(b, d) + uu[a] * uu[d] * _delta(b, c)
                 + uu[b] * uu[c] * _delta(a, d) + uu[b] * uu[d] * _delta(a, c) + uu[c] * uu[d] * _delta(a, b))
        dd = _delta(a, b) * _delta(c, d) + _delta(a, c) * _delta(b, d) + _delta(a, d) * _delta(b, c)
        return quad + theta * pairs + theta * theta * dd
    raise ValueError(n)


def equilibrium(rho, u, T, order: int = 4):
    """f_i^eq(rho, u, T) for all 37 populations (Sec. 3: the equilibrium is a
    function of the macroscopic fields; the fourth-order Hermite form is the
    reading stated in the module docstring).

    rho, T: [...] float64; u: [..., 2] float64.  Returns [37, ...].
    """
    theta = T - 1.0
    out = []
    for i in range(Q):
        xi = XI[i]
        acc = torch.zeros_like(rho)
        for n in range(order + 1):
            for idx in itertools.product(range(D), repeat=n):
                acc = acc + maxwell_coefficient(n, u, theta, idx) * hermite(n, xi, idx) / math.factorial(n)
        out.append(WEIGHTS[i] * rho * acc)
    return torch.stack(out)
