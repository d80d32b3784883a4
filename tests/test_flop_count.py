"""Algorithmic float64 work per site of the fused step, counted, for the FP64 roofline.

The bench reports the float64 step against the FP64 pipe's peak, so its "achieved" figure
rests on a flop count per site.  That count is frozen here: the factored collision that the
float64 kernel evaluates (moments, the gravity-shifted site scalars, per-shell Hermite
coefficients, one even/odd Horner pair per opposite pair of velocities, BGK relaxation;
Sec. 3, eqs. "lbequation" and "macro") is written out once more in plain Python on a number
type that counts every floating-point operation it takes part in.  Operations between
compile-time constants (the lattice scale, weights, shell |xi|^2, 1/6, ...) are folded and
not counted; an FMA counts as 2 flops.  The moments are counted as float64 sums of the
factored form: pair sums P = f_v + f_-v and differences M = f_v - f_-v, grouped by their
integer velocity weights (the kernel takes them on the integer pipe, which moves work
between pipes but is the same algorithm).

The counted formulation is first checked to be the method: on random near-equilibrium
sites it reproduces the oracle's collision (the unfactored tensor-Hermite form) within
rounding.  Then its total is the bench's FLOPS_PER_SITE_FP64.
"""
import os
import sys

import pytest
import torch

from oracle import d2q37 as M
from oracle import lbm as OL

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class Counter:
    def __init__(self):
        self.n = {"add": 0, "mul": 0, "fma": 0, "div": 0}

    def flops(self):
        return self.n["add"] + self.n["mul"] + 2 * self.n["fma"] + self.n["div"]


class Num:
    """A float64 value that records each arithmetic operation it enters in ``Num.ctr``."""
    ctr = None

    def __init__(self, v):
        self.v = float(v)

    @staticmethod
    def val(x):
        return x.v if isinstance(x, Num) else float(x)

    def _op(self, kind, value):
        Num.ctr.n[kind] += 1
        return Num(value)

    def __add__(self, o):
        return self._op("add", self.v + Num.val(o))

    __radd__ = __add__

    def __sub__(self, o):
        return self._op("add", self.v - Num.val(o))

    def __rsub__(self, o):
        return self._op("add", Num.val(o) - self.v)

    def __mul__(self, o):
        return self._op("mul", self.v * Num.val(o))

    __rmul__ = __mul__

    def __truediv__(self, o):
        return self._op("div", self.v / Num.val(o))

    def __rtruediv__(self, o):
        return self._op("div", Num.val(o) / self.v)

    def __neg__(self):                       # a sign flip is free (an operand modifier)
        return Num(-self.v)


def fma(a, b, c):
    Num.ctr.n["fma"] += 1
    return Num(Num.val(a) * Num.val(b) + Num.val(c))


D = 2.0
C = M.C_SCALE
C2 = C * C
W_SHELL = M.W_SHELL
SHELL_V2 = [0, 1, 2, 4, 5, 8, 9, 10]
REPS = M.VELOCITIES[1:19]                    # opposite of rep k is index 18 + k


def shell_of_rep(k):
    vx, vy = REPS[k - 1]
    return SHELL_V2.index(vx * vx + vy * vy)


def factored_collide(f, tau, gx, gy):
    """One site: the 37 post-collision populations, from the 37 gathered ones ``f``
    (Nums).  The host-side constants (omega, 1 - omega, c tau g, the temperature shift) are
    inputs of the step, so they are Nums too; everything else constant is folded."""
    omega, om1 = Num(1.0 / tau), Num(1.0 - 1.0 / tau)
    cgx, cgy = Num(C * tau * gx), Num(C * tau * gy)
    tshift = Num(tau * (1.0 - tau) * (gx * gx + gy * gy) / D - 1.0)
    # moments in integer-velocity units from the pair sums P_k = f_k + f_-k and
    # differences M_k = f_k - f_-k, grouped by their integer weights: P by |v|^2 (the group
    # sums also give rho), M by vx and by |vy| (with the sign of vy); one multiply-add per
    # weight value above 1
    P = {k: f[k] + f[k + 18] for k in range(1, 19)}
    Md = {k: f[k] - f[k + 18] for k in range(1, 19)}

    def group_sum(keys, terms, sign=lambda k: 1):
        acc = None
        for k in keys:
            term = terms[k]
            if acc is None:
                acc = term if sign(k) > 0 else -term
            else:
                acc = acc + term if sign(k) > 0 else acc - term
        return acc

    def weighted(groups):
        """sum_w w groups[w]: the first group taken as it is (weight 1) or times its weight,
        every further one by a multiply-add."""
        ws = sorted(groups)
        acc = groups[ws[0]] if ws[0] == 1 else groups[ws[0]] * float(ws[0])
        for w in ws[1:]:
            acc = fma(float(w), groups[w], acc)
        return acc

    by_v2 = {}
    for k in range(1, 19):
        vx, vy = REPS[k - 1]
        by_v2.setdefault(vx * vx + vy * vy, []).append(k)
    G = {w: group_sum(ks, P) for w, ks in by_v2.items()}
    R = f[0]
    for w in sorted(G):
        R = R + G[w]
    Ei = weighted(G)
    by_vx, by_vy = {}, {}
    for k in range(1, 19):
        vx, vy = REPS[k - 1]
        if vx:
            by_vx.setdefault(vx, []).append(k)          # vx >= 0 for the representatives
        if vy:
            by_vy.setdefault(abs(vy), []).append(k)
    Jx = weighted({w: group_sum(ks, Md) for w, ks in by_vx.items()})
    Jy = weighted({w: group_sum(ks, Md, sign=lambda k: 1 if REPS[k - 1][1] > 0 else -1)
                   for w, ks in by_vy.items()})
    # site scalars: 1/rho, c u, |u|^2, D T, t = T_s - 1, omega rho, c u_s
    inv_rho = 1.0 / R
    c2ir = C2 * inv_rho
    Ux0, Uy0 = Jx * c2ir, Jy * c2ir
    uu = fma(Ux0, Ux0, Uy0 * Uy0) * (1.0 / C2)
    TD = fma(Ei, c2ir, -uu)
    t = fma(TD, 1.0 / D, tshift)
    Rw = omega * R
    Ux, Uy = Ux0 + cgx, Uy0 + cgy
    # Hermite coefficients: C0 = a00 + a01 q + a02 q^2, C1 = a10 + a11 q, C2 = a20 + a21 q
    U = fma(Ux, Ux, Uy * Uy) * (1.0 / C2)
    tU, t2 = t * U, t * t
    a00 = fma(0.125, U * U, fma(-0.5, U, 1.0) - t) + (tU + t2)
    a01 = fma(-0.25, tU, 0.5 * t) - t2
    a02 = 0.125 * t2
    a10 = fma(-0.5, U, 1.0) - 2.0 * t
    a11 = 0.5 * t
    a20 = fma(-0.25, U, 0.5) - 1.5 * t
    a21 = 0.25 * t
    # per-shell Horner coefficients of omega rho w_s (C0 + C1 s + C2 s^2 + s^3/6 + s^4/24)
    K = [None] * 8
    K[0] = ((Rw * W_SHELL[0]) * a00, None, None, None, None)
    for s in range(1, 8):
        q = C2 * SHELL_V2[s]
        W = Rw * W_SHELL[s]
        K[s] = (W * fma(fma(a02, q, a01), q, a00), W * fma(a11, q, a10), W * fma(a21, q, a20),
                W * (1.0 / 6.0), W * (1.0 / 24.0))
    # multiples of c u_s for the integer velocity components 0..3
    X = [0.0, Ux, Ux + Ux, None]
    X[3] = X[2] + Ux
    Y = [0.0, Uy, Uy + Uy, None]
    Y[3] = Y[2] + Uy
    out = [None] * 37
    out[0] = fma(om1, f[0], K[0][0])
    for k in range(1, 19):
        vx, vy = REPS[k - 1]
        if vy == 0:
            s = X[vx]
        elif vx == 0:
            s = Y[vy] if vy > 0 else -Y[-vy]
        else:
            s = X[vx] + Y[vy] if vy > 0 else X[vx] - Y[-vy]
        K0, K1, K2, K3, K4 = K[shell_of_rep(k)]
        s2 = s * s
        E = fma(fma(K4, s2, K2), s2, K0)
        O = s * fma(K3, s2, K1)
        out[k] = fma(om1, f[k], E + O)
        out[k + 18] = fma(om1, f[k + 18], E - O)
    return out


def counted_site(fvals, tau, gx, gy):
    ctr = Counter()
    Num.ctr = ctr
    out = factored_collide([Num(v) for v in fvals], tau, gx, gy)
    Num.ctr = None
    return [Num.val(o) for o in out], ctr


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_counted_formulation_is_the_collision(seed):
    g = torch.Generator().manual_seed(seed)
    rho = 0.8 + 0.4 * torch.rand(1, 1, generator=g, dtype=torch.float64)
    u = 0.05 * (torch.rand(1, 1, 2, generator=g, dtype=torch.float64) - 0.5)
    T = 0.9 + 0.2 * torch.rand(1, 1, generator=g, dtype=torch.float64)
    f = M.equilibrium(rho, u, T) * (1.0 + 0.01 * torch.randn(37, 1, 1, generator=g, dtype=torch.float64))
    tau, gx, gy = 0.7 + 0.1 * seed, 1e-4 * seed, -1e-4
    want = OL.collide(f, OL.Params(1, 1, tau=tau, gx=gx, gy=gy))[:, 0, 0]
    got, _ = counted_site(f[:, 0, 0].tolist(), tau, gx, gy)
    err = max(abs(a - b) / abs(b) for a, b in zip(got, want.tolist()))
    assert err <= 1e-13, err


def test_bench_flop_constant_is_the_counted_total():
    _, ctr = counted_site([w for w in M.WEIGHTS.tolist()], 0.8, 0.0, -1e-4)
    # the count is the same for every input (no data-dependent branches)
    _, ctr2 = counted_site([1.1 * w for w in M.WEIGHTS.tolist()], 0.6, 2e-4, 1e-4)
    assert ctr.n == ctr2.n
    sys.path.insert(0, ROOT)
    import bench
    assert ctr.flops() == bench.FLOPS_PER_SITE_FP64, ctr.n
    assert (ctr.n["add"], ctr.n["mul"], ctr.n["fma"], ctr.n["div"]) == bench.FLOP_MIX_FP64
