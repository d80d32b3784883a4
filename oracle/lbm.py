"""Plain float64 CPU transcription of one D2Q37 time step: propagate -> bc -> collide.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

State layout: a float64 tensor ``f[i, x, y]`` of shape [37, Lx, Ly] holding the
post-collision populations of every fluid site (no padding, no ghost rows).  x is
periodic; y is bounded by thermal walls at y = 0 (bottom) and y = Ly - 1 (top), or
periodic when ``bc == "periodic_y"`` (a test-only mode in which every collision
invariant holds globally).

Readings of points the paper leaves open (each one is stated where it is used):

* units: moments use the scaled molecular velocities xi_i = c v_i; hops use the
  integer vectors v_i; velocity, temperature and gravity are in xi units, T0 = 1.
* gravity: the equilibrium is evaluated at the shifted velocity u + tau g and
  temperature T + tau (1 - tau) |g|^2 / D, which makes one collision change the
  momentum by exactly rho g and leave rho and T unchanged.
* walls: a population pulled from outside the fluid (y_s < 0 or y_s >= Ly) takes the
  wall equilibrium f_i^eq(rho_w, 0, T_wall), where rho_w is the density, at the
  start of the step, of the fluid site next to the wall in the source column x_s.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import d2q37 as M


@dataclass(frozen=True)
class Params:
    """Physical parameters of the problem (Sec. 3: BGK relaxation time, gravity in
    the vertical direction, and the thermal walls of the convective cell)."""
    lx: int
    ly: int
    tau: float = 0.8
    gx: float = 0.0
    gy: float = -1e-4
    t_bottom: float = 1.15
    t_top: float = 0.85
    bc: str = "walls"          # "walls" or "periodic_y"


def moments(f):
    """Density, velocity and temperature of every site (Sec. 3, eq. ``macro``):
    rho = sum_i f_i;  rho u = sum_i xi_i f_i;  D rho T = sum_i |xi_i - u|^2 f_i.

    f: [37, ...].  Returns rho [...], u [..., 2], T [...].
    """
    rho = f.sum(dim=0)
    mom = torch.stack([(M.XI[:, a].reshape(-1, *([1] * (f.dim() - 1))) * f).sum(dim=0)
                       for a in range(M.D)], dim=-1)
    u = mom / rho.unsqueeze(-1)
    dev2 = torch.zeros_like(f)
    for a in range(M.D):
        dev2 = dev2 + (M.XI[:, a].reshape(-1, *([1] * (f.dim() - 1))) - u[..., a].unsqueeze(0)) ** 2
    T = (dev2 * f).sum(dim=0) / (M.D * rho)
    return rho, u, T


def gravity_shift(u, T, p: Params):
    """Velocity and temperature at which the equilibrium is evaluated when gravity
    acts: u + tau g and T + tau (1 - tau) |g|^2 / D (reading stated in the module
    docstring; the paper's continuum equations put the force -rho g in the
    vertical momentum equation, Sec. 3)."""
    g = torch.tensor([p.gx, p.gy], dtype=torch.float64)
    u_s = u + p.tau * g
    T_s = T + p.tau * (1.0 - p.tau) * float((g * g).sum()) / M.D
    return u_s, T_s


def collide(f_tilde, p: Params):
    """BGK collision (Sec. 3, eq. ``lbequation`` with dt = 1):
    f_i' = f_i - (1/tau) (f_i - f_i^eq), with the equilibrium taken at the moments
    of f (eq. ``macro``) shifted by gravity."""
    rho, u, T = moments(f_tilde)
    u_s, T_s = gravity_shift(u, T, p)
    feq = M.equilibrium(rho, u_s, T_s)
    return f_tilde - (f_tilde - feq) / p.tau


def propagate(f, p: Params):
    """Pull-scheme streaming (Sec. 3, eq. ``master2``; Sec. 4 ``propagate``):
    f~_i(x, y) = f_i(x - vx_i mod Lx, y - vy_i).

    With walls, an entry whose source row lies outside the fluid holds a placeholder
    (the clamped row) that ``bc`` overwrites.  With ``periodic_y`` the source row
    wraps modulo Ly."""
    q, lx, ly = f.shape
    out = torch.empty_like(f)
    xs_all = torch.arange(lx)
    ys_all = torch.arange(ly)
    for i in range(q):
        vx, vy = M.VELOCITIES[i]
        xs = (xs_all - vx) % lx
        ys = ys_all - vy
        if p.bc == "periodic_y":
            ys = ys % ly
        else:
            ys = ys.clamp(0, ly - 1)
        out[i] = f[i][xs][:, ys]
    return out


def bc(f_tilde, f_prev, p: Params):
    """Thermal walls at the three lowest and highest rows (Sec. 5: ``bc`` acts on the
    three uppermost and lowermost rows after ``propagate``).  Each population whose
    source lies below y = 0 becomes f_i^eq(rho(x_s, 0), 0, T_bottom); above
    y = Ly - 1 it becomes f_i^eq(rho(x_s, Ly - 1), 0, T_top), where rho is the density
    of the state ``f_prev`` at the start of the step and x_s = x - vx_i mod Lx."""
    if p.bc == "periodic_y":
        return f_tilde
    q, lx, ly = f_tilde.shape
    out = f_tilde.clone()
    rho_bottom = f_prev[:, :, 0].sum(dim=0)          # [Lx]
    rho_top = f_prev[:, :, ly - 1].sum(dim=0)        # [Lx]
    zero_u = torch.zeros(lx, 2, dtype=torch.float64)
    feq_bottom = M.equilibrium(rho_bottom, zero_u, torch.full((lx,), p.t_bottom, dtype=torch.float64))
    feq_top = M.equilibrium(rho_top, zero_u, torch.full((lx,), p.t_top, dtype=torch.float64))
    xs_all = torch.arange(lx)
    for i in range(q):
        vx, vy = M.VELOCITIES[i]
        xs = (xs_all - vx) % lx
        for y in range(ly):
            if 0 <= y - vy < ly:
                continue
            if y - vy < 0:
                out[i, :, y] = feq_bottom[i][xs]
            else:
                out[i, :, y] = feq_top[i][xs]
    return out


def step(f, p: Params):
    """One time step in the paper's kernel order (Sec. 5): propagate -> bc -> collide."""
    f_tilde = propagate(f, p)
    f_tilde = bc(f_tilde, f, p)
    return collide(f_tilde, p)


def run(f, p: Params, n_steps: int):
    for _ in range(n_steps):
        f = step(f, p)
    return f


def init_equilibrium(rho, ux, uy, T):
    """Initial populations at local equilibrium with the given fields (Sec. 3: an LB
    run starts from an assignment of the populations matching the initial
    condition).  rho, ux, uy, T: [Lx, Ly].  Returns [37, Lx, Ly]."""
    return M.equilibrium(rho, torch.stack([ux, uy], dim=-1), T)


def fields(f):
    """(rho, ux, uy, T), each [Lx, Ly], from the populations (eq. ``macro``)."""
    rho, u, T = moments(f)
    return rho, u[..., 0], u[..., 1], T


def kinetic_energy(f):
    """Total kinetic energy sum over fluid sites of rho |u|^2 / 2, with rho and u
    the raw moments of eq. ``macro``."""
    rho, u, _ = moments(f)
    return 0.5 * (rho * (u * u).sum(dim=-1)).sum()
