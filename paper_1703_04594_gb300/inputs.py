"""Seeded synthetic Rayleigh-Taylor initial fields (shared by the product and the tests).

This module holds none of the lattice-Boltzmann arithmetic: it only builds the
macroscopic fields (rho, ux, uy, T) of the initial condition.  The populations are
then set to local equilibrium by the library (``lbm_init``) or by the CPU oracle.

Workload shape (the paper's application, Sec. 3: convective / Rayleigh-Taylor
turbulence on lattices like 2160 x 8192):

* interface y_c(x) = Ly/2 + sum_{k=1..8} a_k cos(2 pi k x / Lx + phi_k), with
  phi_k ~ U[0, 2 pi) and r_k ~ U[-1, 1] drawn from a Philox stream (numpy's
  ``Philox`` bit generator) seeded with ``seed``; a_k are the r_k rescaled so that
  max_x |sum_k| = 0.01 Ly.  The a_k are the parameters a gradient is taken against.
* temperature T = T_b + (T_t - T_b) (1 + tanh((y - y_c(x)) / w)) / 2, w = 2 sites
  (hot below, cold above: unstable under gravity in -y).
* pressure from hydrostatic balance dp/dy = -g rho = -g p / T:
  p(x, y) = exp(-g int_{Ly/2}^{y} dy' / T(x, y')), trapezoid rule over the rows,
  p = 1 at row Ly/2; density rho = p / T; velocity zero.

Fields are float64 tensors of shape [Lx, Ly] (y contiguous).  ``rt_fields`` is
written with torch operations so that it is differentiable in ``a`` and ``tau``-free.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

N_MODES = 8
AMPLITUDE_FRACTION = 0.01
INTERFACE_WIDTH = 2.0


@dataclass
class RTModes:
    a: torch.Tensor      # [8] float64 amplitudes (lattice units)
    phi: torch.Tensor    # [8] float64 phases


def rt_modes(lx: int, ly: int, seed: int, n_modes: int = N_MODES) -> RTModes:
    """Draw the interface modes for one lattice (Philox stream, ``seed``)."""
    rng = np.random.Generator(np.random.Philox(seed))
    phi = rng.uniform(0.0, 2.0 * math.pi, n_modes)
    r = rng.uniform(-1.0, 1.0, n_modes)
    x = np.arange(lx, dtype=np.float64)
    k = np.arange(1, n_modes + 1, dtype=np.float64)
    shape = (r[None, :] * np.cos(2.0 * math.pi * k[None, :] * x[:, None] / lx + phi[None, :])).sum(axis=1)
    scale = AMPLITUDE_FRACTION * ly / np.abs(shape).max()
    return RTModes(a=torch.tensor(r * scale, dtype=torch.float64),
                   phi=torch.tensor(phi, dtype=torch.float64))


def interface(lx: int, ly: int, modes: RTModes, device=None) -> torch.Tensor:
    """y_c(x) for x = 0..Lx-1 (on ``device``, default the modes' device)."""
    device = device if device is not None else modes.a.device
    x = torch.arange(lx, dtype=torch.float64, device=device)
    k = torch.arange(1, modes.a.numel() + 1, dtype=torch.float64, device=device)
    arg = 2.0 * math.pi * k[None, :] * x[:, None] / lx + modes.phi.to(device)[None, :]
    return ly / 2.0 + (modes.a.to(device)[None, :] * torch.cos(arg)).sum(dim=1)


def rt_fields(lx: int, ly: int, modes: RTModes, t_bottom: float = 1.15, t_top: float = 0.85,
              g: float = 1e-4, width: float = INTERFACE_WIDTH, device=None):
    """(rho, ux, uy, T) of the hydrostatic Rayleigh-Taylor initial state, each [Lx, Ly].

    ``g`` is the magnitude of gravity, which acts in -y.  The fields are built on ``device``
    (default: the CPU, or the modes' device); the same operations run on any device.
    """
    yc = interface(lx, ly, modes, device)                           # [Lx]
    device = yc.device
    y = torch.arange(ly, dtype=torch.float64, device=device)
    T = t_bottom + (t_top - t_bottom) * 0.5 * (1.0 + torch.tanh((y[None, :] - yc[:, None]) / width))
    inv_t = 1.0 / T
    # trapezoid cumulative integral of 1/T from row 0, then re-referenced to row Ly/2
    seg = 0.5 * (inv_t[:, 1:] + inv_t[:, :-1])                      # [Lx, Ly-1]
    cum = torch.cat([torch.zeros(lx, 1, dtype=torch.float64, device=device), torch.cumsum(seg, dim=1)], dim=1)
    ref = ly // 2
    integral = cum - cum[:, ref:ref + 1]
    p = torch.exp(-g * integral)
    rho = p / T
    zero = torch.zeros_like(T)
    return rho, zero.clone(), zero.clone(), T


def rt_state(lx: int, ly: int, seed: int, t_bottom: float = 1.15, t_top: float = 0.85, g: float = 1e-4,
             device=None):
    """Convenience: modes drawn from ``seed`` and the resulting fields (on ``device``)."""
    modes = rt_modes(lx, ly, seed)
    return rt_fields(lx, ly, modes, t_bottom=t_bottom, t_top=t_top, g=g, device=device)


def batch_workload(seed: int = 4, n: int = 256, sizes=tuple(range(128, 1025, 64)),
                   tau_range=(0.6, 1.0)):
    """Many independent Rayleigh-Taylor lattices of uneven sizes: for each lattice j,
    Lx drawn from ``sizes`` (128, 192, ..., 1024), Ly = 2 Lx, tau ~ U[tau_range], and its
    own interface seed.  Returns a list of (lx, ly, tau, interface_seed)."""
    rng = np.random.Generator(np.random.Philox(seed))
    lx = rng.choice(np.asarray(sizes), size=n)
    tau = rng.uniform(tau_range[0], tau_range[1], size=n)
    return [(int(a), int(2 * a), float(t), int(seed * 100000 + j)) for j, (a, t) in enumerate(zip(lx, tau))]
