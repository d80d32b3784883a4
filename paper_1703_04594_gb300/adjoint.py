"""Gradients through many FP64 steps: checkpointed reverse mode over the C-ABI adjoint.

``kinetic_energy_after(rho, ux, uy, T, tau, params, n_steps)`` returns the total kinetic
energy after ``n_steps`` fused steps from the equilibrium state of the given fields, as a
differentiable torch scalar: its backward pass gives dE/d(rho, ux, uy, T) and dE/dtau from
the library's hand-written adjoint kernels (``lbm_adjoint_step``, ``lbm_init_adjoint``,
``lbm_kinetic_energy_grad``).  Chain it with fields built by differentiable torch code (for
example ``inputs.rt_fields`` with ``modes.a.requires_grad_()``) to get gradients with
respect to interface-mode amplitudes.

The forward steps (and their recomputation) run in the precision of ``params``: FP64, or
FP64 with the fixed-point relaxation (LBM_FP64_FIXED, the same states within rounding);
the adjoint steps are the FP64 ones either way.

Memory: the forward pass keeps a checkpoint every ``every`` steps (default ceil(sqrt(N)));
the backward pass recomputes each segment's states from its checkpoint, newest segment
first, and walks the adjoint back through it.  On a GPU the recomputation of the next
(earlier) segment runs on a second stream while the adjoint steps of the current one run,
so the two kernels share the SMs.  Peak: ceil(N/every) + 2 every + 3 states.
"""
from __future__ import annotations

import contextlib
import dataclasses
import math

import torch

from . import lbm


def default_every(n_steps: int) -> int:
    return max(1, math.ceil(math.sqrt(n_steps)))


class _KineticEnergyAfter(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, ux, uy, T, tau, params, n_steps, every):
        p = dataclasses.replace(params, tau=float(tau))
        if p.precision not in (lbm.FP64, lbm.FP64_FIXED):
            raise ValueError("the adjoint runs on FP64 states")
        fields = [t.detach().contiguous() for t in (rho, ux, uy, T)]
        a, b = lbm.empty_state(p, rho.device), lbm.empty_state(p, rho.device)
        lbm.init(p, *fields, a)
        checkpoints = {0: a.clone()}
        cur, nxt = a, b
        for n in range(n_steps):
            lbm.step(p, cur, nxt)
            cur, nxt = nxt, cur
            if (n + 1) % every == 0 and n + 1 < n_steps:
                checkpoints[n + 1] = cur.clone()
        energy = lbm.kinetic_energy(p, cur)
        ctx.p, ctx.n_steps, ctx.every = p, n_steps, every
        ctx.checkpoints, ctx.final, ctx.fields = checkpoints, cur.clone(), fields
        ctx.tau_shape = tau.shape if torch.is_tensor(tau) else None
        ctx.tau_device = tau.device if torch.is_tensor(tau) else None
        return energy

    @staticmethod
    def backward(ctx, grad_e):
        p, n_steps, every = ctx.p, ctx.n_steps, ctx.every
        pa = dataclasses.replace(p, precision=lbm.FP64)  # the adjoint kernels (same states)
        dev = ctx.final.device
        lam = lbm.empty_state(pa, dev)
        lbm.kinetic_energy_grad(pa, ctx.final, lam)
        lam.mul_(grad_e.to(dev))
        lam_other = lbm.empty_state(pa, dev)
        dtau = torch.zeros((), dtype=torch.float64, device=dev)
        work = lbm.adjoint_work(pa, dev)
        order = sorted(ctx.checkpoints, reverse=True)      # newest segment first
        cuda = dev.type == "cuda"
        main = torch.cuda.current_stream(dev) if cuda else None
        side = torch.cuda.Stream(dev) if cuda else None
        if cuda:
            side.wait_stream(main)                         # the checkpoints are ready
        # two pools of every - 1 recomputed states, used by alternate segments: no allocation
        # per step, and a segment is recomputed into the pool the adjoint finished with
        pools = [[lbm.empty_state(p, dev) for _ in range(max(every - 1, 0))] for _ in range(2)]
        released = [None, None]                            # main-stream events: pool free again

        def recompute(k, pool):
            """f^k .. f^{end-1} of the segment starting at checkpoint k (on the side stream)."""
            end = min(k + every, n_steps)
            with torch.cuda.stream(side) if cuda else contextlib.nullcontext():
                if cuda and released[pool] is not None:
                    side.wait_event(released[pool])
                states = [ctx.checkpoints[k]]
                for j in range(k, end - 1):
                    nxt = pools[pool][j - k]
                    lbm.step(p, states[-1], nxt)
                    states.append(nxt)
                done = None
                if cuda:
                    done = torch.cuda.Event()
                    done.record(side)
            return k, end, states, done

        pending = recompute(order[0], 0)
        for idx in range(len(order)):
            k, end, states, done = pending
            if cuda:
                main.wait_event(done)
            if idx + 1 < len(order):
                pending = recompute(order[idx + 1], (idx + 1) % 2)   # overlaps the adjoint steps below
            for n in reversed(range(k, end)):
                lbm.adjoint_step(pa, states[n - k], lam, lam_other, dtau, work)
                lam, lam_other = lam_other, lam
            if cuda:
                released[idx % 2] = torch.cuda.Event()
                released[idx % 2].record(main)
            del states
        del pools
        g = lbm.init_adjoint(pa, *ctx.fields, lam)
        g_tau = None
        if ctx.tau_shape is not None:
            g_tau = dtau.to(ctx.tau_device).reshape(ctx.tau_shape)
        return g[0], g[1], g[2], g[3], g_tau, None, None, None


def kinetic_energy_after(rho, ux, uy, T, tau, params: lbm.Params, n_steps: int, every: int | None = None):
    """Differentiable total kinetic energy after n_steps FP64 steps (see module docstring).
    ``tau`` may be a 0-d float64 tensor with requires_grad for dE/dtau."""
    if every is None:
        every = default_every(n_steps)
    if not torch.is_tensor(tau):
        tau = torch.tensor(float(tau), dtype=torch.float64)
    return _KineticEnergyAfter.apply(rho, ux, uy, T, tau, params, int(n_steps), int(every))
