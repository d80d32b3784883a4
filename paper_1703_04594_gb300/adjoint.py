"""Gradients through many FP64 steps: checkpointed reverse mode over the C-ABI adjoint.

``kinetic_energy_after(rho, ux, uy, T, tau, params, n_steps)`` returns the total kinetic
energy after ``n_steps`` fused steps from the equilibrium state of the given fields, as a
differentiable torch scalar: its backward pass gives dE/d(rho, ux, uy, T) and dE/dtau from
the library's hand-written adjoint kernels (``lbm_adjoint_step``, ``lbm_init_adjoint``,
``lbm_kinetic_energy_grad``).  Chain it with fields built by differentiable torch code (for
example ``inputs.rt_fields`` with ``modes.a.requires_grad_()``) to get gradients with
respect to interface-mode amplitudes.

The forward steps run in the precision of ``params``: FP64, or FP64 with the fixed-point
relaxation (LBM_FP64_FIXED, the same states within rounding), so the energy is that of the
plain forward run bit for bit; the recomputation runs in ``recompute_precision``, by
default the fixed-point relaxation (2.8x faster on GB300 than the float64 step): the
recomputed states are only the points the adjoint linearises at, and they agree with the
forward pass's to float64 rounding (the gradient agrees with a float64 recomputation's
to ~1e-12).  ``recompute_precision=LBM_FP64`` recomputes with the float64 step; the
adjoint steps are the FP64 ones either way.

Memory: the forward pass keeps a checkpoint every ``every`` steps (default ceil(sqrt(N)));
the backward pass recomputes each segment's states from its checkpoint, newest segment
first, and walks the adjoint back through it.  On a GPU the recomputation of the next
(earlier) segment runs on a second stream while the adjoint steps of the current one run,
so the two kernels share the SMs.  The states after the newest checkpoint are kept from
the forward pass, so the newest segment is not recomputed.  Peak: ceil(N/every) + 2 every
+ 2 states.  With
``every=1`` every state is kept (N + 1 states: 500 steps of 512 x 1024 hold 78 GB of HBM)
and nothing is recomputed.
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
    def forward(ctx, rho, ux, uy, T, tau, params, n_steps, every, recompute_precision):
        p = dataclasses.replace(params, tau=float(tau))
        if p.precision not in (lbm.FP64, lbm.FP64_FIXED) or recompute_precision not in (lbm.FP64, lbm.FP64_FIXED):
            raise ValueError("the adjoint runs on FP64 states")
        fields = [t.detach().contiguous() for t in (rho, ux, uy, T)]
        dev = rho.device
        a = lbm.empty_state(p, dev)
        lbm.init(p, *fields, a)
        # each checkpoint is the output buffer of its step (no copy); so are the states after
        # the newest checkpoint (the tail), which the backward pass needs first and so need
        # not recompute; the other steps alternate between two working buffers
        last = ((n_steps - 1) // every) * every if n_steps > 0 else 0
        tail = [lbm.empty_state(p, dev) for _ in range(max(n_steps - last - 1, 0))]
        checkpoints = {0: a}
        kept = {id(a)} | {id(t) for t in tail}
        free = [lbm.empty_state(p, dev)]
        cur = a
        for n in range(n_steps):
            m = n + 1                                      # the state this step produces
            keep = m % every == 0 and m < n_steps
            if last < m < n_steps:
                out = tail[m - last - 1]
            else:
                out = lbm.empty_state(p, dev) if keep or not free else free.pop()
            lbm.step(p, cur, out)
            if id(cur) not in kept:
                free.append(cur)
            cur = out
            if keep:
                checkpoints[m] = out
                kept.add(id(out))
        del free
        energy = lbm.kinetic_energy(p, cur)
        ctx.tail = tail
        ctx.p, ctx.n_steps, ctx.every = p, n_steps, every
        ctx.p_recompute = dataclasses.replace(p, precision=recompute_precision)
        ctx.checkpoints, ctx.final, ctx.fields = checkpoints, cur, fields
        ctx.tau_shape = tau.shape if torch.is_tensor(tau) else None
        ctx.tau_device = tau.device if torch.is_tensor(tau) else None
        return energy

    @staticmethod
    def backward(ctx, grad_e):
        dev = ctx.final.device
        if dev.type != "cuda":
            return _KineticEnergyAfter._backward(ctx, grad_e, dev, None, None)
        # the adjoint steps run on a stream of higher priority than the recomputation's:
        # while an adjoint launch has blocks waiting they go first, and the recomputed
        # steps fill the SMs its last wave leaves idle
        caller = torch.cuda.current_stream(dev)
        adj = torch.cuda.Stream(dev, priority=-1)
        side = torch.cuda.Stream(dev)
        adj.wait_stream(caller)                            # the checkpoints are ready
        side.wait_stream(caller)
        with torch.cuda.stream(adj):
            out = _KineticEnergyAfter._backward(ctx, grad_e, dev, adj, side)
        caller.wait_stream(adj)
        for t in out[:4]:
            t.record_stream(caller)
        return out

    @staticmethod
    def _backward(ctx, grad_e, dev, main, side):
        """The backward pass; `main` (the current stream) takes the adjoint steps, `side` the
        recomputation (both None on the CPU)."""
        p, n_steps, every = ctx.p, ctx.n_steps, ctx.every
        pa = dataclasses.replace(p, precision=lbm.FP64)  # the adjoint kernels (same states)
        cuda = main is not None
        lam = lbm.empty_state(pa, dev)
        lbm.kinetic_energy_grad(pa, ctx.final, lam)
        lam.mul_(grad_e.to(dev))
        lam_other = lbm.empty_state(pa, dev)
        dtau = torch.zeros((), dtype=torch.float64, device=dev)
        work = lbm.adjoint_work(pa, dev)
        order = sorted(ctx.checkpoints, reverse=True)      # newest segment first
        # two pools of every - 1 recomputed states, used by alternate segments: no allocation
        # per step, and a segment is recomputed into the pool the adjoint finished with
        pr = ctx.p_recompute
        # pool 0 starts as the forward pass's tail: the newest segment is not recomputed
        tail, ctx.tail = ctx.tail, None
        pools = [tail + [lbm.empty_state(p, dev) for _ in range(max(every - 1 - len(tail), 0))],
                 [lbm.empty_state(p, dev) for _ in range(max(every - 1, 0))]]
        if cuda:
            # buffers used on a stream other than their allocating one: the allocator must not
            # reuse them before that stream's work on them is done
            for t in list(ctx.checkpoints.values()) + pools[0] + pools[1]:
                t.record_stream(main)
                t.record_stream(side)
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
                    lbm.step(pr, states[-1], nxt)
                    states.append(nxt)
                done = None
                if cuda:
                    done = torch.cuda.Event()
                    done.record(side)
            return k, end, states, done

        k0 = order[0]
        end0 = min(k0 + every, n_steps)
        pending = (k0, end0, [ctx.checkpoints[k0]] + tail[: end0 - k0 - 1], None)
        for idx in range(len(order)):
            k, end, states, done = pending
            if cuda and done is not None:
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
        return g[0], g[1], g[2], g[3], g_tau, None, None, None, None


def kinetic_energy_after(rho, ux, uy, T, tau, params: lbm.Params, n_steps: int, every: int | None = None,
                         recompute_precision: int | None = None):
    """Differentiable total kinetic energy after n_steps FP64 steps (see module docstring).
    ``tau`` may be a 0-d float64 tensor with requires_grad for dE/dtau; ``every`` is the
    checkpoint interval (1 keeps every state); ``recompute_precision`` (LBM_FP64_FIXED,
    the default, or LBM_FP64) the precision of the backward pass's recomputed steps."""
    if every is None:
        every = default_every(n_steps)
    if recompute_precision is None:
        recompute_precision = lbm.FP64_FIXED
    if not torch.is_tensor(tau):
        tau = torch.tensor(float(tau), dtype=torch.float64)
    return _KineticEnergyAfter.apply(rho, ux, uy, T, tau, params, int(n_steps), int(every), int(recompute_precision))
