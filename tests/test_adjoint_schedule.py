"""The checkpoint scheduler of paper_1703_04594_gb300/adjoint.py on the CPU.

The scheduler (forward pass with a checkpoint every ``every`` steps, backward pass that
recomputes each segment from its checkpoint, newest first, and walks the adjoint back
through it) is host logic.  Here it drives a stand-in for the library: a small linear
model on CPU tensors, f^{n+1} = A(tau) f^n with A = (1 - 1/tau) I + B / tau, f^0 = M x
for the four input fields x, and E = |f^N|^2 / 2, whose adjoint calls are the exact
transposes.  The gradient it returns must equal torch autograd through the same model for
every schedule: every = 1, every dividing N, not dividing N, every >= N.
"""
import dataclasses
import types

import pytest
import torch

from paper_1703_04594_gb300 import adjoint as A

N_STATE = 6


@dataclasses.dataclass(frozen=True)
class FakeParams:
    tau: float = 0.8
    precision: int = 0


def model(seed=0):
    g = torch.Generator().manual_seed(seed)
    B = 0.3 * torch.randn(N_STATE, N_STATE, generator=g, dtype=torch.float64)
    M = torch.randn(N_STATE, 4, generator=g, dtype=torch.float64)
    return B, M


def fake_library(B, M):
    """The library entry points the scheduler calls, for the linear model."""
    def a_of(tau):
        return (1.0 - 1.0 / tau) * torch.eye(N_STATE, dtype=torch.float64) + B / tau

    def da_dtau(tau):
        return (torch.eye(N_STATE, dtype=torch.float64) - B) / tau ** 2

    lib = types.SimpleNamespace(FP64=0, FP64_FIXED=2)
    lib.empty_state = lambda p, device=None: torch.empty(N_STATE, dtype=torch.float64)
    lib.init = lambda p, rho, ux, uy, T, out: out.copy_(M @ torch.stack([rho, ux, uy, T]))
    lib.step = lambda p, src, dst: dst.copy_(a_of(p.tau) @ src)
    lib.kinetic_energy = lambda p, f: 0.5 * (f * f).sum()
    lib.kinetic_energy_grad = lambda p, f, lam: lam.copy_(f)
    lib.adjoint_work = lambda p, device=None: None

    def adjoint_step(p, f_n, lam_next, lam_n, dtau, work):
        lam_n.copy_(a_of(p.tau).T @ lam_next)
        dtau += lam_next @ (da_dtau(p.tau) @ f_n)
    lib.adjoint_step = adjoint_step
    lib.init_adjoint = lambda p, rho, ux, uy, T, lam0: tuple(M.T @ lam0)
    return lib, a_of


@pytest.mark.parametrize("n_steps,every", [(1, 1), (7, 1), (12, 3), (13, 3), (13, 5), (10, 10), (9, 20), (30, None)])
def test_checkpointed_gradient_equals_autograd(monkeypatch, n_steps, every):
    B, M = model()
    lib, a_of = fake_library(B, M)
    monkeypatch.setattr(A, "lbm", lib)
    x = torch.tensor([1.1, 0.02, -0.03, 0.95], dtype=torch.float64)
    tau0 = 0.8

    # the scheduler's gradient
    xs = [x[k].clone().requires_grad_(True) for k in range(4)]
    tau = torch.tensor(tau0, dtype=torch.float64, requires_grad=True)
    e = A.kinetic_energy_after(*xs, tau, FakeParams(), n_steps, every)
    e.backward()
    got = torch.stack([t.grad for t in xs] + [tau.grad])

    # torch autograd through the same model
    xr = x.clone().requires_grad_(True)
    taur = torch.tensor(tau0, dtype=torch.float64, requires_grad=True)
    f = M @ xr
    a = (1.0 - 1.0 / taur) * torch.eye(N_STATE, dtype=torch.float64) + B / taur
    for _ in range(n_steps):
        f = a @ f
    er = 0.5 * (f * f).sum()
    er.backward()
    want = torch.cat([xr.grad, taur.grad.reshape(1)])

    assert abs(float(e.detach()) - float(er.detach())) <= 1e-12 * abs(float(er.detach()))
    torch.testing.assert_close(got, want, rtol=1e-11, atol=1e-13)


def test_default_interval_is_the_square_root():
    assert [A.default_every(n) for n in (1, 4, 5, 500)] == [1, 2, 3, 23]


@pytest.mark.parametrize("n_steps,every", [(13, 5), (12, 1), (9, 20)])
def test_recomputation_precision_and_step_count(monkeypatch, n_steps, every):
    """Forward steps run in the precision of the params, the backward pass's recomputed
    steps in ``recompute_precision``; the forward pass takes n_steps steps and the backward
    pass recomputes every state that is neither a checkpoint nor after the newest
    checkpoint (those the forward pass keeps); none when every = 1."""
    B, M = model()
    lib, _ = fake_library(B, M)
    calls = []
    step = lib.step
    lib.step = lambda p, src, dst: (calls.append(p.precision), step(p, src, dst))[1]
    monkeypatch.setattr(A, "lbm", lib)
    xs = [torch.tensor(v, dtype=torch.float64, requires_grad=True) for v in (1.1, 0.02, -0.03, 0.95)]
    e = A.kinetic_energy_after(*xs, torch.tensor(0.8, dtype=torch.float64), FakeParams(), n_steps, every,
                               recompute_precision=lib.FP64_FIXED)
    assert calls == [lib.FP64] * n_steps
    e.backward()
    n_checkpoints = len(range(0, n_steps, every))
    newest = ((n_steps - 1) // every) * every
    n_tail = n_steps - newest - 1
    assert calls[n_steps:] == [lib.FP64_FIXED] * (n_steps - n_checkpoints - n_tail)
