"""The oracle's reference gradient (reverse-mode autograd through the plain float64
oracle) is pinned against central finite differences of the oracle itself."""
import torch

from oracle import lbm as OL
from paper_1703_04594_gb300 import inputs as I


def energy(a, phi, tau, lx=8, ly=16, steps=4):
    modes = I.RTModes(a=a, phi=phi)
    fields = I.rt_fields(lx, ly, modes, g=1e-3)
    f = OL.init_equilibrium(*fields)
    p = OL.Params(lx, ly, tau=tau, gx=2e-4, gy=-1e-3)
    return OL.kinetic_energy(OL.run(f, p, steps))


def test_oracle_autograd_matches_central_differences():
    m = I.rt_modes(8, 16, seed=5)
    a = m.a.clone().requires_grad_(True)
    tau = torch.tensor(0.75, dtype=torch.float64, requires_grad=True)
    e = energy(a, m.phi, tau)
    e.backward()
    h = 1e-5
    for k in (0, 3, 7):
        ap, am = m.a.clone(), m.a.clone()
        ap[k] += h
        am[k] -= h
        fd = (energy(ap, m.phi, 0.75) - energy(am, m.phi, 0.75)) / (2 * h)
        assert abs(float(fd) - float(a.grad[k])) <= 1e-6 * float(a.grad.abs().max()), k
    fd_tau = (energy(m.a, m.phi, 0.75 + h) - energy(m.a, m.phi, 0.75 - h)) / (2 * h)
    assert abs(float(fd_tau) - float(tau.grad)) <= 1e-6 * abs(float(tau.grad))
