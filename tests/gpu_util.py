"""Helpers shared by the GPU parity tests: build inputs, move states between the
library's padded device layout and the oracle's [37, lx, ly] CPU layout, and measure
errors the way the parity bar is stated (max over elements of |a - b| / |b|)."""
import os

import pytest
import torch

from oracle import lbm as OL
from paper_1703_04594_gb300 import inputs as I
from paper_1703_04594_gb300 import lbm

_built = False


def ensure_built():
    global _built
    if not _built:
        if not os.path.exists(lbm.LIB_PATH):
            from paper_1703_04594_gb300 import build
            build.build()
        _built = True


def require_gpu():
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected on a machine without CUDA")
    ensure_built()


def oracle_params(p: lbm.Params) -> OL.Params:
    return OL.Params(p.lx, p.ly, tau=p.tau, gx=p.gx, gy=p.gy, t_bottom=p.t_bottom, t_top=p.t_top,
                     bc="periodic_y" if p.bc == lbm.BC_PERIODIC_Y else "walls")


def rt_fields(p: lbm.Params, seed: int):
    return I.rt_state(p.lx, p.ly, seed, t_bottom=p.t_bottom, t_top=p.t_top, g=abs(p.gy))


def device_init(p: lbm.Params, fields):
    dev = [t.contiguous().cuda() for t in fields]
    f = lbm.empty_state(p)
    f.fill_(float("nan"))
    lbm.init(p, *dev, f)
    return f


def to_host(p: lbm.Params, f_dev) -> torch.Tensor:
    """[37, lx, pitch] device state -> [37, lx, ly] float64 CPU."""
    return f_dev[:, :, : p.ly].double().cpu()


def rel_err(a, b):
    return float(((a - b).abs() / b.abs()).max())


def field_errors(a, b):
    """Per-field errors of fields a = (rho, ux, uy, T) against reference b: max and RMS of
    |a - b| / |b| for rho and T; for the velocity (near zero at the start) the max and
    RMS of |u_a - u_b| divided by the RMS of |u_b|."""
    out = {}
    for name, x, y in (("rho", a[0], b[0]), ("T", a[3], b[3])):
        r = ((x - y).abs() / y.abs()).double()
        out[name + "_max"] = float(r.max())
        out[name + "_rms"] = float(torch.sqrt((r * r).mean()))
    du = torch.sqrt((a[1] - b[1]) ** 2 + (a[2] - b[2]) ** 2).double()
    ub = torch.sqrt(b[1] ** 2 + b[2] ** 2).double()
    scale = float(torch.sqrt((ub * ub).mean()))
    out["u_max"] = float(du.max()) / scale
    out["u_rms"] = float(torch.sqrt((du * du).mean())) / scale
    # against the model's velocity scale, the reference sound speed sqrt(T0) = 1 (xi units)
    out["u_max_cs"] = float(du.max())
    return out
