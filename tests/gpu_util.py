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
