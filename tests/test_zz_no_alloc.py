"""lbm_kinetic_energy_noalloc: the kinetic energy for callers that cannot allocate device
memory while they run (their memory is reserved up front, or their stepping loop must
not call cudaMalloc, which can synchronise the device).  It must give the same result as
lbm_kinetic_energy, which takes caller scratch, on consecutive calls that share the
library's fixed scratch array, and reject lattices that do not fit that array.

This file is collected last on purpose, and runs the same alone or after the rest.
"""
import ctypes

import pytest
import torch

from paper_1703_04594_gb300 import lbm
from tests.gpu_util import device_init, require_gpu, rt_fields

pytestmark = pytest.mark.gpu

KE_TOL = 1e-12   # relative, as the other kinetic-energy checks; the kernels are the same


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def evolved(p, seed, steps=3):
    f = device_init(p, rt_fields(p, seed))
    return lbm.run(p, f, lbm.empty_state(p), steps)


def test_noalloc_matches_scratch_version_on_two_calls_in_a_row():
    big = lbm.Params(256, 512)                      # 16 x 64 = 1024 tiles
    small = lbm.Params(64, 96, precision=lbm.FP32_SHIFTED)   # 3 x 16 = 48 tiles
    f_big, f_small = evolved(big, seed=11), evolved(small, seed=12)
    want_big = float(lbm.kinetic_energy(big, f_big))
    want_small = float(lbm.kinetic_energy(small, f_small))
    # two calls in a row through the C-ABI; the second covers fewer tiles than the first
    # left behind in the shared array
    got_big = float(lbm.kinetic_energy_noalloc(big, f_big))
    got_small = float(lbm.kinetic_energy_noalloc(small, f_small))
    torch.cuda.synchronize()
    assert want_big > 0 and want_small > 0
    assert abs(got_big - want_big) <= KE_TOL * want_big
    assert abs(got_small - want_small) <= KE_TOL * want_small


def test_noalloc_rejects_lattices_beyond_its_scratch():
    p = lbm.Params(4100, 8192)                      # 256 x 1025 tiles > LBM_NOALLOC_MAX_TILES
    tiles = ((p.ly + 31) // 32) * ((p.lx + 3) // 4)
    assert tiles > lbm.NOALLOC_MAX_TILES
    dummy = torch.empty(64, dtype=torch.float64, device="cuda")   # never touched
    out = torch.empty((), dtype=torch.float64, device="cuda")
    st = lbm._lib().lbm_kinetic_energy_noalloc(ctypes.byref(p.c()), ctypes.c_void_p(dummy.data_ptr()),
                                               ctypes.c_void_p(out.data_ptr()), None)
    assert st == lbm.ESIZE
    assert b"LBM_NOALLOC_MAX_TILES" in lbm._lib().lbm_strerror(st)
