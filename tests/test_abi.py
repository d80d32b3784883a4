"""C-ABI checks that need no GPU: the library loads, exports every declared entry point,
its model constants satisfy the isotropy conditions and agree with the oracle's
independently solved ones, and invalid arguments are rejected before any launch."""
import ctypes
import math
import os
import re

import pytest
import torch

from paper_1703_04594_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm_d2q37.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(lbm.LIB_PATH):
        from paper_1703_04594_gb300 import build
        build.build()
    return lbm._lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(lbm.exported_symbols()) == names


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(lbm, "_LIB", None)
    monkeypatch.setattr(lbm, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="not built"):
        lbm.version()


def gauss(n):
    return 0 if n % 2 else math.prod(range(n - 1, 0, -2))


def test_library_constants_satisfy_isotropy(lib):
    c, w, vx, vy = lbm.model()
    assert abs(sum(w) - 1.0) < 1e-15 and all(x > 0 for x in w)
    for p in range(9):
        for q in range(9 - p):
            lhs = sum(wi * (c * a) ** p * (c * b) ** q for wi, a, b in zip(w, vx, vy))
            assert abs(lhs - gauss(p) * gauss(q)) <= 2e-14 * max(1, gauss(p) * gauss(q)), (p, q)


def test_library_constants_match_oracle(lib):
    from oracle import d2q37 as M
    c, w, vx, vy = lbm.model()
    assert list(zip(vx, vy)) == M.VELOCITIES
    assert abs(c - M.C_SCALE) <= 2e-16 * c
    for a, b in zip(w, M.WEIGHTS.tolist()):
        assert abs(a - b) <= 2e-16 * b


def test_pitch_and_sizes(lib):
    p = lbm.Params(64, 128)
    assert lbm.pitch(p) == 128 and lbm.buffer_bytes(p) == 37 * 64 * 128 * 8
    p = lbm.Params(37, 45)
    assert lbm.pitch(p) == 64
    p = lbm.Params(37, 45, precision=lbm.FP32_SHIFTED)
    assert lbm.buffer_bytes(p) == 37 * 37 * 64 * 4


@pytest.mark.parametrize("bad", [dict(lx=3), dict(ly=5), dict(tau=0.5), dict(tau=float("nan")),
                                 dict(t_top=-1.0), dict(precision=7), dict(bc=3)])
def test_invalid_params_rejected(lib, bad):
    kw = dict(lx=8, ly=8)
    kw.update(bad)
    p = lbm.Params(**kw)
    assert lib.lbm_pitch(ctypes.byref(p.c())) == -1
    # rejected before any launch: the fake pointers are never touched
    st = lib.lbm_step(ctypes.byref(p.c()), ctypes.c_void_p(1 << 20), ctypes.c_void_p(1 << 30), None)
    assert st == lbm.EINVAL


@pytest.mark.parametrize("lx,ly,ok", [
    (4 * 65535, 6, True),          # the largest lx the launch grid takes (grid.y = lx / 4)
    (4 * 65535 + 1, 6, False),
    (65535, 65504, True),          # one population plane just below 2^32 elements
    (65536, 65536, False),         # a plane of exactly 2^32 elements
    (131072, 32768, False),
])
def test_maximum_sizes(lib, lx, ly, ok):
    """Sizes at the edge of what the 32-bit in-plane offsets and the launch grid allow are
    accepted or rejected by the parameter check alone (no launch, nothing allocated)."""
    p = lbm.Params(lx, ly)
    pitch = lib.lbm_pitch(ctypes.byref(p.c()))
    if ok:
        assert pitch == (ly + 31) // 32 * 32 and lx * pitch < 2 ** 32
    else:
        assert pitch == -1
        st = lib.lbm_step(ctypes.byref(p.c()), ctypes.c_void_p(1 << 20), ctypes.c_void_p(1 << 40), None)
        assert st == lbm.EINVAL


def test_aliasing_and_alignment_rejected(lib):
    p = lbm.Params(8, 8)
    nbytes = lbm.buffer_bytes(p)
    base = 1 << 32
    assert lib.lbm_step(ctypes.byref(p.c()), ctypes.c_void_p(base), ctypes.c_void_p(base + nbytes // 2), None) == lbm.EINVAL
    assert lib.lbm_step(ctypes.byref(p.c()), ctypes.c_void_p(base + 8), ctypes.c_void_p(base + 4 * nbytes), None) == lbm.EINVAL
    assert lib.lbm_run(ctypes.byref(p.c()), ctypes.c_void_p(base), ctypes.c_void_p(base + 4 * nbytes), -1, None) == lbm.EINVAL
    assert lib.lbm_strerror(lbm.EINVAL).startswith(b"invalid")


def test_binding_rejects_host_tensors_and_wrong_buffers_before_any_call(lib):
    """The Python binding checks device, dtype, contiguity and size of every state and
    field argument before it calls into the library (so these run without a GPU)."""
    p = lbm.Params(8, 8)
    n = lbm.buffer_bytes(p) // 8
    host_state = torch.zeros(n, dtype=torch.float64)
    with pytest.raises(ValueError, match="f_in"):
        lbm.step(p, host_state, host_state)
    with pytest.raises(ValueError, match="f_in"):
        lbm.step(p, torch.zeros(n, dtype=torch.float32), host_state)
    p32 = lbm.Params(8, 8, precision=lbm.FP32_SHIFTED)
    assert lbm.state_dtype(p32) == torch.float32 and lbm.buffer_bytes(p32) == lbm.buffer_bytes(p) // 2
    field = torch.zeros(8, 8, dtype=torch.float64)
    with pytest.raises(ValueError):
        lbm.init(p, field, field, field, field, host_state)


def test_batch_plan_rejects_buffers_shared_between_lattices(lib):
    """lbm_batch_plan checks the 2n state buffers of a batch against each other before any
    CUDA call: one lattice's buffer overlapping another lattice's is LBM_EINVAL (the fake
    addresses are never touched)."""
    ps = [lbm.Params(8, 8), lbm.Params(16, 8)]
    arr = (lbm.CParams * 2)(*[p.c() for p in ps])
    nb = [lbm.buffer_bytes(p) for p in ps]
    base = 1 << 36

    def plan(a0, b0, a1, b1):
        pa = (ctypes.c_void_p * 2)(a0, a1)
        pb = (ctypes.c_void_p * 2)(b0, b1)
        h = ctypes.c_void_p()
        return lib.lbm_batch_plan(arr, pa, pb, 2, ctypes.byref(h))

    step = 1 << 24                               # far apart: 16 MiB between buffers
    assert plan(base, base + 2 * step, base + 2 * step + nb[0] // 2, base + 3 * step) == lbm.EINVAL
    assert plan(base, base + step, base + 2 * step, base) == lbm.EINVAL          # shared buffer
    assert plan(base + step, base, base + 2 * step, base + step + 256) == lbm.EINVAL
