"""Thin Python binding of the C-ABI in ``include/lbm_d2q37.h`` (argument marshalling only).

Every entry point has the same name as its C function without the ``lbm_`` prefix.
Device buffers are torch CUDA tensors (PyTorch supplies memory and streams only); the
work itself runs in the library's kernels.  The library is loaded on first use and a
missing library raises ``RuntimeError``: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_native", "liblbm_d2q37.so")

FP64, FP32_SHIFTED, FP64_FIXED, FP32_CONSERVED = 0, 1, 2, 3
BC_WALLS, BC_PERIODIC_Y = 0, 1
Q = 37

OK, EINVAL, ECUDA, ETIMEOUT, ENOMEM, ESIZE = 0, 1, 2, 3, 4, 5
NOALLOC_MAX_TILES = 262144


class CParams(ctypes.Structure):
    _fields_ = [("lx", ctypes.c_int32), ("ly", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("bc", ctypes.c_int32), ("tau", ctypes.c_double), ("gx", ctypes.c_double),
                ("gy", ctypes.c_double), ("t_bottom", ctypes.c_double), ("t_top", ctypes.c_double),
                ("rho0", ctypes.c_double)]


@dataclass(frozen=True)
class Params:
    """Problem parameters (Sec. 3): lattice size, relaxation time, gravity (xi units per
    step), wall temperatures; ``precision`` and ``bc`` select the storage form and the
    y boundary."""
    lx: int
    ly: int
    tau: float = 0.8
    gx: float = 0.0
    gy: float = -1e-4
    t_bottom: float = 1.15
    t_top: float = 0.85
    rho0: float = 1.0
    precision: int = FP64
    bc: int = BC_WALLS

    def c(self) -> CParams:
        return CParams(self.lx, self.ly, self.precision, self.bc, self.tau, self.gx, self.gy,
                       self.t_bottom, self.t_top, self.rho0)


class LbmError(RuntimeError):
    def __init__(self, fn: str, status: int):
        lib = _lib()
        msg = lib.lbm_strerror(status).decode()
        if status == ECUDA:
            msg += f" (cuda error {lib.lbm_last_cuda_error()})"
        super().__init__(f"{fn}: {msg}")
        self.status = status


_LIB = None

_VP = ctypes.c_void_p
_PP = ctypes.POINTER(CParams)
_SIGS = {
    "lbm_version": (ctypes.c_int32, []),
    "lbm_model": (ctypes.c_int32, [_VP, _VP, _VP, _VP]),
    "lbm_pitch": (ctypes.c_int64, [_PP]),
    "lbm_buffer_bytes": (ctypes.c_int64, [_PP]),
    "lbm_init": (ctypes.c_int32, [_PP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "lbm_step": (ctypes.c_int32, [_PP, _VP, _VP, _VP]),
    "lbm_run": (ctypes.c_int32, [_PP, _VP, _VP, ctypes.c_int32, _VP]),
    "lbm_propagate": (ctypes.c_int32, [_PP, _VP, _VP, _VP]),
    "lbm_propagate_push": (ctypes.c_int32, [_PP, _VP, _VP, _VP]),
    "lbm_bc": (ctypes.c_int32, [_PP, _VP, _VP, _VP]),
    "lbm_collide": (ctypes.c_int32, [_PP, _VP, _VP, _VP]),
    "lbm_moments": (ctypes.c_int32, [_PP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "lbm_reduce_scratch_bytes": (ctypes.c_int64, [_PP]),
    "lbm_kinetic_energy": (ctypes.c_int32, [_PP, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    "lbm_kinetic_energy_noalloc": (ctypes.c_int32, [_PP, _VP, _VP, _VP]),
    "lbm_simulate_host": (ctypes.c_int32, [_PP, _VP, _VP, _VP, _VP, ctypes.c_int32, _VP, _VP, _VP, _VP,
                                           _VP, _VP, _VP, _VP]),
    "lbm_convert_layout": (ctypes.c_int32, [_PP, ctypes.c_int32, _VP, ctypes.c_int32, _VP, _VP]),
    "lbm_step_layout": (ctypes.c_int32, [_PP, ctypes.c_int32, _VP, _VP, _VP]),
    "lbm_adjoint_work_bytes": (ctypes.c_int64, [_PP]),
    "lbm_adjoint_step": (ctypes.c_int32, [_PP, _VP, _VP, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    "lbm_kinetic_energy_grad": (ctypes.c_int32, [_PP, _VP, _VP, _VP]),
    "lbm_init_adjoint": (ctypes.c_int32, [_PP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "lbm_batch_plan": (ctypes.c_int32, [_PP, _VP, _VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)]),
    "lbm_batch_configure": (ctypes.c_int32, [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "lbm_batch_config": (ctypes.c_int32, [_VP, _VP, _VP, _VP]),
    "lbm_batch_autotune": (ctypes.c_int32, [_VP, ctypes.c_int32, _VP]),
    "lbm_batch_run": (ctypes.c_int32, [_VP, ctypes.c_int32, _VP]),
    "lbm_batch_parity": (ctypes.c_int32, [_VP]),
    "lbm_batch_sites": (ctypes.c_int64, [_VP]),
    "lbm_batch_status": (ctypes.c_int32, [_VP]),
    "lbm_batch_set_wait": (ctypes.c_int32, [_VP, ctypes.c_int64, ctypes.c_int32]),
    "lbm_batch_destroy": (None, [_VP]),
    "lbm_probe_peak": (ctypes.c_int32, [ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    "lbm_strerror": (ctypes.c_char_p, [ctypes.c_int32]),
    "lbm_last_cuda_error": (ctypes.c_int32, []),
}


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run `python -m paper_1703_04594_gb300.build`)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def exported_symbols():
    return list(_SIGS)


def _check(fn: str, status: int):
    if status != OK:
        raise LbmError(fn, status)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


# ------------------------------------------------------------------------- host-only
def version() -> int:
    return _lib().lbm_version()


def model():
    """(c, w[37], vx[37], vy[37]) as the library defines them (host only)."""
    c = ctypes.c_double()
    w = (ctypes.c_double * Q)()
    vx = (ctypes.c_int32 * Q)()
    vy = (ctypes.c_int32 * Q)()
    _check("lbm_model", _lib().lbm_model(ctypes.byref(c), w, vx, vy))
    return c.value, list(w), list(vx), list(vy)


def pitch(p: Params) -> int:
    v = _lib().lbm_pitch(ctypes.byref(p.c()))
    if v < 0:
        raise LbmError("lbm_pitch", EINVAL)
    return v


def buffer_bytes(p: Params) -> int:
    v = _lib().lbm_buffer_bytes(ctypes.byref(p.c()))
    if v < 0:
        raise LbmError("lbm_buffer_bytes", EINVAL)
    return v


def state_dtype(p: Params):
    return torch.float32 if p.precision in (FP32_SHIFTED, FP32_CONSERVED) else torch.float64


def empty_state(p: Params, device="cuda") -> torch.Tensor:
    """An uninitialised state buffer [37, lx, pitch] of the storage type."""
    return torch.empty((Q, p.lx, pitch(p)), dtype=state_dtype(p), device=device)


def _state(p: Params, t: torch.Tensor, name: str):
    if not (t.is_cuda and t.is_contiguous() and t.dtype == state_dtype(p)
            and t.numel() * t.element_size() >= buffer_bytes(p)):
        raise ValueError(f"{name}: expected a contiguous CUDA {state_dtype(p)} tensor of "
                         f"{buffer_bytes(p)} bytes, got {t.dtype} {tuple(t.shape)} on {t.device}")
    return _ptr(t)


def _field(p: Params, t: torch.Tensor, name: str):
    if not (t.is_cuda and t.is_contiguous() and t.dtype == torch.float64 and t.numel() == p.lx * p.ly):
        raise ValueError(f"{name}: expected a contiguous CUDA float64 [lx, ly] tensor")
    return _ptr(t)


# ------------------------------------------------------------------------- device calls
def init(p: Params, rho, ux, uy, T, f, stream=None):
    _check("lbm_init", _lib().lbm_init(ctypes.byref(p.c()), _field(p, rho, "rho"), _field(p, ux, "ux"),
                                       _field(p, uy, "uy"), _field(p, T, "T"), _state(p, f, "f"),
                                       _stream(stream)))
    return f


def step(p: Params, f_in, f_out, stream=None):
    _check("lbm_step", _lib().lbm_step(ctypes.byref(p.c()), _state(p, f_in, "f_in"),
                                       _state(p, f_out, "f_out"), _stream(stream)))
    return f_out


def run(p: Params, f_a, f_b, n_steps: int, stream=None):
    """n_steps fused steps; returns the tensor holding the result."""
    _check("lbm_run", _lib().lbm_run(ctypes.byref(p.c()), _state(p, f_a, "f_a"), _state(p, f_b, "f_b"),
                                     int(n_steps), _stream(stream)))
    return f_a if n_steps % 2 == 0 else f_b


def propagate(p: Params, f_in, f_tmp, stream=None):
    _check("lbm_propagate", _lib().lbm_propagate(ctypes.byref(p.c()), _state(p, f_in, "f_in"),
                                                 _state(p, f_tmp, "f_tmp"), _stream(stream)))
    return f_tmp


def propagate_push(p: Params, f_in, f_tmp, stream=None):
    _check("lbm_propagate_push", _lib().lbm_propagate_push(ctypes.byref(p.c()), _state(p, f_in, "f_in"),
                                                           _state(p, f_tmp, "f_tmp"), _stream(stream)))
    return f_tmp


def bc(p: Params, f_in, f_tmp, stream=None):
    _check("lbm_bc", _lib().lbm_bc(ctypes.byref(p.c()), _state(p, f_in, "f_in"), _state(p, f_tmp, "f_tmp"),
                                   _stream(stream)))
    return f_tmp


def collide(p: Params, f_tmp, f_out, stream=None):
    _check("lbm_collide", _lib().lbm_collide(ctypes.byref(p.c()), _state(p, f_tmp, "f_tmp"),
                                             _state(p, f_out, "f_out"), _stream(stream)))
    return f_out


def moments(p: Params, f, out=None, stream=None):
    """(rho, ux, uy, T) of a state, each [lx, ly] float64 on the state's device."""
    if out is None:
        out = [torch.empty((p.lx, p.ly), dtype=torch.float64, device=f.device) for _ in range(4)]
    rho, ux, uy, T = out
    _check("lbm_moments", _lib().lbm_moments(ctypes.byref(p.c()), _state(p, f, "f"), _field(p, rho, "rho"),
                                             _field(p, ux, "ux"), _field(p, uy, "uy"), _field(p, T, "T"),
                                             _stream(stream)))
    return rho, ux, uy, T


def reduce_scratch_bytes(p: Params) -> int:
    return _lib().lbm_reduce_scratch_bytes(ctypes.byref(p.c()))


def kinetic_energy(p: Params, f, out=None, scratch=None, stream=None):
    """Total kinetic energy as a 0-d float64 device tensor."""
    if out is None:
        out = torch.empty((), dtype=torch.float64, device=f.device)
    if scratch is None:
        scratch = torch.empty(reduce_scratch_bytes(p) // 8, dtype=torch.float64, device=f.device)
    _check("lbm_kinetic_energy", _lib().lbm_kinetic_energy(
        ctypes.byref(p.c()), _state(p, f, "f"), _ptr(out), _ptr(scratch),
        scratch.numel() * scratch.element_size(), _stream(stream)))
    return out


def kinetic_energy_noalloc(p: Params, f, out=None, stream=None):
    """Total kinetic energy without scratch from the caller: for callers that cannot
    allocate device memory while running (memory fully reserved up front, or loops that
    must not call cudaMalloc).  The partial sums go to a fixed array inside the library
    (LBM_NOALLOC_MAX_TILES doubles per GPU); larger lattices raise LbmError (LBM_ESIZE).
    Calls that overlap on the GPU race on that array.  ``out`` is the only device buffer."""
    if out is None:
        out = torch.empty((), dtype=torch.float64, device=f.device)
    _check("lbm_kinetic_energy_noalloc", _lib().lbm_kinetic_energy_noalloc(
        ctypes.byref(p.c()), _state(p, f, "f"), _ptr(out), _stream(stream)))
    return out


def simulate_host(p: Params, fields_in, n_steps: int, fields_out, f_a, f_b, fields_dev, stream=None):
    """End-to-end run from host tensors (pinned for speed): fields in -> init -> n steps ->
    moments -> fields out.  Synchronous."""
    for t in list(fields_in) + list(fields_out):
        if t.is_cuda or not t.is_contiguous() or t.dtype != torch.float64 or t.numel() != p.lx * p.ly:
            raise ValueError("host fields must be contiguous float64 CPU tensors of lx*ly elements")
    if not (fields_dev.is_cuda and fields_dev.dtype == torch.float64 and fields_dev.numel() >= 4 * p.lx * p.ly):
        raise ValueError("fields_dev must be a CUDA float64 tensor of 4*lx*ly elements")
    fi = [_ptr(t) for t in fields_in]
    fo = [_ptr(t) for t in fields_out]
    _check("lbm_simulate_host", _lib().lbm_simulate_host(
        ctypes.byref(p.c()), *fi, int(n_steps), *fo, _state(p, f_a, "f_a"), _state(p, f_b, "f_b"),
        _ptr(fields_dev), _stream(stream)))
    return fields_out


# ------------------------------------------------------------------------- layouts
LAYOUT_SOA, LAYOUT_AOS, LAYOUT_PSOA, LAYOUT_CAOSOA = 0, 1, 2, 3


def convert_layout(p: Params, src, frm: int, dst, to: int, stream=None):
    _check("lbm_convert_layout", _lib().lbm_convert_layout(ctypes.byref(p.c()), frm, _state(p, src, "src"), to,
                                                           _state(p, dst, "dst"), _stream(stream)))
    return dst


def step_layout(p: Params, layout: int, f_in, f_out, stream=None):
    _check("lbm_step_layout", _lib().lbm_step_layout(ctypes.byref(p.c()), layout, _state(p, f_in, "f_in"),
                                                     _state(p, f_out, "f_out"), _stream(stream)))
    return f_out


# ------------------------------------------------------------------------- adjoint
def adjoint_work(p: Params, device="cuda"):
    n = _lib().lbm_adjoint_work_bytes(ctypes.byref(p.c()))
    if n < 0:
        raise LbmError("lbm_adjoint_work_bytes", EINVAL)
    return torch.empty((n + 7) // 8, dtype=torch.float64, device=device)


def adjoint_step(p: Params, f_n, lam_next, lam_n, dtau_acc, work, stream=None):
    """lam_n = (d step/d f_n)^T lam_next; dtau_acc (0-d device float64) += dL/dtau part."""
    _check("lbm_adjoint_step", _lib().lbm_adjoint_step(
        ctypes.byref(p.c()), _state(p, f_n, "f_n"), _state(p, lam_next, "lam_next"), _state(p, lam_n, "lam_n"),
        _ptr(dtau_acc), _ptr(work), work.numel() * work.element_size(), _stream(stream)))
    return lam_n


def kinetic_energy_grad(p: Params, f, lam, stream=None):
    _check("lbm_kinetic_energy_grad", _lib().lbm_kinetic_energy_grad(ctypes.byref(p.c()), _state(p, f, "f"),
                                                                     _state(p, lam, "lam"), _stream(stream)))
    return lam


def init_adjoint(p: Params, rho, ux, uy, T, lam0, stream=None):
    """(g_rho, g_ux, g_uy, g_T): gradients of the initial fields against lam0."""
    out = [torch.empty((p.lx, p.ly), dtype=torch.float64, device=lam0.device) for _ in range(4)]
    _check("lbm_init_adjoint", _lib().lbm_init_adjoint(
        ctypes.byref(p.c()), _field(p, rho, "rho"), _field(p, ux, "ux"), _field(p, uy, "uy"), _field(p, T, "T"),
        _state(p, lam0, "lam0"), *[_ptr(t) for t in out], _stream(stream)))
    return out


# ------------------------------------------------------------------------- batched lattices
BATCH_PER_STEP, BATCH_PERSISTENT, BATCH_LOOP = 1, 2, 3


class Batch:
    """Many independent lattices stepped together (C-ABI ``lbm_batch_*``).

    ``params``: list of Params (same precision and bc); ``f_a`` / ``f_b``: matching lists of
    state tensors (current state in ``f_a``).  The batch keeps the tensors alive.
    """

    def __init__(self, params, f_a, f_b):
        if not (len(params) == len(f_a) == len(f_b) and len(params) > 0):
            raise ValueError("params, f_a and f_b must be non-empty lists of equal length")
        n = len(params)
        self.params = list(params)
        self.f = [list(f_a), list(f_b)]
        arr = (CParams * n)(*[p.c() for p in params])
        pa = (ctypes.c_void_p * n)(*[_state(p, t, "f_a").value for p, t in zip(params, f_a)])
        pb = (ctypes.c_void_p * n)(*[_state(p, t, "f_b").value for p, t in zip(params, f_b)])
        h = ctypes.c_void_p()
        _check("lbm_batch_plan", _lib().lbm_batch_plan(arr, pa, pb, n, ctypes.byref(h)))
        self._h = h

    def configure(self, mode: int, tile_columns: int = 4, blocks_per_sm: int = 0):
        _check("lbm_batch_configure", _lib().lbm_batch_configure(self._h, mode, tile_columns, blocks_per_sm))

    def config(self):
        m, w, b = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check("lbm_batch_config", _lib().lbm_batch_config(self._h, ctypes.byref(m), ctypes.byref(w),
                                                           ctypes.byref(b)))
        return {"mode": m.value, "tile_columns": w.value, "blocks_per_sm": b.value}

    def autotune(self, trial_steps: int = 3, stream=None):
        _check("lbm_batch_autotune", _lib().lbm_batch_autotune(self._h, trial_steps, _stream(stream)))
        return self.config()

    def run(self, n_steps: int, stream=None):
        _check("lbm_batch_run", _lib().lbm_batch_run(self._h, int(n_steps), _stream(stream)))

    def parity(self) -> int:
        return _lib().lbm_batch_parity(self._h)

    def states(self):
        """The tensors holding the current states."""
        return self.f[self.parity()]

    def sites(self) -> int:
        return _lib().lbm_batch_sites(self._h)

    def status(self) -> int:
        return _lib().lbm_batch_status(self._h)

    def set_wait(self, timeout_ns: int, phantom_arrivals: int = 0):
        _check("lbm_batch_set_wait", _lib().lbm_batch_set_wait(self._h, int(timeout_ns), int(phantom_arrivals)))

    def close(self):
        if getattr(self, "_h", None):
            _lib().lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


PROBE_DFMA, PROBE_FFMA, PROBE_IMAD, PROBE_MULHI64, PROBE_UMULHI64 = 0, 1, 2, 3, 4


def probe_peak(kind: int) -> float:
    """Measured sustained rate (operations per second, one FMA = one operation) of one
    arithmetic pipe on the current device: the roofline denominators of the step kernels."""
    out = ctypes.c_double()
    _check("lbm_probe_peak", _lib().lbm_probe_peak(int(kind), ctypes.byref(out)))
    return out.value
