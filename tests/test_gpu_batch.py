"""Batched stepping of independent lattices of uneven sizes (C-ABI lbm_batch_*).

Each lattice of a batch is checked against the oracle run of that lattice alone (the
parity bars of its form).  Every mode also runs the same per-strip step as the
single-lattice kernel, so each lattice must equal lbm_run on that lattice bit for bit (FP64,
FP64 with the fixed-point relaxation, and FP32 storage).  The
persistent mode's grid barrier is bounded in time: a test makes the wait expire (a
barrier that waits for a block that never arrives) and checks the reported status and
that the GPU context stays usable.
"""
import pytest
import torch

from oracle import lbm as OL
from paper_1703_04594_gb300 import lbm
from tests.gpu_util import field_errors, oracle_params, rel_err, require_gpu, rt_fields, to_host

pytestmark = pytest.mark.gpu

SHAPES = [(32, 64, 0.6), (48, 96, 0.7), (64, 128, 0.75), (40, 80, 0.9), (96, 192, 1.0), (33, 45, 0.65)]


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def smooth_periodic_fields(p, seed):
    """A state that is smooth across the periodic-y wrap: the RT state at one temperature
    (hydrostatic density, interface modes of ``seed``) with a uniform drift.  The RT state
    itself puts the hot bottom layer next to the cold top layer at the wrap, a one-site jump
    that drives some populations near zero, where the elementwise relative bar is
    ill-conditioned (rounding-level input changes move the oracle's own outputs there by
    ~2e-13 after 5 steps)."""
    rho, ux, uy, T = rt_fields(lbm.Params(p.lx, p.ly, tau=p.tau, t_bottom=1.0, t_top=1.0), seed)
    return rho, ux + 0.01, uy - 0.005, T


def make_batch(precision, bc=lbm.BC_WALLS, seed0=100, with_fields=False, smooth_periodic=False):
    params, fa, fb, fields = [], [], [], []
    for j, (lx, ly, tau) in enumerate(SHAPES):
        p = lbm.Params(lx, ly, tau=tau, gx=1e-4 * (j % 2), precision=precision, bc=bc)
        fl = smooth_periodic_fields(p, seed0 + j) if smooth_periodic else rt_fields(p, seed0 + j)
        dev = [t.contiguous().cuda() for t in fl]
        a, b = lbm.empty_state(p), lbm.empty_state(p)
        lbm.init(p, *dev, a)
        params.append(p)
        fa.append(a)
        fb.append(b)
        fields.append(fl)
    return (params, fa, fb, fields) if with_fields else (params, fa, fb)


def reference(params, fa, steps):
    out = []
    for p, a in zip(params, fa):
        x, y = a.clone(), lbm.empty_state(p)
        out.append(lbm.run(p, x, y, steps).clone())
    return out


def assert_equal_states(params, got, want):
    for p, g, w in zip(params, got, want):
        assert torch.equal(g[:, :, : p.ly], w[:, :, : p.ly]), p


@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP32_SHIFTED, lbm.FP64_FIXED, lbm.FP32_CONSERVED])
@pytest.mark.parametrize("mode,tx", [(lbm.BATCH_PER_STEP, 4), (lbm.BATCH_PER_STEP, 1), (lbm.BATCH_PER_STEP, 8),
                                      (lbm.BATCH_PERSISTENT, 4), (lbm.BATCH_PERSISTENT, 2), (lbm.BATCH_LOOP, 4)])
def test_batch_equals_single_lattice_runs(precision, mode, tx):
    params, fa, fb = make_batch(precision)
    want = reference(params, fa, 5)
    b = lbm.Batch(params, fa, fb)
    b.configure(mode, tx, 0)
    b.run(2)
    b.run(3)                      # parity carried across runs
    torch.cuda.synchronize()
    assert b.status() == lbm.OK
    assert b.parity() == 1
    assert_equal_states(params, b.states(), want)
    b.close()


ORACLE_STEPS = 5


@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP64_FIXED, lbm.FP32_SHIFTED, lbm.FP32_CONSERVED])
@pytest.mark.parametrize("mode", [lbm.BATCH_PER_STEP, lbm.BATCH_PERSISTENT])
@pytest.mark.parametrize("bc", [lbm.BC_WALLS, lbm.BC_PERIODIC_Y])
def test_batch_matches_oracle(precision, mode, bc):
    """Every lattice of a batch against the oracle run of that lattice alone (its own size,
    tau, gravity and interface): populations within 1e-12 relative after 5 steps for the
    float64 forms; the FP32 form's per-field bar (density and temperature max and RMS
    relative, velocity relative to the sound speed) within 1e-5."""
    params, fa, fb, fields = make_batch(precision, bc=bc, seed0=600, with_fields=True,
                                        smooth_periodic=bc == lbm.BC_PERIODIC_Y)
    b = lbm.Batch(params, fa, fb)
    b.configure(mode, 4)
    b.run(ORACLE_STEPS)
    torch.cuda.synchronize()
    assert b.status() == lbm.OK
    for p, got, fl in zip(params, b.states(), fields):
        want = OL.run(OL.init_equilibrium(*fl), oracle_params(p), ORACLE_STEPS)
        if precision in (lbm.FP32_SHIFTED, lbm.FP32_CONSERVED):
            err = field_errors([t.cpu() for t in lbm.moments(p, got)], OL.fields(want))
            assert max(err[k] for k in ("rho_max", "rho_rms", "T_max", "T_rms", "u_max_cs")) <= 1e-5, (p, err)
        else:
            assert rel_err(to_host(p, got), want) <= 1e-12, p
    b.close()


def test_batch_periodic_mode():
    params, fa, fb = make_batch(lbm.FP64, bc=lbm.BC_PERIODIC_Y)
    want = reference(params, fa, 4)
    b = lbm.Batch(params, fa, fb)
    b.configure(lbm.BATCH_PERSISTENT, 4)
    b.run(4)
    assert_equal_states(params, b.states(), want)
    b.close()


def test_autotune_then_correct_run():
    params, fa, fb = make_batch(lbm.FP32_SHIFTED)
    b = lbm.Batch(params, fa, fb)
    cfg = b.autotune(trial_steps=2)          # advances the (throw-away) states
    assert cfg["mode"] in (lbm.BATCH_PER_STEP, lbm.BATCH_PERSISTENT)
    assert cfg["tile_columns"] in (2, 4, 8)
    b.close()
    params, fa, fb = make_batch(lbm.FP32_SHIFTED, seed0=200)
    want = reference(params, fa, 6)
    b = lbm.Batch(params, fa, fb)
    b.configure(cfg["mode"], cfg["tile_columns"], cfg["blocks_per_sm"])
    b.run(6)
    assert_equal_states(params, b.states(), want)
    b.close()


def test_persistent_run_in_cuda_graph():
    params, fa, fb = make_batch(lbm.FP64, seed0=300)
    start = [t.clone() for t in fa]
    want = reference(params, start, 8)
    b = lbm.Batch(params, fa, fb)
    b.configure(lbm.BATCH_PERSISTENT, 4)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.run(2)                              # warm-up outside capture (even: parity back to 0)
    torch.cuda.current_stream().wait_stream(s)
    for t, s0 in zip(fa, start):
        t.copy_(s0)
    with torch.cuda.graph(g):
        b.run(4)                              # even step count: replays keep the parity
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    assert b.status() == lbm.OK and b.parity() == 0
    assert_equal_states(params, b.states(), want)
    b.close()


def test_barrier_wait_expires_and_reports_timeout():
    params, fa, fb = make_batch(lbm.FP64, seed0=400)
    b = lbm.Batch(params, fa, fb)
    b.configure(lbm.BATCH_PERSISTENT, 4)
    b.set_wait(timeout_ns=200_000_000, phantom_arrivals=1)   # waits for a block that never comes
    b.run(3)
    torch.cuda.synchronize()
    assert b.status() == lbm.ETIMEOUT
    # the context is still usable and a normal run afterwards is correct
    b.close()
    params, fa, fb = make_batch(lbm.FP64, seed0=500)
    want = reference(params, fa, 3)
    b = lbm.Batch(params, fa, fb)
    b.configure(lbm.BATCH_PERSISTENT, 4)
    b.run(3)
    assert b.status() == lbm.OK
    assert_equal_states(params, b.states(), want)
    b.close()


def test_timeout_of_an_earlier_run_is_not_erased_by_a_later_one():
    """Two persistent runs queued before the status is read: the first one's barrier wait
    expires (a block that never arrives), the second one runs normally.  The status still
    reports the first run's timeout, once."""
    params, fa, fb = make_batch(lbm.FP64, seed0=450)
    b = lbm.Batch(params, fa, fb)
    b.configure(lbm.BATCH_PERSISTENT, 4)
    b.set_wait(timeout_ns=200_000_000, phantom_arrivals=1)
    b.run(3)
    b.set_wait(timeout_ns=2_000_000_000, phantom_arrivals=0)
    b.run(3)
    torch.cuda.synchronize()
    assert b.status() == lbm.ETIMEOUT
    assert b.status() == lbm.OK
    b.close()


def test_plan_rejects_mixed_precision_and_aliasing():
    params, fa, fb = make_batch(lbm.FP64)
    bad = list(params)
    bad[1] = lbm.Params(bad[1].lx, bad[1].ly, precision=lbm.FP32_SHIFTED)
    with pytest.raises((lbm.LbmError, ValueError)):
        lbm.Batch(bad, fa, fb)
    with pytest.raises(lbm.LbmError):
        lbm.Batch(params, fa, fa)                             # f_a == f_b
    with pytest.raises(lbm.LbmError):
        lbm.Batch([params[0], params[0]], [fa[0], fb[0]], [fb[1], fa[0]])   # one buffer in two lattices
