#!/usr/bin/env python
"""Throughput of the GB300 D2Q37 thermal lattice-Boltzmann step, in MLUPS.

Workload: one 4096 x 8192 lattice (33,554,432 fluid sites), periodic in x, thermal
walls T = 1.15 (bottom) / 0.85 (top), tau = 0.8, g = 1e-4 in -y, Rayleigh-Taylor
initial state from seed 2 (synthetic; the paper's convective-turbulence workload
shape).  One bench step = one fused propagate + bc + collide pass over the whole
lattice (one kernel launch).  Each state buffer is 9.9 GB, far larger than the 129 MB
L2, so no L2 flush is needed between steps.

The default line also carries the other forms of the step, each with its own roofline,
clock samples and baseline: ``fp64_fixed_relax`` (float64 states, fixed-point relaxation),
``fp32`` (FP32 shifted storage, same lattice), ``batch_fp64`` / ``batch_fp32`` (256
independent RT lattices, Lx in 128..1024, Ly = 2 Lx, K steps, against looping the
single-lattice kernel) and ``adjoint`` (gradient of the kinetic energy after 500 steps of a
512 x 1024 lattice with checkpoints every 22 steps, against the forward run, and the
adjoint step kernel against its HBM roofline).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--variant fused|separate|push|aos|psoa|caosoa]
    python bench.py --workload batch --steps 200 [--precision fp32|fp64|fp64fix] [--batch-kind small]
    python bench.py --workload adjoint
    python bench.py --impl reference      # the float64 CPU oracle on a bounded sample

Under torchrun (N > 1) every rank steps its own replica lattice (independent problems:
weak scaling, no collective on the data path); rank 0 prints one JSON line with the
headline forms only.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

LX, LY, SEED = 4096, 8192, 2
TAU, GY, T_BOTTOM, T_TOP = 0.8, -1e-4, 1.15, 0.85

# Algorithmic work per site of the fused FP64 step: the factored collision (moments as
# pair sums grouped by their integer velocity weights, per-shell Hermite coefficients, one
# even/odd Horner pair per opposite pair, BGK relaxation), FMA = 2 flops:
#   138 add + 97 mul + 138 fma + 1 div = 512 flops, 374 operations.
# tests/test_flop_count.py counts it mechanically on a formulation checked against the
# oracle's collision.
FLOP_MIX_FP64 = (138, 97, 138, 1)      # add, mul, fma, div
FLOPS_PER_SITE_FP64 = 512
BYTES_PER_SITE_FP64 = 592          # 37 x 8 B read + 37 x 8 B written
BYTES_PER_SITE_FP32 = 296          # 37 x 4 B read + 37 x 4 B written
# FP64 peak from unit counts and clocks: 152 SMs x 2 DFMA/clk/SM x 2 flops x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# DRAM bytes per site (dram__bytes_read.sum + dram__bytes_write.sum of one launch of the
# current kernel, from an ncu capture on a smaller lattice or batch, divided by its sites;
# profiles/ holds the captures).  A launch's `traffic` is this times its sites.  None where
# no capture of the current kernel exists.  Reads equal the algorithmic bytes; writes read
# a little low on the captured cases because their tail is still in L2 when the kernel ends.
TRAFFIC_BYTES_PER_SITE = {
    "fused": 540.6,        # k_step_fp64, 512 x 2048
    "fp64fix": 569.7,      # k_step_fix64, 1024 x 2048
    "fp32": 272.8,         # k_step_fp32 (shifted), 1024 x 2048
    "fp32c": 273.3,        # k_step_fp32 (conserved moments), 1024 x 2048
    "adjoint": 828.3,      # k_adj_collide, 512 x 1024 (the adjoint workload's own lattice)
    "batch_fp32": 259.4,   # k_batch_step<fp32>, 64 small lattices
    "batch_fp64": 587.0,   # k_batch_step<double>, 8 lattices Lx 128..1024
    "separate": None,
}


def traffic(key, sites):
    """DRAM bytes of one launch over `sites` sites, from the captured bytes per site."""
    b = TRAFFIC_BYTES_PER_SITE.get(key)
    return None if b is None else b * sites



def _hbm_peak(root=None):
    """Measured STREAM-style copy bandwidth of the GB300s (GB/s) and where the
    figure comes from: MEASURED_PEAKS.json, else one earlier GB300 measurement (6.8 TB/s)."""
    try:
        with open(os.path.join(root or ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except (OSError, KeyError, ValueError, TypeError):
        return 6800.0, "6.8 TB/s, an earlier GB300 copy measurement (of fallback)"


HBM_PEAK_GBS, HBM_PEAK_SOURCE = _hbm_peak()


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--variant", choices=["fused", "separate", "push", "aos", "psoa", "caosoa"], default="fused",
                    help="fused SoA step; separate propagate/bc/collide kernels with the pull or push "
                         "propagate; fused step in the AoS, partitioned-SoA or CAoSoA layout (FP64)")
    ap.add_argument("--precision", choices=["fp64", "fp32", "fp32c", "fp64fix"], default="fp64",
                    help="fp32 = FP32 shifted-deviation storage (fused only); fp32c = the same storage with "
                         "the conserved-moment correction; fp64fix = float64 storage "
                         "with the fixed-point relaxation (fused only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fixed", action="store_true",
                    help="skip the extra timing of the fixed-point-relaxation FP64 step")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the FP32, batched and adjoint forms that the default line adds")
    ap.add_argument("--batch-kind", choices=["uneven", "small"], default="uneven",
                    help="uneven = 256 lattices, Lx in 128..1024, Ly = 2 Lx; small = 1024 lattices, "
                         "Lx in 32..128 (a launch-bound batch)")
    ap.add_argument("--workload", choices=["single", "batch", "adjoint", "adjoint-step"], default="single",
                    help="batch = 256 independent lattices of uneven sizes; adjoint = gradient of the "
                         "kinetic energy after 500 steps of a 512x1024 lattice (checkpoints every 22); "
                         "adjoint-step = the adjoint step kernel alone on --lx x --ly (default 512x1024)")
    ap.add_argument("--batch-n", type=int, default=0, help="lattices of the batch (default 256, or 1024 small)")
    ap.add_argument("--lx", type=int, default=LX, help="lattice width (profiling of smaller cases)")
    ap.add_argument("--ly", type=int, default=LY, help="lattice height (profiling of smaller cases)")
    return ap.parse_args()


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, device="cpu") -> float:
    """The largest value over all ranks (the slowest rank's time); identity on one rank."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t)


def whole_job_mlups(sites_per_rank: int, steps: int, world: int, slowest_ms: float) -> float:
    """Whole-job throughput: every rank's site updates over the slowest rank's time."""
    return world * sites_per_rank * steps / (slowest_ms * 1e-3) / 1e6


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[4:8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        loaded = [r[0] for r in rows if r[0] > 0.5 * r[1]] or [r[0] for r in rows]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------- CPU oracle
def oracle_sample(steps: int, cols: int = 16, threads: int | None = None):
    """Time the float64 CPU oracle on a bounded crop of the same workload: ``cols`` full-
    height columns (cols x 8192 sites) of the seed-2 Rayleigh-Taylor lattice, on torch's
    default thread count or on ``threads`` threads."""
    import torch

    from oracle import lbm as OL
    from paper_1703_04594_gb300 import inputs as I

    modes = I.rt_modes(LX, LY, SEED)
    fields = [t[:cols].contiguous() for t in I.rt_fields(LX, LY, modes, T_BOTTOM, T_TOP, abs(GY))]
    p = OL.Params(cols, LY, tau=TAU, gy=GY, t_bottom=T_BOTTOM, t_top=T_TOP)
    f = OL.init_equilibrium(*fields)
    saved = torch.get_num_threads()
    if threads is not None:
        torch.set_num_threads(threads)
    try:
        used = torch.get_num_threads()
        t0 = time.perf_counter()
        for _ in range(steps):
            f = OL.step(f, p)
        dt = time.perf_counter() - t0
    finally:
        torch.set_num_threads(saved)
    return {"value": cols * LY * steps / dt / 1e6, "unit": "MLUPS", "cores": used,
            "kind": "oracle",
            "sample": f"{cols}x{LY} column crop of the {LX}x{LY} seed-{SEED} RT lattice, {steps} steps, "
                      f"{dt:.1f} s"}


def headline_config(lx: int, ly: int, variant: str, precision: str, world: int) -> dict:
    """The `config` of the single-lattice line (both arms report the same one)."""
    name = {"fp32": "FP32-shifted", "fp32c": "FP32-conserved", "fp64fix": "FP64 fixed-point-relax"}.get(precision,
                                                                                                      "FP64")
    return {"workload": f"D2Q37 {name} {variant} step, {lx}x{ly} Rayleigh-Taylor lattice",
            "lx": lx, "ly": ly, "tau": TAU, "gy": GY, "t_bottom": T_BOTTOM, "t_top": T_TOP,
            "seed": SEED, "variant": variant, "precision": precision,
            "l2": "state buffers >= 4.9 GB >> 129 MB L2; no flush needed",
            "parallelism": f"replicas x{world}"}


def run_reference(a):
    world, rank, _ = _dist()
    if rank != 0:
        return
    oracle_sample(max(1, a.warmup))                    # warm-up steps, untimed
    cb = oracle_sample(a.steps)
    line = {"impl": "reference", "metric": "D2Q37 MLUPS", "value": cb["value"], "unit": "MLUPS",
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 16 * LY / cb["value"] / 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": headline_config(LX, LY, "fused", "fp64", a.gpus),
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------- GPU
def run_ours(a):
    import torch
    import torch.distributed as dist

    from paper_1703_04594_gb300 import inputs as I
    from paper_1703_04594_gb300 import lbm

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if not os.path.exists(lbm.LIB_PATH):
        raise RuntimeError("CUDA library missing: run __graft_entry__.build() first")

    lx, ly = a.lx, a.ly
    fp32 = a.precision in ("fp32", "fp32c")
    fix = a.precision == "fp64fix"
    if (fp32 or fix) and a.variant != "fused":
        raise SystemExit(f"--precision {a.precision} supports the fused step only")
    p = lbm.Params(lx, ly, tau=TAU, gy=GY, t_bottom=T_BOTTOM, t_top=T_TOP, precision=prec_enum(lbm, a.precision))
    sites = lx * ly
    dev = [t.contiguous() for t in I.rt_state(lx, ly, SEED + rank, t_bottom=T_BOTTOM, t_top=T_TOP, g=abs(GY),
                                              device="cuda")]
    fields = [t.cpu() for t in dev]
    fa, fb = lbm.empty_state(p), lbm.empty_state(p)
    separate = a.variant in ("separate", "push")
    ftmp = lbm.empty_state(p) if separate else None
    lbm.init(p, *dev, fa)
    stream = torch.cuda.current_stream()
    layout = {"aos": lbm.LAYOUT_AOS, "psoa": lbm.LAYOUT_PSOA, "caosoa": lbm.LAYOUT_CAOSOA}.get(a.variant)
    prop = lbm.propagate_push if a.variant == "push" else lbm.propagate
    if layout is not None:
        if fp32:
            raise SystemExit("layout variants run the FP64 step")
        lbm.convert_layout(p, fa, lbm.LAYOUT_SOA, fb, layout, stream)
        fa, fb = fb, fa

    def one_step(src, dst):
        if a.variant == "fused":
            lbm.step(p, src, dst, stream)
        elif layout is not None:
            lbm.step_layout(p, layout, src, dst, stream)
        else:
            prop(p, src, ftmp, stream)
            lbm.bc(p, src, ftmp, stream)
            lbm.collide(p, ftmp, dst, stream)

    bufs = [fa, fb]
    # the float64 FMA rate measured by the library's probe kernel (TFLOP/s, FMA = 2 flops),
    # beside the peak derived from unit counts and the maximum clock
    fp64_measured = 2 * lbm.probe_peak(lbm.PROBE_DFMA) / 1e12 if not (fp32 or fix) else None
    for k in range(a.warmup):
        one_step(bufs[k % 2], bufs[(k + 1) % 2])
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps + 1)]
    with ClockSampler(local) as clk:
        ev[0].record(stream)
        for k in range(a.steps):
            one_step(bufs[(a.warmup + k) % 2], bufs[(a.warmup + k + 1) % 2])
            ev[k + 1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    per_step = [ev[k].elapsed_time(ev[k + 1]) for k in range(a.steps)]
    total_ms = max_over_ranks(ev[0].elapsed_time(ev[-1]), "cuda")
    ms_per_step = total_ms / a.steps
    value = whole_job_mlups(sites, a.steps, world, total_ms)

    # dominant kernel: the fused step is the only launch of a fused bench step
    kern_ms = statistics.mean(per_step)
    if fp32 or fix:
        achieved = (BYTES_PER_SITE_FP32 if fp32 else BYTES_PER_SITE_FP64) * sites / (kern_ms * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                    "frac": achieved / HBM_PEAK_GBS, "traffic": traffic(a.precision, sites),
                    "kernel": "k_step_fp32" if fp32 else "k_step_fix64",
                    "peak_source": HBM_PEAK_SOURCE}
    else:
        achieved = FLOPS_PER_SITE_FP64 * sites / (kern_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic(a.variant, sites),
                    "peak_measured": fp64_measured,
                    "frac_of_measured": achieved / fp64_measured if fp64_measured else None,
                    "kernel": {"fused": "k_step_fp64", "separate": "whole step (3 kernels)",
                               "push": "whole step (3 kernels)", "aos": "k_step_layout<AoS>",
                               "psoa": "k_step_layout<PSoA>", "caosoa": "k_step_layout<CAoSoA>"}[a.variant],
                    "peak_source": "152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz",
                    "hbm_gbs_equiv": BYTES_PER_SITE_FP64 * sites / (kern_ms * 1e-3) / 1e9}

    # end to end through the C-ABI from pinned host fields: H2D, init, K steps, moments, D2H
    pinned_in = [t.contiguous().pin_memory() for t in fields]
    pinned_out = [torch.empty(lx, ly, dtype=torch.float64).pin_memory() for _ in range(4)]
    fdev = torch.empty(4 * sites, dtype=torch.float64, device="cuda")
    lbm.simulate_host(p, pinned_in, 1, pinned_out, fa, fb, fdev, stream)
    runs = []
    with ClockSampler(local) as eclk:
        for _ in range(3):                    # median of three end-to-end runs
            if world > 1:
                dist.barrier()
            t0 = time.perf_counter()
            lbm.simulate_host(p, pinned_in, a.steps, pinned_out, fa, fb, fdev, stream)
            runs.append(max_over_ranks(time.perf_counter() - t0, "cuda"))
    e2e_s = statistics.median(runs)
    field_bytes = 4 * sites * 8
    e2e = {"value": whole_job_mlups(sites, a.steps, world, e2e_s * 1e3), "unit": "MLUPS",
           "h2d_bytes_per_step": field_bytes / a.steps, "d2h_bytes_per_step": field_bytes / a.steps,
           "what": "lbm_simulate_host: fields H2D + init + K steps + moments + fields D2H, amortised per "
                   "step; median of 3 calls",
           "runs_s": runs, "clocks": eclk.summary()}
    del pinned_in, pinned_out, fdev

    # the same FP64 step with the fixed-point relaxation (LBM_FP64_FIXED), on the same lattice
    fixed_line = None
    if a.precision == "fp64" and a.variant == "fused" and not a.no_fixed:
        pf = lbm.Params(lx, ly, tau=TAU, gy=GY, t_bottom=T_BOTTOM, t_top=T_TOP, precision=lbm.FP64_FIXED)
        lbm.init(pf, *dev, bufs[0])
        for k in range(a.warmup):
            lbm.step(pf, bufs[k % 2], bufs[(k + 1) % 2], stream)
        torch.cuda.synchronize()
        fev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        with ClockSampler(local) as fclk:
            fev[0].record(stream)
            for k in range(a.steps):
                lbm.step(pf, bufs[(a.warmup + k) % 2], bufs[(a.warmup + k + 1) % 2], stream)
            fev[1].record(stream)
            torch.cuda.synchronize()
        f_ms = max_over_ranks(fev[0].elapsed_time(fev[1]), "cuda")
        f_kern = f_ms / a.steps
        f_gbs = BYTES_PER_SITE_FP64 * sites / (f_kern * 1e-3) / 1e9
        fixed_line = {"value": whole_job_mlups(sites, a.steps, world, f_ms), "unit": "MLUPS",
                      "ms_per_step": f_kern, "dtype": "f64+i64", "kernel": "k_step_fix64",
                      "what": "float64 states; equilibrium and relaxation in 64-bit fixed point on the "
                              "integer pipes (float64 outside its range); same parity bars as FP64",
                      "roofline": {"bound": "hbm", "achieved": f_gbs, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                                   "frac": f_gbs / HBM_PEAK_GBS,
                                   "traffic": traffic("fp64fix", sites),
                                   "peak_source": HBM_PEAK_SOURCE},
                      "gpu_launches": a.steps, "clocks": fclk.summary()}

    # the propagate kernel alone (Table "propagate-kernel" of Sec. 4): a pure copy of every
    # population whose source is inside the fluid, timed over the same number of launches
    prop_line = None
    if separate:
        wall_entries = 0 if p.bc == lbm.BC_PERIODIC_Y else lx * sum(abs(v) for v in lbm.model()[3])
        prop_bytes = 2 * 8 * (37 * sites - wall_entries)
        pev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        prop(p, bufs[0], ftmp, stream)
        pev[0].record(stream)
        for k in range(a.steps):
            prop(p, bufs[k % 2], ftmp, stream)
        pev[1].record(stream)
        torch.cuda.synchronize()
        prop_ms = pev[0].elapsed_time(pev[1]) / a.steps
        gbs = prop_bytes / (prop_ms * 1e-3) / 1e9
        prop_line = {"kernel": "k_propagate_push_fp64" if a.variant == "push" else "k_propagate_fp64",
                     "ms": prop_ms, "bytes": prop_bytes, "achieved": gbs, "unit": "GB/s",
                     "frac": gbs / HBM_PEAK_GBS, "peak": HBM_PEAK_GBS}

    # the other forms of the step, each with its own roofline, clocks and baseline (one GPU:
    # they are per-GPU forms; the replicas of N > 1 report the headline only)
    forms = {}
    if (world == 1 and a.precision == "fp64" and a.variant == "fused" and not a.no_forms
            and (lx, ly) == (LX, LY)):
        del bufs, fa, fb, ftmp
        torch.cuda.empty_cache()
        forms["fp32"] = single_form(a, "fp32", dev)
        forms["fp32_conserved"] = single_form(a, "fp32c", dev)
        del dev
        torch.cuda.empty_cache()
        forms["batch_fp64"] = batch_form(a, "fp64")
        forms["batch_fp32"] = batch_form(a, "fp32")
        forms["adjoint"] = adjoint_form(a, repeats=3)

    if rank == 0:
        line = {"metric": "D2Q37 MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+i64+f64" if fp32 else ("f64+i64" if fix else "f64"),
                "data": "synthetic",
                "config": headline_config(lx, ly, a.variant, a.precision, world),
                "roofline": roofline, "e2e": e2e,
                **({"propagate_kernel": prop_line} if prop_line else {}),
                **({"fp64_fixed_relax": fixed_line} if fixed_line else {}),
                **forms,
                "gpu_launches": a.steps * (3 if separate else 1),
                "clocks": clk.summary()}
        if not a.no_cpu_baseline and world == 1 and (lx, ly) == (LX, LY):
            line["cpu_baseline"] = oracle_sample(16)   # ~14 s of CPU work on 16 cores
            # the same oracle on one thread, on a smaller crop (~5 s)
            line["cpu_baseline"]["single_thread"] = oracle_sample(4, cols=2, threads=1)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


DTYPE = {"fp32": "f32+i64+f64", "fp32c": "f32+i64+f64", "fp64fix": "f64+i64", "fp64": "f64"}


def prec_enum(lbm, precision):
    return {"fp32": lbm.FP32_SHIFTED, "fp32c": lbm.FP32_CONSERVED, "fp64fix": lbm.FP64_FIXED,
            "fp64": lbm.FP64}[precision]


def kernel_roofline(bound, work_per_site, sites, ms, kernel, traffic=None):
    """Roofline record of one kernel: algorithmic bytes (hbm) or flops (alu) per launch over
    its CUDA-event time, against the measured HBM copy rate or the FP64 unit-count peak."""
    if bound == "hbm":
        achieved = work_per_site * sites / (ms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": achieved, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                "frac": achieved / HBM_PEAK_GBS, "traffic": traffic, "kernel": kernel,
                "peak_source": HBM_PEAK_SOURCE}
    achieved = work_per_site * sites / (ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic, "kernel": kernel,
            "peak_source": "152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz"}


def single_form(a, precision, dev_fields):
    """One 4096 x 8192 lattice in another storage form (fp32 = FP32 shifted deviations):
    K steps timed with CUDA events, against its HBM roofline."""
    import torch

    from paper_1703_04594_gb300 import lbm

    p = lbm.Params(LX, LY, tau=TAU, gy=GY, t_bottom=T_BOTTOM, t_top=T_TOP,
                   precision={"fp32": lbm.FP32_SHIFTED, "fp32c": lbm.FP32_CONSERVED,
                              "fp64fix": lbm.FP64_FIXED}[precision])
    bufs = [lbm.empty_state(p), lbm.empty_state(p)]
    lbm.init(p, *dev_fields, bufs[0])
    stream = torch.cuda.current_stream()
    for k in range(a.warmup):
        lbm.step(p, bufs[k % 2], bufs[(k + 1) % 2], stream)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with ClockSampler(0) as clk:
        ev[0].record(stream)
        for k in range(a.steps):
            lbm.step(p, bufs[(a.warmup + k) % 2], bufs[(a.warmup + k + 1) % 2], stream)
        ev[1].record(stream)
        torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / a.steps
    sites = LX * LY
    fp32 = precision in ("fp32", "fp32c")
    kernel = {"fp32": "k_step_fp32", "fp32c": "k_step_fp32 (conserved moments)", "fp64fix": "k_step_fix64"}[precision]
    out = {"value": sites / (ms * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": ms, "steps": a.steps,
           "dtype": "f32+i64+f64" if fp32 else "f64+i64",
           "workload": f"{LX}x{LY} RT lattice, seed {SEED}",
           "roofline": kernel_roofline("hbm", BYTES_PER_SITE_FP32 if fp32 else BYTES_PER_SITE_FP64, sites, ms,
                                       kernel, traffic(precision, sites)),
           "gpu_launches": a.steps, "clocks": clk.summary()}
    del bufs
    torch.cuda.empty_cache()
    return out


def batch_lattices(kind, n, seed):
    """(lx, ly, tau, interface seed) of every lattice of a batched workload."""
    from paper_1703_04594_gb300 import inputs as I

    if kind == "small":
        return I.batch_workload(seed=seed, n=n, sizes=tuple(range(32, 129, 16)))
    return I.batch_workload(seed=seed, n=n)


def build_batch(kind, n, seed, precision):
    """Plans the batch, initialises every lattice from its own RT state (fields built on the
    GPU), autotunes on those states, re-initialises, and returns (batch, spec, params, fa,
    fb, tuned configuration)."""
    import torch

    from paper_1703_04594_gb300 import inputs as I
    from paper_1703_04594_gb300 import lbm

    prec = prec_enum(lbm, precision)
    spec = batch_lattices(kind, n, seed)
    params, fa, fb = [], [], []
    for lx, ly, tau, s in spec:
        p = lbm.Params(lx, ly, tau=tau, gy=GY, t_bottom=T_BOTTOM, t_top=T_TOP, precision=prec)
        params.append(p)
        fa.append(lbm.empty_state(p))
        fb.append(lbm.empty_state(p))

    def init_all():
        for (lx, ly, tau, s), p, t in zip(spec, params, fa):
            lbm.init(p, *[x.contiguous() for x in I.rt_state(lx, ly, s, t_bottom=T_BOTTOM, t_top=T_TOP,
                                                               g=abs(GY), device="cuda")], t)
        torch.cuda.synchronize()

    init_all()
    b = lbm.Batch(params, fa, fb)
    cfg = b.autotune(trial_steps=2)                  # advances the states: initialise again
    b.close()
    init_all()
    b = lbm.Batch(params, fa, fb)
    b.configure(cfg["mode"], cfg["tile_columns"], cfg["blocks_per_sm"])
    return b, spec, params, fa, fb, cfg


def time_batch(b, mode_cfg, steps, warmup, graph=False):
    """ms for `steps` steps of the batch in configuration mode_cfg = (mode, tile columns,
    blocks per SM); with graph=True the steps are one captured CUDA graph, replayed once."""
    import torch

    from paper_1703_04594_gb300 import lbm

    b.configure(*mode_cfg)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.run(2 * ((warmup + 1) // 2), s)            # even: the parity comes back
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if graph:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            b.run(steps, s)
        # the capture recorded the launches without running them; the batch's parity moved
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            e0.record(s)
            g.replay()
            e1.record(s)
    else:
        with torch.cuda.stream(s):
            e0.record(s)
            b.run(steps, s)
            e1.record(s)
    torch.cuda.synchronize()
    if b.status() != lbm.OK:
        raise RuntimeError("batched run reported a barrier timeout")
    return e0.elapsed_time(e1)


def batch_roofline(precision, sites, ms_step, cfg):
    from paper_1703_04594_gb300 import lbm

    kname = {"fp32": "fp32", "fp32c": "fp32 conserved", "fp64fix": "fix64", "fp64": "double"}[precision]
    kernel = ("k_batch_persistent<" if cfg["mode"] == lbm.BATCH_PERSISTENT else "k_batch_step<") + kname + ">"
    # the captures are of the per-step kernel
    tr = (traffic({"fp32": "batch_fp32", "fp64": "batch_fp64"}.get(precision, ""), sites)
          if cfg["mode"] == lbm.BATCH_PER_STEP else None)
    if precision == "fp64":
        return kernel_roofline("alu", FLOPS_PER_SITE_FP64, sites, ms_step, kernel, tr)
    return kernel_roofline("hbm", BYTES_PER_SITE_FP32 if precision in ("fp32", "fp32c") else BYTES_PER_SITE_FP64, sites,
                           ms_step, kernel, tr)


def batch_form(a, precision, kind="uneven", n=None, seed=4):
    """The batched workload at K steps in the autotuned configuration, against looping the
    single-lattice kernel over the lattices (both eager launches)."""
    import torch

    from paper_1703_04594_gb300 import lbm

    n = n or (1024 if kind == "small" else 256)
    b, spec, params, fa, fb, cfg = build_batch(kind, n, seed, precision)
    sites = b.sites()
    tuned = (cfg["mode"], cfg["tile_columns"], cfg["blocks_per_sm"])
    with ClockSampler(0) as clk:
        ms = time_batch(b, tuned, a.steps, a.warmup)
    ms_loop = time_batch(b, (lbm.BATCH_LOOP, 4, 0), a.steps, a.warmup)
    out = {"value": sites * a.steps / (ms * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": ms / a.steps,
           "steps": a.steps, "dtype": DTYPE[precision],
           "workload": (f"{len(spec)} RT lattices, " +
                        ("Lx in 32..128" if kind == "small" else "Lx in 128..1024") + ", Ly = 2 Lx, tau in [0.6, 1.0]"),
           "sites": sites, "autotuned": cfg,
           "loop_baseline": {"value": sites * a.steps / (ms_loop * 1e-3) / 1e6, "unit": "MLUPS",
                             "what": "single-lattice kernel launched per lattice per step"},
           "roofline": batch_roofline(precision, sites, ms / a.steps, cfg),
           "gpu_launches": a.steps if cfg["mode"] == lbm.BATCH_PER_STEP else 1, "clocks": clk.summary()}
    b.close()
    del fa, fb
    torch.cuda.empty_cache()
    return out


def run_batch(a):
    """Batched workload (one JSON line): Lx drawn by seed 4 from 128..1024 (or 32..128 with
    --batch-kind small), Ly = 2 Lx, tau ~ U[0.6, 1.0], own interface seeds.  The autotuned
    configuration, the persistent launch and the per-step launches each run --steps steps
    captured in one CUDA graph; the loop over the single-lattice kernel runs eagerly."""
    import torch

    from paper_1703_04594_gb300 import lbm

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    n = a.batch_n or (256 if a.batch_kind == "uneven" else 1024)
    b, spec, params, fa, fb, cfg = build_batch(a.batch_kind, n, 4 + rank, a.precision)
    sites = b.sites()
    tuned = (cfg["mode"], cfg["tile_columns"], cfg["blocks_per_sm"])
    with ClockSampler(local) as clk:
        ms = time_batch(b, tuned, a.steps, a.warmup, graph=True)
    modes = {}
    for name, mc in (("persistent_graph", (lbm.BATCH_PERSISTENT, cfg["tile_columns"], 0)),
                     ("per_step_graph", (lbm.BATCH_PER_STEP, cfg["tile_columns"], 0)),
                     ("per_step_eager", (lbm.BATCH_PER_STEP, cfg["tile_columns"], 0)),
                     ("loop_eager", (lbm.BATCH_LOOP, 4, 0))):
        t = time_batch(b, mc, a.steps, a.warmup, graph=name.endswith("graph"))
        modes[name] = {"MLUPS": sites * a.steps / (t * 1e-3) / 1e6, "ms_per_step": t / a.steps}
    value = sites * a.steps / (ms * 1e-3) / 1e6
    if rank == 0:
        line = {"metric": "D2Q37 MLUPS (batched)", "value": value, "unit": "MLUPS", "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": DTYPE[a.precision],
                "data": "synthetic",
                "config": {"workload": f"{len(spec)} RT lattices ({a.batch_kind}), Ly = 2 Lx, tau in [0.6, 1.0]",
                           "sites": sites, "precision": a.precision, "autotuned": cfg,
                           "timed": f"{a.steps} steps in one CUDA graph",
                           "l2": "states total >> 129 MB L2" if sites > 1e7 else "states partly L2-resident"},
                "modes": modes,
                "roofline": batch_roofline(a.precision, sites, ms / a.steps, cfg),
                "gpu_launches": a.steps if cfg["mode"] == lbm.BATCH_PER_STEP else 1,
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    b.close()


ADJ_LX, ADJ_LY, ADJ_N, ADJ_EVERY = 512, 1024, 500, 22
# algorithmic bytes per site of one adjoint step: the gathered f~ (37 x 8), lambda^{n+1}
# read (37 x 8) and lambda^n written (37 x 8)
BYTES_PER_SITE_ADJ = 888


def adjoint_step_ms(lx, ly, modes, warmup, calls):
    """The adjoint step alone (collide VJP with the transposed propagate as its store, wall
    slots, tau partials): CUDA events over back-to-back calls on a mid-run RT state (100
    steps in).  Returns (ms per call, clock summary)."""
    import torch

    from paper_1703_04594_gb300 import inputs as I
    from paper_1703_04594_gb300 import lbm

    p64 = lbm.Params(lx, ly, tau=TAU, gy=GY, t_bottom=T_BOTTOM, t_top=T_TOP)
    fields = [t.contiguous() for t in I.rt_fields(lx, ly, modes, T_BOTTOM, T_TOP, abs(GY), device="cuda")]
    f = lbm.empty_state(p64)
    lbm.init(p64, *fields, f)
    f = lbm.run(p64, f, lbm.empty_state(p64), 100).clone()
    lam = [lbm.empty_state(p64), lbm.empty_state(p64)]
    lbm.kinetic_energy_grad(p64, f, lam[0])
    work = lbm.adjoint_work(p64)
    dtau = torch.zeros((), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for k in range(warmup):
        lbm.adjoint_step(p64, f, lam[k % 2], lam[(k + 1) % 2], dtau, work, stream)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with ClockSampler(0) as aclk:
        ev[0].record(stream)
        for k in range(calls):
            lbm.adjoint_step(p64, f, lam[(warmup + k) % 2], lam[(warmup + k + 1) % 2], dtau, work, stream)
        ev[1].record(stream)
        torch.cuda.synchronize()
    return ev[0].elapsed_time(ev[1]) / calls, aclk.summary()


def run_adjoint_step(a):
    """The adjoint step kernel alone on an --lx x --ly RT lattice (default 512 x 1024): one
    JSON line with its time and HBM roofline (the profiling target of the adjoint)."""
    import torch

    from paper_1703_04594_gb300 import inputs as I

    torch.cuda.set_device(0)
    lx, ly = (a.lx, a.ly) if (a.lx, a.ly) != (LX, LY) else (ADJ_LX, ADJ_LY)
    ms, clk = adjoint_step_ms(lx, ly, I.rt_modes(lx, ly, 5), warmup=a.warmup, calls=a.steps)
    sites = lx * ly
    print(json.dumps({"metric": "D2Q37 adjoint step MLUPS", "value": sites / (ms * 1e-3) / 1e6, "unit": "MLUPS",
                      "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
                      "higher_is_better": True, "dtype": "f64+i64", "data": "synthetic",
                      "config": {"workload": f"lbm_adjoint_step on a {lx}x{ly} RT state"},
                      "roofline": kernel_roofline("hbm", BYTES_PER_SITE_ADJ, sites, ms,
                                                  "lbm_adjoint_step (k_adj_collide, then k_adj_walls with the fixed-order dL/dtau sum)",
                                                  traffic("adjoint", sites)),
                      "clocks": clk}), flush=True)


def adjoint_form(a, repeats, precision="fp64", seed=5):
    """dE/d(a_1..a_8, tau) of the total kinetic energy after 500 steps of a 512 x 1024 RT
    lattice, checkpoints every 22 steps, against the plain forward run; and the adjoint step
    kernel alone against its HBM roofline."""
    import torch

    from paper_1703_04594_gb300 import adjoint as A
    from paper_1703_04594_gb300 import inputs as I
    from paper_1703_04594_gb300 import lbm

    lx, ly, n, every = ADJ_LX, ADJ_LY, ADJ_N, ADJ_EVERY
    p = lbm.Params(lx, ly, tau=TAU, gy=GY, t_bottom=T_BOTTOM, t_top=T_TOP,
                   precision=lbm.FP64_FIXED if precision == "fp64fix" else lbm.FP64)
    modes = I.rt_modes(lx, ly, seed)

    # the fields are built on the device in both runs (the same torch operations; the
    # gradient's backward pass through them then runs there too)
    def forward_only():
        fields = [t.contiguous() for t in I.rt_fields(lx, ly, modes, T_BOTTOM, T_TOP, abs(GY), device="cuda")]
        f = lbm.empty_state(p)
        lbm.init(p, *fields, f)
        res = lbm.run(p, f, lbm.empty_state(p), n)
        return float(lbm.kinetic_energy(p, res))

    def gradient(every=every, recompute=None):
        amp = modes.a.clone().requires_grad_(True)
        tau = torch.tensor(TAU, dtype=torch.float64, requires_grad=True)
        fields = I.rt_fields(lx, ly, I.RTModes(a=amp, phi=modes.phi), T_BOTTOM, T_TOP, abs(GY), device="cuda")
        e = A.kinetic_energy_after(*[t.contiguous() for t in fields], tau, p, n, every, recompute_precision=recompute)
        e.backward()
        return amp.grad, tau.grad

    def one(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    def timed_against_forward(fn):
        """Mean times of fn and of the forward run, the two alternated `repeats` times (so
        that a drift of the GPU's speed over the run cancels in their ratio)."""
        fn()
        forward_only()
        tf = tg = 0.0
        for _ in range(repeats):
            tf += one(forward_only)
            tg += one(fn)
        return tg / repeats, tf / repeats

    # the default schedule, and the same gradient under two others: the segments recomputed
    # with the float64 step (the default recomputes them with the fixed-point relaxation),
    # and every state kept in HBM (no recomputation)
    with ClockSampler(0) as clk:
        t_grad, t_fwd = timed_against_forward(gradient)
    other = {"float64_recomputation": timed_against_forward(lambda: gradient(recompute=lbm.FP64)),
             "every_state_kept": timed_against_forward(lambda: gradient(every=1))}
    torch.cuda.empty_cache()
    schedules = {k: {"gradient_s": g, "forward_s": f, "gradient_over_forward": g / f} for k, (g, f) in other.items()}
    schedules["every_state_kept"]["memory_gb"] = (n + 1) * lbm.buffer_bytes(p) / 1e9
    ms_adj, aclk = adjoint_step_ms(lx, ly, modes, warmup=4, calls=40)
    sites = lx * ly
    return {"value": whole_job_mlups(sites, n, 1, t_grad * 1e3), "unit": "MLUPS",
            "what": "MLUPS of the whole gradient: forward run with checkpoints, then recomputation and the "
                    "adjoint step per segment, per site and forward step",
            "workload": f"dE/d(a_1..a_8, tau), E = kinetic energy after {n} steps of {lx}x{ly}, checkpoints "
                        f"every {every}", "repeats": repeats,
            "forward_steps": "fixed-point relaxation" if precision == "fp64fix" else "float64",
            "recomputed_steps": "fixed-point relaxation",
            "gradient_s": t_grad, "forward_s": t_fwd, "gradient_over_forward": t_grad / t_fwd,
            "forward_baseline": {"value": whole_job_mlups(sites, n, 1, t_fwd * 1e3), "unit": "MLUPS",
                                 "what": "the same 500 forward steps and the energy, no gradient"},
            "other_schedules": schedules,
            "adjoint_step_ms": ms_adj,
            "roofline": kernel_roofline("hbm", BYTES_PER_SITE_ADJ, sites, ms_adj,
                                        "lbm_adjoint_step (k_adj_collide, then k_adj_walls with the fixed-order dL/dtau sum)",
                                        traffic("adjoint", sites)),
            "clocks": clk.summary(), "adjoint_step_clocks": aclk}


def run_adjoint(a):
    """Differentiation workload (one JSON line): the gradient of the kinetic energy after 500
    steps of a 512 x 1024 RT lattice (seed 5), checkpoints every 22 steps."""
    import torch

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    r = adjoint_form(a, repeats=max(1, a.steps), precision=a.precision, seed=5 + rank)
    if rank == 0:
        line = {"metric": "D2Q37 MLUPS (gradient: forward + checkpointed adjoint)", "value": r["value"],
                "unit": "MLUPS", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
                "ms_per_step": r["gradient_s"] * 1e3 / ADJ_N, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64+i64" if a.precision == "fp64fix" else "f64",
                "data": "synthetic",
                "config": {"workload": r["workload"], "checkpoint_every": ADJ_EVERY, "repeats": r["repeats"],
                           "forward_steps": r["forward_steps"], "recomputed_steps": r["recomputed_steps"]},
                **{k: r[k] for k in ("forward_s", "gradient_s", "gradient_over_forward", "forward_baseline",
                                     "other_schedules", "adjoint_step_ms", "roofline", "clocks")}}
        print(json.dumps(line), flush=True)


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "batch":
        run_batch(a)
    elif a.workload == "adjoint":
        run_adjoint(a)
    elif a.workload == "adjoint-step":
        run_adjoint_step(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
