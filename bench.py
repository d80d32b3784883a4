#!/usr/bin/env python
"""Throughput of the GB300 D2Q37 thermal lattice-Boltzmann step, in MLUPS.

Workload: one 4096 x 8192 lattice (33,554,432 fluid sites), periodic in x, thermal
walls T = 1.15 (bottom) / 0.85 (top), tau = 0.8, g = 1e-4 in -y, Rayleigh-Taylor
initial state from seed 2 (synthetic; the paper's convective-turbulence workload
shape).  One bench step = one fused propagate + bc + collide pass over the whole
lattice (one kernel launch).  Each state buffer is 9.9 GB, far larger than the 129 MB
L2, so no L2 flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--variant fused|separate|push|aos|psoa|caosoa]
    python bench.py --impl reference      # the float64 CPU oracle on a bounded sample

Under torchrun (N > 1) every rank steps its own replica lattice (independent problems:
weak scaling, no collective on the data path); rank 0 prints one JSON line.
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

# Algorithmic work per site of the fused FP64 step (counted from the factored
# formulation in csrc/collide_fp64.cuh; FMA = 2 flops):
#   138 add + 97 mul + 138 fma + 1 div = 512 flops, 374 FP64-pipe operations.
FLOPS_PER_SITE_FP64 = 512
BYTES_PER_SITE_FP64 = 592          # 37 x 8 B read + 37 x 8 B written
BYTES_PER_SITE_FP32 = 296          # 37 x 4 B read + 37 x 4 B written
# FP64 peak from unit counts and clocks: 152 SMs x 2 DFMA/clk/SM x 2 flops x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum from an ncu capture
# of the current kernel on a smaller lattice, scaled to 4096 x 8192 by the site count;
# profiles/ holds the captures).  None where no capture of the current kernel exists: the
# float64 and fixed-point steps gained the moments' range check (integer instructions, the
# same memory accesses) after their captures (18.13 GB and 19.10 GB per launch then).
TRAFFIC_BYTES_PER_LAUNCH = {"fused": None, "separate": None, "fp32": 9.16e9, "fp64fix": None}


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
    ap.add_argument("--precision", choices=["fp64", "fp32", "fp64fix"], default="fp64",
                    help="fp32 = FP32 shifted-deviation storage (fused only); fp64fix = float64 storage "
                         "with the fixed-point relaxation (fused only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fixed", action="store_true",
                    help="skip the extra timing of the fixed-point-relaxation FP64 step")
    ap.add_argument("--workload", choices=["single", "batch", "adjoint"], default="single",
                    help="batch = 256 independent lattices of uneven sizes; adjoint = gradient of the "
                         "kinetic energy after 500 steps of a 512x1024 lattice (checkpoints every 22)")
    ap.add_argument("--batch-n", type=int, default=256)
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
def oracle_sample(steps: int, cols: int = 16):
    """Time the float64 CPU oracle on a bounded crop of the same workload: ``cols`` full-
    height columns (cols x 8192 sites) of the seed-2 Rayleigh-Taylor lattice."""
    import torch

    from oracle import lbm as OL
    from paper_1703_04594_gb300 import inputs as I

    modes = I.rt_modes(LX, LY, SEED)
    fields = [t[:cols].contiguous() for t in I.rt_fields(LX, LY, modes, T_BOTTOM, T_TOP, abs(GY))]
    p = OL.Params(cols, LY, tau=TAU, gy=GY, t_bottom=T_BOTTOM, t_top=T_TOP)
    f = OL.init_equilibrium(*fields)
    t0 = time.perf_counter()
    for _ in range(steps):
        f = OL.step(f, p)
    dt = time.perf_counter() - t0
    return {"value": cols * LY * steps / dt / 1e6, "unit": "MLUPS", "cores": torch.get_num_threads(),
            "kind": "oracle",
            "sample": f"{cols}x{LY} column crop of the {LX}x{LY} seed-{SEED} RT lattice, {steps} steps, "
                      f"{dt:.1f} s"}


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
            "config": {"workload": f"D2Q37 FP64 step, {LX}x{LY} RT lattice (oracle on a bounded crop)",
                       "lx": LX, "ly": LY, "tau": TAU, "gy": GY},
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
    fp32 = a.precision == "fp32"
    fix = a.precision == "fp64fix"
    if (fp32 or fix) and a.variant != "fused":
        raise SystemExit(f"--precision {a.precision} supports the fused step only")
    p = lbm.Params(lx, ly, tau=TAU, gy=GY, t_bottom=T_BOTTOM, t_top=T_TOP,
                   precision=lbm.FP32_SHIFTED if fp32 else (lbm.FP64_FIXED if fix else lbm.FP64))
    sites = lx * ly
    fields = I.rt_state(lx, ly, SEED + rank, t_bottom=T_BOTTOM, t_top=T_TOP, g=abs(GY))
    dev = [t.contiguous().cuda() for t in fields]
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
                    "frac": achieved / HBM_PEAK_GBS, "traffic": TRAFFIC_BYTES_PER_LAUNCH.get(a.precision),
                    "kernel": "k_step_fp32" if fp32 else "k_step_fix64",
                    "peak_source": HBM_PEAK_SOURCE}
    else:
        achieved = FLOPS_PER_SITE_FP64 * sites / (kern_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_PEAK_TFLOPS, "traffic": TRAFFIC_BYTES_PER_LAUNCH.get(a.variant),
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
                                   "traffic": TRAFFIC_BYTES_PER_LAUNCH.get("fp64fix"),
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

    if rank == 0:
        line = {"metric": "D2Q37 MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+i64+f64" if fp32 else ("f64+i64" if fix else "f64"),
                "data": "synthetic",
                "config": {"workload": f"D2Q37 {'FP32-shifted' if fp32 else ('FP64 fixed-point-relax' if fix else 'FP64')} "
                                       f"{a.variant} step, "
                                       f"{lx}x{ly} Rayleigh-Taylor lattice",
                           "lx": lx, "ly": ly, "tau": TAU, "gy": GY, "t_bottom": T_BOTTOM, "t_top": T_TOP,
                           "seed": SEED, "variant": a.variant,
                           "precision": a.precision,
                           "l2": "state buffers >= 4.9 GB >> 129 MB L2; no flush needed",
                           "parallelism": f"replicas x{world}"},
                "roofline": roofline, "e2e": e2e,
                **({"propagate_kernel": prop_line} if prop_line else {}),
                **({"fp64_fixed_relax": fixed_line} if fixed_line else {}),
                "gpu_launches": a.steps * (3 if separate else 1),
                "clocks": clk.summary()}
        if not a.no_cpu_baseline and world == 1 and (lx, ly) == (LX, LY):
            line["cpu_baseline"] = oracle_sample(16)   # ~14 s of CPU work on 16 cores
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_batch(a):
    """Batched form: independent RT lattices (Lx in 128..1024 step 64 drawn by seed 4,
    Ly = 2 Lx, tau ~ U[0.6, 1.0], own interface seeds) stepped by one persistent launch
    (autotuned), against looping the single-lattice kernel over the lattices."""
    import torch

    from paper_1703_04594_gb300 import inputs as I
    from paper_1703_04594_gb300 import lbm

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    fp32 = a.precision == "fp32"
    fix = a.precision == "fp64fix"
    prec = lbm.FP32_SHIFTED if fp32 else (lbm.FP64_FIXED if fix else lbm.FP64)
    spec = I.batch_workload(seed=4 + rank, n=a.batch_n)
    params, fa, fb = [], [], []
    for lx, ly, tau, s in spec:
        p = lbm.Params(lx, ly, tau=tau, gy=GY, t_bottom=T_BOTTOM, t_top=T_TOP, precision=prec)
        params.append(p)
        fa.append(lbm.empty_state(p))
        fb.append(lbm.empty_state(p))
    b = lbm.Batch(params, fa, fb)
    cfg = b.autotune(trial_steps=2)                       # on the not-yet-initialised buffers
    for (lx, ly, tau, s), p, t in zip(spec, params, fa):
        dev = [x.contiguous().cuda() for x in I.rt_state(lx, ly, s, t_bottom=T_BOTTOM, t_top=T_TOP, g=abs(GY))]
        lbm.init(p, *dev, t)
    b.close()
    b = lbm.Batch(params, fa, fb)
    b.configure(cfg["mode"], cfg["tile_columns"], cfg["blocks_per_sm"])
    sites = b.sites()
    stream = torch.cuda.current_stream()

    def timed(mode_cfg, steps):
        b.configure(*mode_cfg)
        b.run(a.warmup, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.run(steps, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if b.status() != lbm.OK:
            raise RuntimeError("batched run reported a barrier timeout")
        return e0.elapsed_time(e1)

    with ClockSampler(local) as clk:
        ms = timed((cfg["mode"], cfg["tile_columns"], cfg["blocks_per_sm"]), a.steps)
    ms_loop = timed((lbm.BATCH_LOOP, 4, 0), a.steps)
    value = sites * a.steps / (ms * 1e-3) / 1e6
    bytes_site = BYTES_PER_SITE_FP32 if fp32 else BYTES_PER_SITE_FP64
    kind = "fp32" if fp32 else ("fix64" if fix else "fp64")
    if fp32 or fix:
        achieved = bytes_site * sites * a.steps / (ms * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                    "frac": achieved / HBM_PEAK_GBS, "traffic": None, "peak_source": HBM_PEAK_SOURCE,
                    "kernel": ("k_batch_persistent<" if cfg["mode"] == lbm.BATCH_PERSISTENT
                               else "k_batch_step<") + kind + ">"}
    else:
        achieved = FLOPS_PER_SITE_FP64 * sites * a.steps / (ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                    "kernel": ("k_batch_persistent<double>" if cfg["mode"] == lbm.BATCH_PERSISTENT
                               else "k_batch_step<double>")}
    if rank == 0:
        line = {"metric": "D2Q37 MLUPS (batched)", "value": value, "unit": "MLUPS", "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+i64+f64" if fp32 else ("f64+i64" if fix else "f64"),
                "data": "synthetic",
                "config": {"workload": f"{len(spec)} RT lattices, Lx in 128..1024, Ly = 2 Lx, tau in [0.6, 1.0]",
                           "sites": sites, "precision": a.precision, "autotuned": cfg,
                           "l2": "states total >> 129 MB L2"},
                "loop_baseline": {"value": sites * a.steps / (ms_loop * 1e-3) / 1e6, "unit": "MLUPS",
                                  "what": "single-lattice kernel launched per lattice per step"},
                "roofline": roofline, "gpu_launches": a.steps if cfg["mode"] == lbm.BATCH_PER_STEP else 1,
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    b.close()


def run_adjoint(a):
    """Differentiation workload: dE/d(a_1..a_8, tau) of the total kinetic energy after 500
    FP64 steps of a 512 x 1024 RT lattice (seed 5), checkpoints every 22 steps, against the
    plain forward run of the same 500 steps."""
    import torch

    from paper_1703_04594_gb300 import adjoint as A
    from paper_1703_04594_gb300 import inputs as I
    from paper_1703_04594_gb300 import lbm

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    lx, ly, n, every, seed = 512, 1024, 500, 22, 5 + rank
    fix = a.precision == "fp64fix"   # forward steps with the fixed-point relaxation
    p = lbm.Params(lx, ly, tau=TAU, gy=GY, t_bottom=T_BOTTOM, t_top=T_TOP,
                   precision=lbm.FP64_FIXED if fix else lbm.FP64)
    modes = I.rt_modes(lx, ly, seed)

    def forward_only():
        fields = [t.contiguous().cuda() for t in I.rt_fields(lx, ly, modes, T_BOTTOM, T_TOP, abs(GY))]
        f = lbm.empty_state(p)
        lbm.init(p, *fields, f)
        res = lbm.run(p, f, lbm.empty_state(p), n)
        return float(lbm.kinetic_energy(p, res))

    def gradient():
        amp = modes.a.clone().requires_grad_(True)
        tau = torch.tensor(TAU, dtype=torch.float64, requires_grad=True)
        fields = I.rt_fields(lx, ly, I.RTModes(a=amp, phi=modes.phi), T_BOTTOM, T_TOP, abs(GY))
        e = A.kinetic_energy_after(*[t.cuda() for t in fields], tau, p, n, every)
        e.backward()
        return amp.grad, tau.grad

    for _ in range(max(1, a.warmup)):
        forward_only()
        gradient()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            forward_only()
        torch.cuda.synchronize()
        t_fwd = max_over_ranks((time.perf_counter() - t0) / a.steps, "cuda")
        t0 = time.perf_counter()
        for _ in range(a.steps):
            gradient()
        torch.cuda.synchronize()
        t_grad = max_over_ranks((time.perf_counter() - t0) / a.steps, "cuda")
    if rank == 0:
        sites = lx * ly
        line = {"metric": "D2Q37 MLUPS (gradient: forward + checkpointed adjoint)",
                "value": whole_job_mlups(sites, n, world, t_grad * 1e3), "unit": "MLUPS", "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": t_grad * 1e3 / n, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64+i64" if fix else "f64",
                "data": "synthetic",
                "config": {"workload": f"dE/d(a_1..a_8, tau), E = kinetic energy after {n} steps of {lx}x{ly}",
                           "checkpoint_every": every, "repeats": a.steps,
                           "forward_steps": "fixed-point relaxation" if fix else "float64"},
                "forward_s": t_fwd, "gradient_s": t_grad, "gradient_over_forward": t_grad / t_fwd,
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "batch":
        run_batch(a)
    elif a.workload == "adjoint":
        run_adjoint(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
