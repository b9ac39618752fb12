#!/usr/bin/env python
"""Benchmark of the WENO5-CT MHD step (libw5ct) on one GB300.

Workload (default): 256^3 periodic box, uniform rho = 1, beta = 1 mean field
along x, solenoidal Gaussian random-phase velocity with a k^-5/3 spectrum
for 2 <= |k| <= 32 at rms Mach 1 (seed 1812), divergence-free field
perturbation of 10% rms from an edge vector potential (seed 1813); WENO-Z,
CFL 0.8, dt from the device CFL reduction every step.  The state (>= 4 GB)
is far larger than L2, so no L2 flush is needed between steps.

One JSON line: `value` = FP64 zone-updates/s (the paper's 8-byte
arithmetic); `fp32_bulk` = the FP32-bulk form (float flux arithmetic,
double accumulation) with its L1 error against the FP64 run after the same
steps at the same dt sequence.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference] [--n 256]

With N > 1 (torchrun) every rank advances its own independent replica
("replicas only": the path has no data exchange) and the slowest rank's time
is used.  --impl reference times the CPU oracle on the host cores on the
same 256^3 workload (K whole steps, about 10 s each on 16 cores).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic flop counts per WENO variant (0 = JS, 1 = Z), from the
# oracle's own source compiled with a counting scalar type
# (oracle/flopcount.cpp; +, -, *, / and sqrt count 1; negation,
# comparisons, max and |x| count 0; tests/test_flop_count.py rebuilds the
# counter and checks these numbers): per cell of one sweep (primitives,
# flux, three speeds), per interface of one sweep (interface average,
# Appendix A eigensystem, 6-point projection of F and q onto 7 fields, LF
# split and two phi_N per field, back-projection), the two CT transport
# fluxes that the sweep kernel forms at each interface (Eqs. fct1-fct6), and
# per zone-update of the whole RK4 + CT step.
CELL_FLOPS = 93
FACE_FLOPS = {0: 2760, 1: 2858}
CT_FLUX_FLOPS = 10
SWEEP_FLOPS_PER_ZONE = {v: CELL_FLOPS + FACE_FLOPS[v] + CT_FLUX_FLOPS for v in (0, 1)}
STEP_FLOPS_PER_ZONE = {0: 34881, 1: 36057}
# The vector-Jacobian product of one step, per zone: the step's forward
# operations (its stages recomputed once) plus the reverse-mode operations of
# differentiating it with respect to its input state, counted by the same
# program operation by operation (each partial contribution costs its
# multiplications / divisions plus one accumulating addition; operations on
# values that do not depend on the state cost nothing in reverse).
ADJOINT_STEP_FLOPS_PER_ZONE = {0: 129072, 1: 132768}
# Peaks: FP32 from the unit counts (152 SMs x 128 FMA lanes x 2 flop x 2.07 GHz);
# FP64 from the published GB300 rate (1.25 TFLOP/s); measured copy bandwidth.
PEAK_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
PEAK_FP64_TFLOPS = 1.25


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None, help="timed steps (default per workload)")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--n", type=int, default=None, help="box edge (default per workload)")
    p.add_argument("--e2e-steps", type=int, default=5)
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-sub-records", action="store_true",
                   help="default workload only: skip the compact batched and adjoint records")
    p.add_argument("--cpu-steps", type=int, default=2, help="oracle steps of the cpu_baseline leg")
    p.add_argument("--workload", default="turb", choices=["turb", "blast", "wave", "batched", "adjoint"],
                   help="turb: 256^3 turbulence, 50 steps (default); blast: 512^3 blast in Mach-5 turbulence, "
                        "100 steps; wave: the 32^3 fast eigenmode, 20 steps; batched: 512 uneven patches, "
                        "10 steps; adjoint: 64^3 rollout gradient, 10 steps")
    p.add_argument("--err-steps", type=int, default=5, help="FP64 steps of the blast error statement")
    p.add_argument("--patches", type=int, default=512, help="patches of the batched workload")
    args = p.parse_args(argv)
    n, steps = WORKLOAD_DEFAULTS[args.workload]
    if args.n is None:
        args.n = n
    if args.steps is None:
        args.steps = steps
    return args


# box edge and timed steps of each workload when not given
WORKLOAD_DEFAULTS = {"turb": (256, 50), "blast": (512, 100), "wave": (32, 20), "batched": (256, 10),
                     "adjoint": (64, 10)}


def workload_config(n):
    return {
        "workload": f"periodic {n}^3 MHD turbulence: rho=1, beta=1 mean B along x, k^-5/3 solenoidal velocity "
                    f"2<=|k|<=32 at rms Mach 1 (seed 1812), 10% rms div-free dB (seed 1813); WENO-Z, CFL 0.8, "
                    f"gamma 5/3, dt from the CFL reduction each step",
        "zones": n ** 3,
        "grid": [n, n, n],
        "l2_policy": "state larger than L2 (>= 4 GB), no flush",
        "parallelism": "replicas",
    }


def make_ic(n):
    """The workload's initial state (2 <= |k| <= 32 at 256^3; boxes too small
    to hold |k| = 32 keep the modes below their Nyquist wavenumber)."""
    from paper_1812_04278_gb300 import inputs
    return inputs.turbulent_state(n, seed=1812, seed_b=1813, mach=1.0, beta=1.0, dB_frac=0.1, kmin=2,
                                  kmax=min(32, n // 2 - 1))


# ------------------------------------------------------------------ clocks


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            try:
                pw.append(float(parts[3]))
            except ValueError:
                pass
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm), "power_w": float(np.median(pw)) if pw else None}


# ------------------------------------------------------------------ helpers


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("w5ct_physics.cuh", "w5ct_kernels.cuh", "w5ct_internal.h", "w5ct_sweep32.cu", "w5ct_sweep64.cu",
              "w5ct_sweep64dw.cu"):
        h.update(open(os.path.join(ROOT, "paper_1812_04278_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


# DRAM bytes (read + write) per zone of one sweep launch, from ncu captures
# at 128^3 (dram__bytes_read.sum + dram__bytes_write.sum / 128^3), valid for
# the sweep source with the given hash; scaled to a launch by the zone count
# (traffic grows with the zones: one tile pass per zone).
SWEEP_TRAFFIC = {"src": "94dd87415640b72f", "fp64": 103.51, "fp32": 43.84, "fp64dw": 105.32}


def hbm_gbs(traffic, launch_ms):
    """Achieved DRAM bandwidth of a launch moving `traffic` bytes (None when
    the traffic is unknown)."""
    return None if traffic is None else traffic / (launch_ms * 1e-3) / 1e9


def sweep_traffic(key, zones):
    if SWEEP_TRAFFIC.get("src") != kernel_source_hash() or key not in SWEEP_TRAFFIC:
        return None
    return SWEEP_TRAFFIC[key] * zones


def conservation_drift(s, cons, bface, dx):
    """Largest change of the eight volume totals (mass, momentum, energy,
    face field) of a periodic run from its initial state, relative to the
    volume integral of |state|."""
    dv = dx[0] * dx[1] * dx[2]
    tot0 = np.concatenate([cons.reshape(5, -1).sum(axis=1), bface.reshape(3, -1).sum(axis=1)]) * dv
    scale = (np.abs(cons).sum() + np.abs(bface).sum()) * dv
    return float(np.abs(s.conserved_totals() - tot0).max() / scale)


def l1_error(a_cons, a_b, b_cons, b_b):
    """Geometric L1 norm over the state components (Sec. 4 of the paper)."""
    n = a_cons[0].size
    comps = [np.abs(a_cons[f] - b_cons[f]).sum() / n for f in range(5)] + \
            [np.abs(a_b[f] - b_b[f]).sum() / n for f in range(3)]
    return float(np.sqrt(np.sum(np.square(comps))))


def max_over_ranks_of(x, dist, device):
    """The largest value of x over all ranks (the slowest replica's time)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, zones, steps, ms):
    """Whole-job zone-updates/s of `world` independent replicas of `zones`
    cells advanced `steps` steps in `ms` milliseconds (the slowest rank)."""
    return world * zones * steps / (ms * 1e-3)


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "native" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local, dist


# ------------------------------------------------------------------ reference arm


def oracle_timed_steps(oracle, o, nsteps):
    """Seconds of each of nsteps oracle steps, dt from the oracle's own CFL
    reduction (timed with the step, as on the GPU)."""
    times = []
    for _ in range(nsteps):
        t0 = time.perf_counter()
        o.step(o.cfl_dt())
        times.append(time.perf_counter() - t0)
    return times


def run_reference(args):
    """The oracle, as it stands, on the host cores, on the workload the line
    names: the full n^3 turbulence box (the same initial state as the native
    arm), `steps` whole RK4 + CT steps timed.  Warm-up on the CPU only pages
    memory in, so one untimed step is run instead of `warmup` (the line says
    so); at about 10 s per 256^3 step on 16 cores the run takes ~4 minutes."""
    world, rank, local, dist = dist_setup(args)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    import oracle
    oracle.build()
    n = args.n
    cons, bface = make_ic(n)
    o = oracle.Oracle((n, n, n), 1.0 / n, oracle.make_config(weno_variant=oracle.WENO_Z))
    o.set_state(cons, bface)
    warm = 1 if args.warmup > 0 else 0
    oracle_timed_steps(oracle, o, warm)
    times = oracle_timed_steps(oracle, o, args.steps)
    el = sum(times)
    value = n ** 3 * args.steps / el
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": "zone-updates/s (3D WENO5-CT MHD, full RK4 step)", "value": value,
        "unit": "zone-updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": warm,
        "warmup_requested": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(n),
        "cpu_baseline": {"value": value, "unit": "zone-updates/s", "cores": cores, "kind": "oracle",
                         "sample": f"the {n}^3 workload itself, {args.steps} full steps after {warm} untimed",
                         "step_seconds_min_max": [min(times), max(times)], "cpu_model": cpu_model(),
                         "nproc": os.cpu_count()},
        "e2e": {"value": value, "unit": "zone-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------------ native arm


def timed_run(torch, w5, shape, dx, cons_d, bface_d, precision, steps, warmup, dt_log=None, sampler=None,
              barrier=None, variant=1, floors=0):
    stream = torch.cuda.current_stream()
    s = w5.Solver(shape, dx, w5.make_config(precision=precision, weno_variant=variant, floors=floors),
                  stream=stream.cuda_stream)
    s.set_state(cons_d, bface_d)
    for k in range(warmup):
        s.step_cfl(None if dt_log is None else dt_log[k:k + 1])
    torch.cuda.synchronize()
    if barrier:
        barrier()
    launches0 = w5.w5ct_launch_count(s.ctx)
    w5.w5ct_set_timing(s.ctx, True)
    if sampler:
        sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(steps):
        s.step_cfl(None if dt_log is None else dt_log[warmup + k:warmup + k + 1])
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    ms = e0.elapsed_time(e1)
    nsweep, sweep_ms = w5.w5ct_sweep_timing(s.ctx)
    w5.w5ct_set_timing(s.ctx, False)
    launches = w5.w5ct_launch_count(s.ctx) - launches0
    return s, ms, nsweep, sweep_ms, launches, clocks


def run_native(args):
    import torch
    world, rank, local, dist = dist_setup(args)
    torch.cuda.set_device(local)
    from paper_1812_04278_gb300 import build
    build.build()
    from paper_1812_04278_gb300 import w5ct as w5

    n = args.n
    shape = (n, n, n)
    dx = (1.0 / n,) * 3
    zones = n ** 3
    cons, bface = make_ic(n)
    cons_d = torch.from_numpy(cons).cuda()
    bface_d = torch.from_numpy(bface).cuda()
    barrier = (lambda: dist.barrier()) if dist is not None else None

    def max_over_ranks(x):
        return max_over_ranks_of(x, dist, "cuda")

    # ---- FP64 (headline)
    nlog = args.warmup + args.steps
    dt_log = torch.zeros(nlog, dtype=torch.float64, device="cuda")
    sampler = ClockSampler(local) if rank == 0 else None
    s64, ms64, nsw64, swms64, launches64, clocks = timed_run(torch, w5, shape, dx, cons_d, bface_d, w5.W5CT_FP64,
                                                             args.steps, args.warmup, dt_log, sampler, barrier)
    ms64 = max_over_ranks(ms64)
    c64 = torch.empty_like(cons_d)
    b64 = torch.empty_like(bface_d)
    w5.w5ct_get_state(s64.ctx, c64, b64, None, 1)
    divb64 = s64.div_b_norm()[0]
    drift64 = conservation_drift(s64, cons, bface, dx)
    s64.close()

    # ---- FP64 with the WENO part in double-word arithmetic: timed like the
    # FP64 run, then its deviation from the FP64 state at the FP64 run's dt
    # sequence
    sdw, msdw, nswdw, swmsdw, launchesdw, _ = timed_run(torch, w5, shape, dx, cons_d, bface_d, w5.W5CT_FP64_DW,
                                                        args.steps, args.warmup, None, None, barrier)
    msdw = max_over_ranks(msdw)
    sdw.set_state(cons_d, bface_d)
    for k in range(nlog):
        w5.w5ct_step_dev(sdw.ctx, dt_log[k:k + 1])
    cdw = torch.empty_like(cons_d)
    bdw = torch.empty_like(bface_d)
    w5.w5ct_get_state(sdw.ctx, cdw, bdw, None, 1)
    divbdw = sdw.div_b_norm()[0]
    sdw.close()
    reldw = float(max((cdw - c64).abs().max().item(), (bdw - b64).abs().max().item()) /
                  max(c64.abs().max().item(), b64.abs().max().item()))
    del cdw, bdw

    # ---- FP32-bulk
    s32, ms32, nsw32, swms32, launches32, _ = timed_run(torch, w5, shape, dx, cons_d, bface_d, w5.W5CT_FP32_BULK,
                                                        args.steps, args.warmup, None, None, barrier)
    ms32 = max_over_ranks(ms32)
    # error pass: same IC and the FP64 run's dt sequence
    s32.set_state(cons_d, bface_d)
    for k in range(nlog):
        w5.w5ct_step_dev(s32.ctx, dt_log[k:k + 1])
    c32 = torch.empty_like(cons_d)
    b32 = torch.empty_like(bface_d)
    w5.w5ct_get_state(s32.ctx, c32, b32, None, 1)
    divb32 = s32.div_b_norm()[0]
    drift32 = conservation_drift(s32, cons, bface, dx)
    s32.close()
    c64h, b64h, c32h, b32h = (t.cpu().numpy() for t in (c64, b64, c32, b32))
    l1 = l1_error(c32h, b32h, c64h, b64h)
    l1_ref = l1_error(c64h, b64h, cons, bface)     # how far the FP64 state moved
    relmax = float(max(np.abs(c32h - c64h).max(), np.abs(b32h - b64h).max()) /
                   max(np.abs(c64h).max(), np.abs(b64h).max()))
    del c64, b64, c32, b32

    # ---- WENO-JS, both forms, same steps (the robust variant)
    sjs, msjs, _, _, _, _ = timed_run(torch, w5, shape, dx, cons_d, bface_d, w5.W5CT_FP64, args.steps, args.warmup,
                                      None, None, barrier, variant=w5.W5CT_WENO_JS)
    sjs.close()
    fjs, msfjs, _, _, _, _ = timed_run(torch, w5, shape, dx, cons_d, bface_d, w5.W5CT_FP32_BULK, args.steps,
                                       args.warmup, None, None, barrier, variant=w5.W5CT_WENO_JS)
    fjs.close()
    msjs, msfjs = max_over_ranks(msjs), max_over_ranks(msfjs)

    # ---- end to end through the C ABI with host buffers (FP64)
    e2e_steps = max(1, min(args.e2e_steps, args.steps))
    hc = torch.from_numpy(cons).pin_memory()
    hb = torch.from_numpy(bface).pin_memory()
    oc = torch.empty_like(hc).pin_memory()
    ob = torch.empty_like(hb).pin_memory()
    se = w5.Solver(shape, dx, w5.make_config(precision=w5.W5CT_FP64), stream=torch.cuda.current_stream().cuda_stream)
    w5.w5ct_set_state(se.ctx, hc.data_ptr(), hb.data_ptr(), 0)
    se.step_cfl()
    w5.w5ct_get_state(se.ctx, oc.data_ptr(), ob.data_ptr(), None, 0)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    e2e_sampler = ClockSampler(local) if rank == 0 else None
    if e2e_sampler:
        e2e_sampler.start()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        w5.w5ct_set_state(se.ctx, hc.data_ptr(), hb.data_ptr(), 0)
        se.step_cfl()
        w5.w5ct_get_state(se.ctx, oc.data_ptr(), ob.data_ptr(), None, 0)
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e_clocks = e2e_sampler.stop() if e2e_sampler else None
    se.close()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    peaks = load_peaks()
    value64 = replica_throughput(world, zones, args.steps, ms64)
    value32 = replica_throughput(world, zones, args.steps, ms32)
    sweep_flops = SWEEP_FLOPS_PER_ZONE[1] * zones
    ach64 = sweep_flops / (swms64 / nsw64 * 1e-3) / 1e12
    ach32 = sweep_flops / (swms32 / nsw32 * 1e-3) / 1e12
    achdw = sweep_flops / (swmsdw / nswdw * 1e-3) / 1e12
    valuedw = replica_throughput(world, zones, args.steps, msdw)
    line = {
        "metric": "zone-updates/s (3D WENO5-CT MHD, full RK4 step)",
        "value": value64,
        "unit": "zone-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms64 / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(n),
        "roofline": {"kernel": "sweep_kernel (FP64)", "bound": "alu", "achieved": ach64, "peak": PEAK_FP64_TFLOPS,
                     "unit": "TFLOP/s", "frac": ach64 / PEAK_FP64_TFLOPS,
                     "traffic": sweep_traffic("fp64", zones), "launch_ms": swms64 / nsw64,
                     "algorithmic_flops_per_launch": sweep_flops,
                     "hbm_gbs": hbm_gbs(sweep_traffic("fp64", zones), swms64 / nsw64),
                     "hbm_peak_gbs": peaks.get("hbm_gbs"),
                     "step_tflops": STEP_FLOPS_PER_ZONE[1] * value64 / world / 1e12,
                     "peak_source": "GB300 FP64 unit count: 152 SMs x 2 DFMA/clk x 2 x 2.07 GHz = 1.26; "
                                    "published 1.25 TFLOP/s (probe measured 1.0 TFLOP/s DFMA)"},
        "fp32_bulk": {
            "value": value32, "unit": "zone-updates/s", "ms_per_step": ms32 / args.steps, "dtype": "f32",
            "accumulate": "f64", "speedup_vs_fp64": value32 / value64,
            "l1_vs_fp64": l1, "l1_fp64_change": l1_ref, "max_rel_vs_fp64": relmax, "div_b_linf": divb32,
            "conservation_drift": drift32,
            "error_steps": nlog,
            "roofline": {"kernel": "sweep_kernel (FP32)", "bound": "alu", "achieved": ach32,
                         "peak": PEAK_FP32_TFLOPS, "unit": "TFLOP/s", "frac": ach32 / PEAK_FP32_TFLOPS,
                         "traffic": sweep_traffic("fp32", zones), "launch_ms": swms32 / nsw32,
                         "hbm_gbs": hbm_gbs(sweep_traffic("fp32", zones), swms32 / nsw32),
                         "step_tflops": STEP_FLOPS_PER_ZONE[1] * value32 / world / 1e12,
                         "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"},
            "gpu_launches": launches32,
        },
        "fp64_dw": {
            "value": valuedw, "unit": "zone-updates/s", "ms_per_step": msdw / args.steps,
            "dtype": "f64; WENO indicators, weights and interpolants in double-word f32 pairs (48-bit significand)",
            "speedup_vs_fp64": valuedw / value64, "max_rel_vs_fp64": reldw, "error_steps": nlog,
            "div_b_linf": divbdw,
            "roofline": {"kernel": "sweep_kernel (FP64, double-word WENO)", "bound": "alu", "achieved": achdw,
                         "peak": PEAK_FP64_TFLOPS, "unit": "TFLOP/s", "frac": achdw / PEAK_FP64_TFLOPS,
                         "traffic": sweep_traffic("fp64dw", zones), "launch_ms": swmsdw / nswdw,
                         "hbm_gbs": hbm_gbs(sweep_traffic("fp64dw", zones), swmsdw / nswdw),
                         "note": "the WENO part runs on the FP32 pipe, so the FP64 unit-count peak does not "
                                 "bound this kernel; frac compares it with the FP64-only form's ceiling"},
            "gpu_launches": launchesdw,
        },
        "weno_js": {"fp64_value": replica_throughput(world, zones, args.steps, msjs),
                    "fp64_ms_per_step": msjs / args.steps,
                    "fp32_bulk_value": replica_throughput(world, zones, args.steps, msfjs),
                    "fp32_bulk_ms_per_step": msfjs / args.steps},
        "div_b_linf": divb64,
        "conservation_drift": drift64,
        "e2e": {"value": world * zones * e2e_steps / e2e_s, "unit": "zone-updates/s",
                "h2d_bytes_per_step": int(cons.nbytes + bface.nbytes),
                "d2h_bytes_per_step": int(cons.nbytes + bface.nbytes), "steps": e2e_steps,
                "clocks": e2e_clocks},
        "gpu_launches": launches64,
        "clocks": clocks,
        "kernel_src": kernel_source_hash(),
        "hbm_peak_gbs": peaks.get("hbm_gbs"),
    }
    if not args.no_sub_records and rank == 0 and world == 1:
        # the other two forms of the path, compact: the 512-patch batch and the
        # 64^3 adjoint rollout (each also runs alone with --workload)
        import copy
        ab = copy.copy(args)
        ab.n, ab.steps, ab.warmup, ab.err_steps = 256, 5, 3, 3
        line["batched"] = batched_record(ab, compact=True)
        aa = copy.copy(args)
        aa.n, aa.steps = 64, 10
        line["adjoint"] = adjoint_record(aa, compact=True)
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        line["cpu_baseline"] = cpu_baseline(args, cons, bface)
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def cpu_model() -> str:
    """The host CPU's model name (or its architecture when /proc does not say)."""
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":")[0].strip().lower()
            if key in ("model name", "cpu model", "hardware"):
                return line.split(":", 1)[1].strip()
        import platform
        parts = {}
        for line in open("/proc/cpuinfo"):
            if ":" in line:
                k, v = line.split(":", 1)
                parts.setdefault(k.strip(), v.strip())
        return f"{platform.machine()} implementer {parts.get('CPU implementer', '?')} part {parts.get('CPU part', '?')}"
    except OSError:
        import platform
        return platform.machine()


def cpu_baseline(args, cons, bface):
    """The oracle, as it stands, on the host cores: args.cpu_steps whole
    steps of the n^3 workload itself (the native arm's initial state), and
    for the single-core figure a bounded 64^3 box of the same generator for
    about a quarter of args.cpu_seconds."""
    import oracle
    from paper_1812_04278_gb300 import inputs
    oracle.build()
    n = args.n
    o = oracle.Oracle((n, n, n), 1.0 / n, oracle.make_config(weno_variant=oracle.WENO_Z))
    o.set_state(cons, bface)
    times = oracle_timed_steps(oracle, o, args.cpu_steps)
    el = sum(times)
    cores = oracle.num_threads()
    value = n ** 3 * args.cpu_steps / el
    o.close()
    ns = 64
    c64, b64 = inputs.turbulent_state(ns, seed=1812, seed_b=1813, mach=1.0, beta=1.0, dB_frac=0.1,
                                      kmin=2, kmax=min(32, ns // 2 - 1))
    oracle.set_num_threads(1)
    o1 = oracle.Oracle((ns, ns, ns), 1.0 / ns, oracle.make_config(weno_variant=oracle.WENO_Z))
    o1.set_state(c64, b64)
    steps1 = 0
    t0 = time.perf_counter()
    while True:
        o1.step(o1.cfl_dt())
        steps1 += 1
        el1 = time.perf_counter() - t0
        if el1 >= 0.25 * args.cpu_seconds:
            break
    oracle.set_num_threads(cores)
    return {"value": value, "unit": "zone-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"{args.cpu_steps} full steps of the {n}^3 workload itself", "seconds": el,
            "single_core_value": ns ** 3 * steps1 / el1,
            "single_core_sample": f"{steps1} full steps of a {ns}^3 box of the same generator on 1 core",
            "cpu_model": cpu_model(), "nproc": os.cpu_count()}


def run_blast(args):
    """Magnetised blast in Mach-5 turbulence (beta 0.2, P 0.1 -> 100 inside
    r < 0.05), WENO-JS, floors on (rho, P >= 1e-8): FP32-bulk timed; the L1
    error against FP64 after --err-steps steps at the FP64 run's dt sequence."""
    import torch
    torch.cuda.set_device(0)
    from paper_1812_04278_gb300 import build, inputs
    build.build()
    from paper_1812_04278_gb300 import w5ct as w5
    n = args.n
    shape, dx, zones = (n, n, n), (1.0 / n,) * 3, n ** 3
    cons, bface = inputs.blast_turbulence_state(n)
    cons_d, bface_d = torch.from_numpy(cons).cuda(), torch.from_numpy(bface).cuda()
    sampler = ClockSampler(0)
    s32, ms32, nsw, swms, launches, clocks = timed_run(torch, w5, shape, dx, cons_d, bface_d, w5.W5CT_FP32_BULK,
                                                       args.steps, args.warmup, None, sampler, None,
                                                       variant=w5.W5CT_WENO_JS, floors=1)
    hits, bad = s32.status()
    divb32 = s32.div_b_norm()[0]
    s32.close()
    # error statement: FP64 and FP32-bulk from the same input at the same dt sequence
    ne = args.err_steps
    dts = torch.zeros(ne, dtype=torch.float64, device="cuda")
    cfg64 = w5.make_config(precision=w5.W5CT_FP64, weno_variant=w5.W5CT_WENO_JS, floors=1)
    g = w5.Solver(shape, dx, cfg64, stream=torch.cuda.current_stream().cuda_stream)
    g.set_state(cons_d, bface_d)
    t0 = time.perf_counter()
    for k in range(ne):
        g.step_cfl(dts[k:k + 1])
    g.synchronize()
    ms64 = 1e3 * (time.perf_counter() - t0) / ne
    c64, b64, _ = g.get_state()
    g.close()
    cfg32 = w5.make_config(precision=w5.W5CT_FP32_BULK, weno_variant=w5.W5CT_WENO_JS, floors=1)
    f = w5.Solver(shape, dx, cfg32, stream=torch.cuda.current_stream().cuda_stream)
    f.set_state(cons_d, bface_d)
    for k in range(ne):
        w5.w5ct_step_dev(f.ctx, dts[k:k + 1])
    c32, b32, _ = f.get_state()
    f.close()
    value = zones * args.steps / (ms32 * 1e-3)
    ach = SWEEP_FLOPS_PER_ZONE[0] * zones / (swms / nsw * 1e-3) / 1e12
    line = {
        "metric": "zone-updates/s (3D WENO5-CT MHD, full RK4 step)", "value": value, "unit": "zone-updates/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms32 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "accumulate": "f64",
        "data": "synthetic",
        "config": {"workload": f"periodic {n}^3 magnetised blast (P 0.1 -> 100 inside r < 0.05, B = (1,1,1)/sqrt3, "
                               f"beta 0.2) in k^-5/3 turbulence at rms Mach 5 (seed 1815); WENO-JS, CFL 0.8, "
                               f"floors rho, P >= 1e-8", "zones": zones, "grid": [n, n, n],
                   "l2_policy": "state larger than L2, no flush"},
        "roofline": {"kernel": "sweep_kernel (FP32)", "bound": "alu", "achieved": ach, "peak": PEAK_FP32_TFLOPS,
                     "unit": "TFLOP/s", "frac": ach / PEAK_FP32_TFLOPS, "traffic": sweep_traffic("fp32", zones),
                     "launch_ms": swms / nsw},
        "floor_hits": hits, "nonphysical": bad, "div_b_linf": divb32,
        "fp64": {"ms_per_step": ms64, "value": zones / (ms64 * 1e-3), "error_steps": ne,
                 "l1_fp32_vs_fp64": l1_error(c32, b32, c64, b64), "l1_fp64_change": l1_error(c64, b64, cons, bface),
                 "max_rel_fp32_vs_fp64": float(max(np.abs(c32 - c64).max(), np.abs(b32 - b64).max()) /
                                               max(np.abs(c64).max(), np.abs(b64).max()))},
        "gpu_launches": launches, "clocks": clocks, "kernel_src": kernel_source_hash(),
    }
    print(json.dumps(line))


def run_wave(args):
    """The 32^3 fast magnetosonic eigenmode (amplitude 1e-6 along (1,2,2)/3),
    FP64, WENO-Z, CFL 0.8: GPU steps and the oracle's steps on the host."""
    import torch
    torch.cuda.set_device(0)
    import oracle
    from paper_1812_04278_gb300 import build, inputs
    build.build()
    oracle.build()
    from paper_1812_04278_gb300 import w5ct as w5
    n = args.n
    shape, zones = (n, n, n), n ** 3
    cons, bface = inputs.fast_wave_config(shape)
    s, ms, nsw, swms, launches, clocks = timed_run(torch, w5, shape, (1.0 / n,) * 3, torch.from_numpy(cons).cuda(),
                                                   torch.from_numpy(bface).cuda(), w5.W5CT_FP64, args.steps,
                                                   args.warmup, None, ClockSampler(0), None)
    s.close()
    o = oracle.Oracle(shape, 1.0 / n, oracle.make_config(weno_variant=oracle.WENO_Z))
    o.set_state(cons, bface)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(o.cfl_dt())
    el = time.perf_counter() - t0
    value = zones * args.steps / (ms * 1e-3)
    line = {
        "metric": "zone-updates/s (3D WENO5-CT MHD, full RK4 step)", "value": value, "unit": "zone-updates/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"periodic {n}^3 fast magnetosonic eigenmode, amplitude 1e-6 along (1,2,2)/3, "
                               f"rho=1, P=1, B=(1,sqrt2,1/2) in the wave frame; WENO-Z, CFL 0.8",
                   "zones": zones, "grid": [n, n, n], "l2_policy": "state fits in L2 (launch-bound size)"},
        "sweep_launch_ms": swms / nsw, "gpu_launches": launches, "clocks": clocks,
        "cpu_baseline": {"value": zones * args.steps / el, "unit": "zone-updates/s", "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": f"the same {args.steps} steps of the same {n}^3 input",
                         "seconds": el},
    }
    print(json.dumps(line))


SCHEDULES = ["one launch per kernel", "persistent sweeps per tile variant", "whole step in one persistent launch"]


def _patch_state_job(spec):
    from paper_1812_04278_gb300 import inputs
    return inputs.patch_state(spec)


def batch_states(specs, workers):
    """Turbulent states of every patch, generated by a pool of host threads
    (numpy's FFTs and array arithmetic release the interpreter lock)."""
    if workers <= 1:
        return [_patch_state_job(sp) for sp in specs]
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(_patch_state_job, specs))


def run_batched(args):
    print(json.dumps(batched_record(args)))


def batched_record(args, compact=False):
    """512 independent periodic patches of uneven sizes (each of nx, ny, nz
    from {16, 24, 32, 48, 64}, seed 1803) with their own turbulent states
    and dts, FP32-bulk, advanced by one context: every step is one replay of
    a CUDA graph of the batched launches.  Beside it: the same patches in
    FP64 (batched, eager), the L1 error of FP32-bulk against FP64 at the
    FP64 run's per-patch dt sequence, and the patches advanced one context
    per patch (unbatched launches).  Floors rho, P >= 1e-8 are on: the
    supersonic low-beta patches reach P <= 0 within a few steps without them
    (the oracle's too).  compact: the record the default benchmark line
    carries (no model-tile run and no one-context-per-patch run)."""
    from paper_1812_04278_gb300 import inputs
    specs = inputs.patch_batch_spec(npatch=args.patches, seed=1803)
    states = batch_states(specs, min(16, os.cpu_count() or 1))
    import torch
    torch.cuda.set_device(0)
    from paper_1812_04278_gb300 import build
    build.build()
    from paper_1812_04278_gb300 import w5ct as w5
    shapes = [sp["shape"] for sp in specs]
    dxs = [sp["dx"] for sp in specs]
    zones = int(sum(np.prod(sh) for sh in shapes))
    npatch = len(specs)
    stream = torch.cuda.current_stream()

    def reset(b):
        for p, (c, f) in enumerate(states):
            b.set_state(p, c, f)

    def make(precision):
        b = w5.Batch(shapes, dxs, w5.make_config(precision=precision, floors=1), stream=stream.cuda_stream)
        reset(b)
        return b

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def graph_steps(b, nsteps):
        e0.record(stream)
        b.step_graph(nsteps)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    # ---- FP32-bulk, graph replay (headline): tile shapes from the model,
    # then from the measuring autotuner; each timed run starts from the
    # initial state (the supersonic patches stay physical for about 15 steps
    # from it; the scheme has no protection fluxes)
    b32 = make(w5.W5CT_FP32_BULK)
    tiles_model = b32.tile_variants().tolist()
    ms_model, bad_model = float("nan"), 0
    if not compact:
        b32.step_graph(args.warmup)
        torch.cuda.synchronize()
        ms_model = graph_steps(b32, args.steps)
        bad_model = b32.status()[1]
    t0 = time.perf_counter()
    b32.autotune(w5.W5CT_TUNE_MEASURE, 3)
    tune_s = time.perf_counter() - t0
    tiles_tuned = b32.tile_variants().tolist()
    schedule = b32.schedule()
    # every schedule, for the record
    ms_sched = {}
    for sc in (0, 1, 2):
        b32.set_schedule(sc)
        reset(b32)
        b32.step_graph(args.warmup)
        torch.cuda.synchronize()
        ms_sched[sc] = graph_steps(b32, args.steps)
        if b32.status()[1]:
            ms_sched[sc] = float("nan")
    b32.set_schedule(schedule)
    reset(b32)
    b32.step_graph(args.warmup)
    torch.cuda.synchronize()
    launches0 = w5.w5ct_launch_count(b32.ctx)
    sampler = ClockSampler(0)
    sampler.start()
    ms32 = graph_steps(b32, args.steps)
    clocks = sampler.stop()
    launches = w5.w5ct_launch_count(b32.ctx) - launches0
    hits, bad = b32.status()
    # per-launch time of the sweeps (eager steps with the launch timers on,
    # one launch per axis and variant)
    reset(b32)
    b32.set_schedule(0)
    w5.w5ct_set_timing(b32.ctx, True)
    for _ in range(2):
        b32.step_cfl()
    torch.cuda.synchronize()
    nsw, swms = w5.w5ct_sweep_timing(b32.ctx)
    w5.w5ct_set_timing(b32.ctx, False)
    b32.set_schedule(schedule)
    divb32 = max(b32.div_b_norm(p)[0] for p in range(npatch))
    b32.close()

    # ---- FP64, batched, eager, logging every patch's dt
    ne = args.err_steps
    dts = torch.zeros((ne, npatch), dtype=torch.float64, device="cuda")
    b64 = make(w5.W5CT_FP64)
    torch.cuda.synchronize()
    b64.autotune(w5.W5CT_TUNE_MEASURE, 1)
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(ne):
        b64.step_cfl(dts[k])
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1)
    s64 = [b64.get_state(p) for p in range(npatch)]
    divb64 = max(b64.div_b_norm(p)[0] for p in range(npatch))
    b64.close()
    # ---- FP32-bulk at the FP64 dts: per-patch L1 error
    f32 = make(w5.W5CT_FP32_BULK)
    for k in range(ne):
        f32.step_dev(dts[k])
    l1s, l1c = [], []
    for p in range(npatch):
        c32, bb32, _ = f32.get_state(p)
        c64, bb64, _ = s64[p]
        l1s.append(l1_error(c32, bb32, c64, bb64))
        l1c.append(l1_error(c64, bb64, *states[p]))
    f32.close()
    del s64

    value = zones * args.steps / (ms32 * 1e-3)
    sched_values = {SCHEDULES[k]: zones * args.steps / (v * 1e-3) for k, v in ms_sched.items()}
    if compact:
        return {"workload": f"{npatch} uneven periodic patches (seed 1803), {zones} zones, FP32-bulk, WENO-Z, "
                            f"floors on, one CUDA graph replay per step",
                "value": value, "unit": "zone-updates/s", "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms32 / args.steps, "schedule": SCHEDULES[schedule], "schedule_values": sched_values,
                "fp64_batched_value": zones * ne / (ms64 * 1e-3),
                "l1_fp32_vs_fp64": {"mean": float(np.mean(l1s)), "max": float(np.max(l1s)), "steps": ne,
                                    "fp64_change_mean": float(np.mean(l1c))},
                "nonphysical": bad + bad_model, "floor_hits": hits, "div_b_linf": divb32,
                "gpu_launches": launches}

    # ---- unbatched: one context per patch, eager steps
    solvers = []
    for p, (c, f) in enumerate(states):
        sv = w5.Solver(shapes[p], dxs[p], w5.make_config(precision=w5.W5CT_FP32_BULK, floors=1),
                       stream=stream.cuda_stream)
        sv.set_state(c, f)
        solvers.append(sv)
    for sv in solvers:
        sv.step_cfl()
    nu = max(1, min(3, args.steps))
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(nu):
        for sv in solvers:
            sv.step_cfl()
    e1.record(stream)
    torch.cuda.synchronize()
    msu = e0.elapsed_time(e1)
    for sv in solvers:
        sv.close()

    ach = SWEEP_FLOPS_PER_ZONE[1] * zones / (swms / nsw * 1e-3) / 1e12
    sizes = np.array([np.prod(sh) for sh in shapes])
    line = {
        "metric": "zone-updates/s (3D WENO5-CT MHD, full RK4 step)", "value": value, "unit": "zone-updates/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms32 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "accumulate": "f64",
        "data": "synthetic",
        "config": {"workload": f"{npatch} independent periodic unit-box patches, each of nx, ny, nz uniform in "
                               f"{{16,24,32,48,64}} (seed 1803); per patch: rho=1, P=1/gamma, k^-5/3 turbulence "
                               f"(2 <= k <= max(2, min(n)/8)) at rms Mach U[0.5,3], beta log-uniform [0.1,10], mean B "
                               f"along a random unit vector; own dt per patch; WENO-Z, CFL 0.8, floors rho, P >= 1e-8; "
                               f"one CUDA graph replay per step", "zones": zones, "patches": npatch,
                   "patch_cells_min": int(sizes.min()), "patch_cells_max": int(sizes.max()),
                   "l2_policy": "state larger than L2, no flush"},
        "roofline": {"kernel": "sweep_batched_kernel (FP32)", "bound": "alu", "achieved": ach,
                     "peak": PEAK_FP32_TFLOPS, "unit": "TFLOP/s", "frac": ach / PEAK_FP32_TFLOPS,
                     "traffic": None, "launch_ms": swms / nsw, "algorithmic_flops_per_launch":
                     SWEEP_FLOPS_PER_ZONE[1] * zones, "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"},
        "fp64_batched": {"value": zones * ne / (ms64 * 1e-3), "ms_per_step": ms64 / ne, "steps": ne,
                         "div_b_linf": divb64},
        "l1_fp32_vs_fp64": {"mean": float(np.mean(l1s)), "max": float(np.max(l1s)), "steps": ne,
                            "fp64_change_mean": float(np.mean(l1c))},
        "tiles": {"variants": "0: 32x16, 1: 16x16, 2: 8x16, 3: 8x8 (lanes along x x faces)",
                  "patches_per_axis_and_variant_tuned": tiles_tuned,
                  "patches_per_axis_and_variant_model": tiles_model,
                  "model_value": zones * args.steps / (ms_model * 1e-3), "autotune_seconds": tune_s,
                  "schedule": SCHEDULES[schedule],
                  "schedule_values": sched_values},
        "unbatched_fp32": {"value": zones * nu / (msu * 1e-3), "ms_per_step": msu / nu, "steps": nu,
                           "contexts": npatch},
        "floor_hits": hits, "nonphysical": bad + bad_model, "div_b_linf": divb32,
        "gpu_launches": launches, "clocks": clocks, "kernel_src": kernel_source_hash(),
    }
    return line


def run_adjoint(args):
    print(json.dumps(adjoint_record(args)))


def adjoint_record(args, compact=False):
    """Gradient of the L2 misfit after --steps steps (fixed dt = the CFL dt of
    the initial state) with respect to the initial rho, v and edge vector
    potential, on the n^3 oblique circularly polarised Alfven wave (amplitude
    0.1 along (1,2,2)/3) plus a Gaussian overpressure (P x10, radius 0.1 L);
    target: the wave without the overpressure.  FP64 and FP32-bulk: forward
    (with per-step checkpoints) and backward times, the adjoint sweep launch
    time, and central-difference checks of a random directional derivative
    (h = 1e-6) on this state and on a textured copy (WENO-Z is not
    differentiable where a field is exactly uniform).  compact: the record
    the default benchmark line carries (the textured WENO-Z check only)."""
    import torch
    torch.cuda.set_device(0)
    from paper_1812_04278_gb300 import adjoint, build, inputs
    build.build()
    from paper_1812_04278_gb300 import w5ct as w5
    n = args.n
    shape, dx, zones = (n, n, n), (1.0 / n,) * 3, n ** 3
    stream = torch.cuda.current_stream()

    def setup(texture):
        rho, v, P, A, B0 = inputs.cpaw_overpressure(shape)
        P_wave = inputs.cpaw_overpressure(shape, peak=1.0)[2]
        if texture:
            X, Y, Z, _ = inputs.cell_centres(shape)
            ph = np.random.default_rng(42).uniform(0, 2 * np.pi, 6)
            tp = 2 * np.pi
            rho = rho * (1 + texture * (np.sin(tp * X + ph[0]) + np.sin(tp * Y + ph[1]) + np.sin(tp * Z + ph[2])) / 3)
            f = 1 + texture * (np.cos(tp * X + ph[3]) + np.cos(tp * Y + ph[4]) + np.cos(tp * Z + ph[5])) / 3
            P, P_wave = P * f, P_wave * f
        tc, tb = inputs.ic_from_potential(rho, v, P_wave, A, B0, dx)
        g = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        return dict(rho=g(rho), v=g(v), P=g(P), A=g(A), B0=B0, tc=g(tc), tb=g(tb))

    def solver(precision):
        return w5.Solver(shape, dx, w5.make_config(precision=precision), stream=stream.cuda_stream)

    def grad(s, pb, dt):
        rho, v, A = (pb[k].clone().requires_grad_() for k in ("rho", "v", "A"))
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        L = adjoint.rollout_misfit(rho, v, A, s, pb["P"], pb["B0"], pb["tc"], pb["tb"], dt, args.steps)
        e1.record(stream)
        L.backward()
        e2.record(stream)
        torch.cuda.synchronize()
        return float(L.detach()), (rho.grad, v.grad, A.grad), e0.elapsed_time(e1), e1.elapsed_time(e2)

    X, Y, Z, _ = inputs.cell_centres(shape)

    def smooth_field(rng, scale):
        f = np.zeros_like(X)
        for _ in range(3):
            kv = rng.integers(-2, 3, size=3)
            f += rng.standard_normal() * np.sin(2 * np.pi * (kv[0] * X + kv[1] * Y + kv[2] * Z) + rng.uniform(0, 6.3))
        return scale * f

    def fd_check(s, pb, dt, g, seed):
        # a smooth random direction (low Fourier modes): a pointwise random
        # one flips |IS_0 - IS_2| of WENO-Z wherever the data are smoother
        # than the perturbation
        rng = np.random.default_rng(seed)
        d = [torch.from_numpy(np.ascontiguousarray(np.stack([smooth_field(rng, sc) for _ in range(m)])
                                                   if m > 1 else smooth_field(rng, sc))).cuda()
             for m, sc in ((1, 0.05), (3, 0.05), (3, 0.002))]
        gd = float(sum((gi * di).sum() for gi, di in zip(g, d)))
        h = 1e-6
        Lp = adjoint.rollout_value(pb["rho"] + h * d[0], pb["v"] + h * d[1], pb["A"] + h * d[2], s, pb["P"], pb["B0"],
                                   pb["tc"], pb["tb"], dt, args.steps)
        Lm = adjoint.rollout_value(pb["rho"] - h * d[0], pb["v"] - h * d[1], pb["A"] - h * d[2], s, pb["P"], pb["B0"],
                                   pb["tc"], pb["tb"], dt, args.steps)
        fd = (Lp - Lm) / (2 * h)
        return gd, fd, abs(gd - fd) / abs(fd)

    pb = setup(0.0)
    pbt = setup(0.02)
    out = {}
    grads = {}
    for prec, name in ((w5.W5CT_FP64, "fp64"), (w5.W5CT_FP32_BULK, "fp32_bulk")):
        s = solver(prec)
        cons = torch.empty((5, n, n, n), dtype=torch.float64, device="cuda")
        bface = torch.empty((3, n, n, n), dtype=torch.float64, device="cuda")
        w5.w5ct_ic_from_potential(shape, dx, 5.0 / 3.0, pb["B0"], pb["rho"], pb["v"], pb["P"], pb["A"], cons, bface,
                                  stream.cuda_stream)
        s.set_state(cons, bface)
        dt = s.cfl_dt()
        grad(s, pb, dt)                                   # warm-up
        L, g, ms_f, ms_b = grad(s, pb, dt)
        grads[name] = g
        # one adjoint step with the launch timers: the sweep-adjoint share
        lq = torch.zeros((5, n, n, n), dtype=torch.float64, device="cuda")
        lb = torch.zeros((3, n, n, n), dtype=torch.float64, device="cuda")
        lq[0] = 1.0
        s.set_state(cons, bface)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        w5.w5ct_adjoint_step(s.ctx, dt, lq, lb, torch.empty_like(lq), torch.empty_like(lb))
        e1.record(stream)
        torch.cuda.synchronize()
        ms_adj_step = e0.elapsed_time(e1)
        rec = {"misfit": L, "dt": dt, "forward_ms": ms_f, "backward_ms": ms_b,
               "adjoint_ms_per_step": ms_b / args.steps, "forward_ms_per_step": ms_f / args.steps,
               "one_adjoint_step_ms": ms_adj_step,
               "adjoint_zone_steps_per_s": zones * args.steps / (ms_b * 1e-3)}
        # roofline of the whole adjoint step (every kernel of the backward
        # pass) on the algorithmic count of a vector-Jacobian product
        ach = ADJOINT_STEP_FLOPS_PER_ZONE[1] * zones / (ms_b / args.steps * 1e-3) / 1e12
        pk = PEAK_FP64_TFLOPS if name == "fp64" else PEAK_FP32_TFLOPS
        rec["roofline"] = {"kernel": "one adjoint step (all kernels of the backward pass)", "bound": "alu",
                           "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk, "traffic": None,
                           "algorithmic_flops_per_zone": ADJOINT_STEP_FLOPS_PER_ZONE[1],
                           "peak_source": "GB300 FP64 published rate" if name == "fp64"
                           else "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}
        if name == "fp64" and compact:
            st = solver(prec)
            _, gt, _, _ = grad(st, pbt, dt)
            gd, fd, rel = fd_check(st, pbt, dt, gt, 12)
            rec["fd_check_textured"] = {"g_dot_delta": gd, "central_difference": fd, "rel_err": rel, "h": 1e-6,
                                        "state": "rho and P textured by 2% smooth modes"}
            st.close()
        elif name == "fp64":
            gd, fd, rel = fd_check(s, pb, dt, g, 11)
            rec["fd_check"] = {"g_dot_delta": gd, "central_difference": fd, "rel_err": rel, "h": 1e-6,
                               "state": "the workload's state (uniform rho: WENO-Z weights not differentiable there)"}
            st = solver(prec)
            _, gt, _, _ = grad(st, pbt, dt)
            gd, fd, rel = fd_check(st, pbt, dt, gt, 12)
            rec["fd_check_textured"] = {"g_dot_delta": gd, "central_difference": fd, "rel_err": rel, "h": 1e-6,
                                        "state": "rho and P textured by 2% smooth modes"}
            st.close()
            sj = w5.Solver(shape, dx, w5.make_config(precision=prec, weno_variant=w5.W5CT_WENO_JS),
                           stream=stream.cuda_stream)
            _, gj, _, _ = grad(sj, pbt, dt)
            gd, fd, rel = fd_check(sj, pbt, dt, gj, 13)
            rec["fd_check_textured_js"] = {"g_dot_delta": gd, "central_difference": fd, "rel_err": rel, "h": 1e-6,
                                           "state": "textured, WENO-JS"}
            sj.close()
        out[name] = rec
        s.close()
    rel32 = max(float((a - b).abs().max() / a.abs().max()) for a, b in zip(grads["fp64"], grads["fp32_bulk"]))
    # directional derivatives of the two forms along one smooth direction
    rng = np.random.default_rng(14)
    d = [torch.from_numpy(np.ascontiguousarray(np.stack([smooth_field(rng, sc) for _ in range(m)])
                                               if m > 1 else smooth_field(rng, sc))).cuda()
         for m, sc in ((1, 0.05), (3, 0.05), (3, 0.002))]
    gd64 = float(sum((g * e).sum() for g, e in zip(grads["fp64"], d)))
    gd32 = float(sum((g * e).sum() for g, e in zip(grads["fp32_bulk"], d)))
    value = out["fp64"]["adjoint_zone_steps_per_s"]
    if compact:
        return {"workload": f"{n}^3 circularly polarised Alfven wave + overpressure, gradient of the misfit after "
                            f"{args.steps} fixed-dt steps in rho, v and the vector potential, WENO-Z, one checkpoint "
                            f"per step", "value": value, "unit": "adjoint zone-steps/s",
                "fp64_adjoint_ms_per_step": out["fp64"]["adjoint_ms_per_step"],
                "fp64_forward_ms_per_step": out["fp64"]["forward_ms_per_step"],
                "fp64_roofline": out["fp64"]["roofline"], "fp32_bulk_roofline_frac": out["fp32_bulk"]["roofline"]["frac"],
                "fp32_bulk_value": out["fp32_bulk"]["adjoint_zone_steps_per_s"],
                "fp32_bulk_adjoint_ms_per_step": out["fp32_bulk"]["adjoint_ms_per_step"],
                "fd_check_textured_rel_err": out["fp64"]["fd_check_textured"]["rel_err"],
                "fp32_vs_fp64_grad_max_rel": rel32, "fp32_vs_fp64_directional_rel": abs(gd32 - gd64) / abs(gd64)}
    line = {
        "metric": "adjoint zone-steps/s (gradient of a 10-step rollout misfit, backward pass)", "value": value,
        "unit": "zone-steps/s", "n_gpus": 1, "steps": args.steps, "warmup": 1,
        "ms_per_step": out["fp64"]["adjoint_ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"periodic {n}^3 oblique circularly polarised Alfven wave (amplitude 0.1, k = 2 pi "
                               f"(1,2,2), rho = 1, P = 0.1, B_par = 1) plus a Gaussian overpressure (P x10 peak, "
                               f"radius 0.1); misfit to the wave without the overpressure after {args.steps} steps "
                               f"of fixed dt (CFL 0.8 of the initial state); gradient in rho, v and the edge vector "
                               f"potential; WENO-Z; one checkpoint per step", "zones": zones, "grid": [n, n, n]},
        "roofline": out["fp64"]["roofline"],
        "fp64": out["fp64"], "fp32_bulk": out["fp32_bulk"], "fp32_vs_fp64_grad_max_rel": rel32,
        "fp32_vs_fp64_directional_rel": abs(gd32 - gd64) / abs(gd64),
        "kernel_src": kernel_source_hash(),
    }
    print(json.dumps(line))


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "blast":
        run_blast(args)
    elif args.workload == "wave":
        run_wave(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
