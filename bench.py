#!/usr/bin/env python
"""Benchmark of the FP64 particle step (one classic RK4 step of every particle:
deposit, interpolation, Hamiltonian, commutators, update) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

Prints one JSON line (rank 0).  The default workload is the throughput-scale
1D box: 16384 cells x 1000 directions = 16.4M particles, per-cell densities
and flux factors drawn from a seeded generator.  `value` is particle-updates/s
over all ranks (one update = one full RK4 step of one particle), timed with
CUDA events on the box's stream over exactly K steps with inputs resident in
HBM.  With N > 1 (torchrun) every rank runs its own independent box
(replicas, weak scaling; the path has no data exchange between boxes).

`--impl reference` times the CPU oracle (the plain FP64 C implementation the
tests check the kernels against) on the host cores, each step a bounded sample
of the workload (its first 256 cells, all directions).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "particle-updates/s (FP64, 1 GB300) & % HBM roofline; batched and adjoint vs plain"
UNIT = "particle-updates/s"
# Algorithmic HBM bytes per particle-step: the 313 FP64 values classic RK4 must
# move when the state crosses the all-particle deposit barrier four times.
B_ALG_PER_UPDATE = 313 * 8
# Algorithmic FP64 flops per particle of one RK-stage launch (FMA = 2), counted
# from the formulation the kernel implements, on the 8 traceless components of
# H (the trace drops out of the commutator): G = A0 - Omega.A at the own cell
# (48), 3-tap interpolation with the deposit's shape weights (40), the third
# diagonal difference (1), two packed Hermitian commutators (162), RK update
# (72; stage 4: 36 + 2 for z).
FLOPS_RK = {1: 323, 2: 323, 3: 323, 4: 289}
# ... and of one deposit launch: position and shape weights (12), the 8
# traceless components of B = N rho - Nbar rhobar^* (29), 3-tap gather (40),
# accumulation of (1, Omega) x C (56).
FLOPS_DEPOSIT = 137
# Other shape orders change the stencil's taps (per component: order 0 has no
# gather, the cubic shape 5 taps instead of 3): RK stage -40 / +32, deposit
# -40 / +32 (+8 for the cubic weights); the vacuum and matter terms add 16 adds.
TAPS_DELTA = {0: -40, 1: 0, 2: 0, 3: 32}
WEIGHTS_DELTA = {0: -12, 1: -6, 2: 0, 3: 8}
# FP64 pipe, nominal: 2 DFMA per clock per SM (nominal 1.25 TFLOP/s / (2 flop x 152 SMs x 2.07 GHz) = 1.99),
# so 2 x 2 flop x 152 SMs x 2.07 GHz.  The roofline's denominator is the FP64 peak measured in the
# same run (fp64_peak: cuBLAS DGEMM); this derived figure is reported beside it.
PEAK_FP64_DERIVED_TFLOPS = 2 * 2 * 152 * 2.07e9 / 1e12
# Bytes per particle of one launch: RK stage (average over s = 1..4 of 57, 93, 93, 59
# doubles, the shape weights included), deposit (21 read + 3 weights written).
BYTES_RK = (57 + 93 + 93 + 59) / 4 * 8
BYTES_DEPOSIT = 24 * 8
# DRAM read + write per particle of one launch, from an ncu capture of the current
# kernels (2048 cells x 1000 directions, 2.048M particles, stages 1-4 averaged):
# scaled by the particles of the timed launch.
TRAFFIC_RK = 691.7   # k_rk_stage32 (32 cells per warp, traceless potential, autotuned grid)
TRAFFIC_DEPOSIT = 304.0   # k_deposit<5> (traceless potential)


# 3D boxes (quadratic shape: each particle reaches 3 x 3 neighbour rows), FP64
# flops per particle of one launch, counted from the kernels' formulation:
#   prep (k3_prep, once per particle and stage): the weights on 3 axes (3 x 12)
#     and the 8 traceless components of B (29);
#   deposit (k3_deposit_bw): per neighbour row, the particle's x-y share (1),
#     its z-weights scaled by it (3), the z-spread (40) and the sum (8): 52;
#     x 9 rows, plus the direction's moments (1, Omega) x S (56);
#   G field (k3_gfield, once per direction and cell): A0 - Omega . A (48);
#   RK stage: per neighbour row the x-y weight (1), the z-gather (40) and its
#     weighted sum (16): 57; x 9 rows; the third diagonal difference (1), two
#     commutators (162), RK update (72).
# 3D step, algorithmic FP64 flops per particle (= per direction and cell):
# k3_prep (lattice check 36, B 29); each separable pass along one axis (8
# components x one multiply and two FMA); k3_spread_x_sum, the deposit's last
# pass with the sum over directions (x pass 40 + moments 56); the G field; the
# RK stage (z interpolation 40, third diagonal difference 1, commutators 162, RK 72)
FLOPS3_PREP = 36 + 29
FLOPS3_PASS = 8 * 5
FLOPS3_DEPOSIT = FLOPS3_PASS + 56
FLOPS3_GFIELD = 48
FLOPS3_RK = FLOPS3_PASS + 1 + 162 + 72


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        try:
            return json.loads(p.read_text())
        except Exception:
            pass
    return {}


# ------------------------------------------------------------ distributed

def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def dist_init(world: int, use_cuda: bool):
    if world <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group(backend="nccl" if use_cuda else "gloo")
    return dist


def barrier(dist, device=None):
    if dist is not None:
        if device is not None and dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def max_over_ranks(dist, x: float, device=None) -> float:
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        try:
            for line in Path(self.path).read_text().splitlines():
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
            os.unlink(self.path)
        except OSError:
            pass
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        loaded = [v for v in sm if mx and v >= 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# Vacuum and matter terms of the --osc runs: three masses and angles, the phase,
# 50 MeV (the paper's energy), matter of 1e9 g/cm^3 with Ye 0.4.
OSC_BENCH = dict(mass_eV=(0.0, 8.6e-3, 5.0e-2), theta12=0.59, theta13=0.15, theta23=0.84, delta_cp=1.2,
                 energy_MeV=50.0, rho_g_cm3=1e9, Ye=0.4)


def workload(args):
    from paper_2101_02745_gb300 import workloads as W
    if args.workload == "throughput_1d" and (args.nz or args.ndir):
        wl = W.throughput_1d(nz=args.nz or 16384, ndir=args.ndir or 1000)
    else:
        wl = W.by_name(args.workload)
    if args.shape_order != 2:
        wl = W.with_shape(wl, args.shape_order)
    return wl


def fp64_peak(device, n: int = 8192, reps: int = 3):
    """FP64 peak measured on this GPU in this run: cuBLAS DGEMM through
    torch.matmul on float64 n x n matrices (2 n^3 flop), best of `reps` after
    one warm-up, CUDA events on the current stream, SM clocks sampled meanwhile.
    (GB300's FP64 matrix path shares the FP64 pipe with DFMA, so a DGEMM
    measures the same pipe the kernels use.)"""
    import torch
    g = torch.Generator(device=device).manual_seed(0)
    a = torch.rand(n, n, dtype=torch.float64, device=device, generator=g)
    b = torch.rand(n, n, dtype=torch.float64, device=device, generator=g)
    c = torch.matmul(a, b)
    torch.cuda.synchronize(device)
    clk = ClockSampler(device.index).start()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize(device)
        best = min(best, e0.elapsed_time(e1))
    clocks = clk.stop()
    del a, b, c
    torch.cuda.empty_cache()
    return {"tflops": 2.0 * n ** 3 / (best * 1e-3) / 1e12, "ms": best, "n": n, "reps": reps, "clocks": clocks,
            "how": f"cuBLAS DGEMM (torch.matmul, float64, {n}^3, 2 n^3 flop), best of {reps}, CUDA events"}


# ------------------------------------------------------------ CPU oracle

def oracle_rate(wl, steps: int, osc=None):
    """Particle-updates/s of the CPU oracle running `steps` RK4 steps of wl (single thread)."""
    from oracle import oracle as O
    cfg = O.config(wl.nz, wl.ndir, wl.Lz, wl.kappa, wl.c_light, wl.cfl_adv, wl.cfl_flavor, wl.area,
                   shape_order=wl.shape_order, osc=osc)
    parts = O.init(cfg, wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar, wl.alpha, wl.seed, wl.dirs)
    dt = O.timestep(cfg, O.deposit(cfg, parts))
    t0 = time.perf_counter()
    O.run(cfg, parts, dt, steps)
    el = time.perf_counter() - t0
    return wl.P * steps / el, el


def _oracle_job(job):
    wl, steps, osc = job
    return oracle_rate(wl, steps, osc)


def cpu_baseline(wl_full, budget_s: float = 12.0, osc=None):
    """The oracle, unchanged, on the host: single-threaded on a sample of the
    workload (the reported value), the same program in one process per host
    core on samples of the workload (aggregate rate), and single-threaded on
    the small (32 x 16, 100 steps) and paper-shaped (1024 x 378) boxes."""
    from concurrent.futures import ProcessPoolExecutor
    import multiprocessing as mp

    from paper_2101_02745_gb300 import workloads as W
    sample = W.head(wl_full, 1024)
    rate1, el1 = oracle_rate(sample, 1, osc)
    steps = max(1, int(budget_s / max(el1, 1e-3)) - 1)
    rate, el = oracle_rate(sample, steps, osc)
    out = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{sample.nz} cells x {sample.ndir} directions ({sample.P} particles) of the workload, "
                     f"{steps} RK4 steps in {el:.1f} s, single-threaded C (-O2)"}
    ncores = os.cpu_count() or 1
    small = W.head(wl_full, 256)
    psteps = max(1, int(0.6 * budget_s / max(el1 / 4, 1e-3)))
    try:
        with ProcessPoolExecutor(ncores, mp_context=mp.get_context("spawn")) as ex:
            list(ex.map(_oracle_job, [(W.head(wl_full, 8), 1, osc)] * ncores))     # start the workers
            t0 = time.perf_counter()
            list(ex.map(_oracle_job, [(small, psteps, osc)] * ncores))
            wall = time.perf_counter() - t0
        out["all_cores"] = {"value": ncores * small.P * psteps / wall, "cores": ncores,
                            "sample": f"{ncores} processes, each {small.nz} cells x {small.ndir} directions, "
                                      f"{psteps} steps, in {wall:.1f} s"}
    except Exception as e:  # keep the line even if the host refuses a process pool
        out["all_cores"] = {"unavailable": str(e)[:200]}
    per = {}
    for wl, st in ((W.tiny_fiducial(), 100), (W.paper_1d(), 3)):
        r, e = oracle_rate(wl, st, osc)
        per[wl.name] = {"value": r, "steps": st, "seconds": e}
    out["per_config"] = per
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_2101_02745_gb300 import workloads as W
    O.build()
    wl = workload(args)
    sample = W.head(wl, args.ref_cells)
    cfg = O.config(sample.nz, sample.ndir, sample.Lz, sample.kappa, sample.c_light, sample.cfl_adv,
                   sample.cfl_flavor, sample.area)
    parts = O.init(cfg, sample.n_nu, sample.n_nubar, sample.f_nu, sample.f_nubar, sample.alpha, sample.seed)
    dt = O.timestep(cfg, O.deposit(cfg, parts))
    O.run(cfg, parts, dt, args.warmup)
    t0 = time.perf_counter()
    O.run(cfg, parts, dt, args.steps)
    el = time.perf_counter() - t0
    value = sample.P * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / max(args.steps, 1) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "nz": wl.nz, "ndir": wl.ndir, "particles": wl.P,
                   "sample": f"first {sample.nz} cells x {sample.ndir} directions ({sample.P} particles) per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{sample.P} particles per step, {args.steps} timed steps, single-threaded C"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU

def run_gpu(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2101_02745_gb300 import build as B
    from paper_2101_02745_gb300 import emu as E
    from paper_2101_02745_gb300 import workloads as W

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the CUDA path has no CPU fallback)")
    if rank == 0:
        B.build()
    dist = dist_init(world, True)
    device = torch.device("cuda", local_rank)
    torch.cuda.set_device(device)
    barrier(dist, device)
    if rank != 0:
        B.build()  # no-op once rank 0 built it

    wl = workload(args)
    box = E.Box.from_workload(wl, device=device)
    if args.osc:
        box.set_oscillation(W.oscillation(**OSC_BENCH))
    stream = box.stream
    dt = box.timestep()
    # launch configuration: grid x RK-stage form, timed on dry steps (state untouched);
    # --choice fixes it instead (profiling runs, where timings under the profiler
    # would pick another candidate)
    if args.choice >= 0:
        box.apply_choice(args.choice)
        tune_choice, tune_ms = args.choice, [-1.0] * E.AUTOTUNE_CANDIDATES
    else:
        tune_choice, tune_ms = box.autotune(trial_steps=2)
    box.step(args.warmup, dt)
    box.sync()

    # ---- timed region: exactly K steps, inputs resident in HBM (state 7.9 GB >> 129 MB L2)
    barrier(dist, device)
    torch.cuda.synchronize(device)
    clocks = ClockSampler(device.index).start()
    E.emu_profile(box.box, True)
    n0 = box.launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    box.step(args.steps, dt)
    ev1.record(stream)
    torch.cuda.synchronize(device)
    barrier(dist, device)
    elapsed_ms = ev0.elapsed_time(ev1)
    launches = box.launches() - n0
    ktimes = E.emu_kernel_times(box.box)
    E.emu_profile(box.box, False)
    box.sync()
    t_ms = max_over_ranks(dist, elapsed_ms, device)
    value = world * wl.P * args.steps / (t_ms * 1e-3)

    # ---- end to end through the public API with host buffers: every step the
    # state (z, rho, rhobar) comes from pinned host memory through the C ABI's
    # host-buffer path (emu_set_particles with host pointers) and the step's
    # diagnostics are read back to pinned host memory (emu_diagnostics into a
    # device buffer, then a copy on the box's stream; all arrive before the
    # timed region ends).  Two boxes with their own streams take turns
    # (E.PingPongFeed): the next step's upload into the idle box overlaps the
    # other box's step, and neither step waits for the other's diagnostics.
    host = box.get_host()
    pin = {k: torch.from_numpy(host[k]).pin_memory() for k in ("z", "rho", "rhobar")}
    diag_dev = [torch.zeros(E.N_DIAG, dtype=torch.float64, device=device) for _ in range(2)]
    diag = [torch.zeros(E.N_DIAG, dtype=torch.float64).pin_memory() for _ in range(2)]
    box2 = E.Box.from_workload(wl, device=device, stream=torch.cuda.Stream(device))
    if args.osc:
        box2.set_oscillation(W.oscillation(**OSC_BENCH))
    box2.apply_choice(tune_choice)   # the first box's tuned configuration
    # the uploaded state is the boxes' own lattice state: a fixed layout, so
    # the uploads are not checked (and synchronised) one by one; the kernels
    # still flag particles off their sites.  The copies are asynchronous
    # (on_host = 2): the host arrays stay unchanged throughout.
    box.set_layout(0)
    box2.set_layout(0)
    feed = E.PingPongFeed([box, box2], pin, asynchronous=True)

    def step_and_read(bx):
        k = 0 if bx is box else 1
        E.emu_step(bx.box, 1, dt)
        E.emu_diagnostics(bx.box, diag_dev[k].data_ptr(), 0)
        with torch.cuda.stream(bx.stream):
            diag[k].copy_(diag_dev[k], non_blocking=True)

    def e2e_step():
        feed.step(step_and_read)

    # the host link's copy rate alone (the e2e step cannot beat the copy of its
    # inputs), timed on the second upload (the first touches the pinned pages)
    feed.install(1)
    torch.cuda.synchronize(device)
    t_c = time.perf_counter()
    feed.install(1)
    torch.cuda.synchronize(device)
    h2d_gbs = feed.h2d_bytes / (time.perf_counter() - t_c) / 1e9
    feed.prime()
    e2e_step()
    e2e_step()   # both boxes have captured their step graphs
    barrier(dist, device)
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize(device)
    e2e_s = max_over_ranks(dist, time.perf_counter() - t0, device)
    clk = clocks.stop()
    box.sync()
    box2.sync()
    e2e_value = world * wl.P * args.steps / e2e_s
    h2d = feed.h2d_bytes
    d2h = E.N_DIAG * 8
    del feed, box2, pin

    # ---- roofline of the dominant kernel from the live per-launch events,
    # against the FP64 peak measured in this run
    per = {k: (ms / n if n else 0.0, n, ms) for k, (ms, n) in ktimes.items()}
    total = sum(ms for (_, _, ms) in per.values()) or 1.0
    dominant = max(per, key=lambda k: per[k][2])
    avg_ms = per[dominant][0]
    flops_dep = FLOPS_DEPOSIT + TAPS_DELTA[wl.shape_order] + WEIGHTS_DELTA[wl.shape_order]
    flops_rk = sum(FLOPS_RK.values()) / 4 + TAPS_DELTA[wl.shape_order] + (16 if args.osc else 0)
    if dominant == "deposit":
        flops, bytes_, traffic = flops_dep * wl.P, BYTES_DEPOSIT * wl.P, TRAFFIC_DEPOSIT * wl.P
        kname = "k_deposit"
    elif dominant == "step":    # the fused step: all four stages' deposits and RK stages in one launch
        flops, bytes_, traffic = 4 * (flops_dep + flops_rk) * wl.P, 4 * (BYTES_DEPOSIT + BYTES_RK) * wl.P, None
        kname = "k_step"
    else:
        flops, bytes_ = flops_rk * wl.P, BYTES_RK * wl.P
        traffic = TRAFFIC_RK * wl.P if TRAFFIC_RK else None
        kname = "k_rk_stage"
    achieved = flops / (avg_ms * 1e-3) / 1e12
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    pk = fp64_peak(device) if not args.no_fp64_peak else None
    peak = pk["tflops"] if pk else PEAK_FP64_DERIVED_TFLOPS
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "traffic_unit": "bytes per launch (ncu dram read + write, scaled by particles)",
                "kernel": kname, "flops_per_launch": flops, "avg_launch_ms": avg_ms,
                "peak_source": ("measured in this run: " + pk["how"]) if pk else
                               "derived: 2 FP64 FMA/clk/SM x 152 SMs x 2.07 GHz (nominal 1.25 TFLOP/s)",
                "peak_measured": pk,
                "peak_derived": PEAK_FP64_DERIVED_TFLOPS, "frac_of_derived": achieved / PEAK_FP64_DERIVED_TFLOPS,
                "hbm_gbs_of_kernel": bytes_ / (avg_ms * 1e-3) / 1e9}
    hbm = {"achieved_gbs": value / world * B_ALG_PER_UPDATE / 1e9, "peak_gbs": hbm_peak,
           "frac": value / world * B_ALG_PER_UPDATE / 1e9 / hbm_peak, "bytes_per_update": B_ALG_PER_UPDATE,
           "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks else "fallback"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "nz": wl.nz, "ndir": wl.ndir, "particles_per_gpu": wl.P,
                       "shape_order": wl.shape_order, "vacuum_matter": bool(args.osc),
                       "dt_s": dt, "parallelism": f"replicas{world}" if world > 1 else "single",
                       "autotune_choice": tune_choice, "autotune_ms": [round(float(x), 4) for x in tune_ms],
                       "l2": "inputs larger than L2 (particle state %.2f GB per GPU vs 129 MB L2)" % (wl.P * 480 / 1e9)},
            "roofline": roofline, "hbm": hbm,
            "kernels": {k: {"launches": n, "avg_ms": a, "share": ms / total} for k, (a, n, ms) in per.items() if n},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": e2e_s / args.steps * 1e3, "h2d_gbs_alone": h2d_gbs,
                    "h2d_ms_alone": h2d / h2d_gbs / 1e6},
            "gpu_launches": launches,
            "clocks": clk,
        }
    del box
    torch.cuda.empty_cache()
    extras = {}
    if not args.no_extras:
        extras["batched"] = measure_sweep(args, dist, device, rank, world, min(args.steps, 20))
        extras["adjoint"] = measure_adjoint(dist, device, world, reps=1)
        extras["paper_shape"] = measure_paper_shape(args, dist, device, world)
        extras["anywhere"] = measure_anywhere(args, dist, device, world, steps=min(args.steps, 20))
        extras["box_3d"] = measure_box3d(args, dist, device, world, steps=min(args.steps, 10),
                                         fp64_peak_tflops=roofline["peak"] if pk else None)
    if rank == 0:
        line.update(extras)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(wl, osc=W.oscillation(**OSC_BENCH) if args.osc else None)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def measure_box3d(args, dist, device, world, steps=20, fp64_peak_tflops=None):
    """A 3D box (Sec. 5's future-work geometry): 64 x 64 x 64 cells of 1/16 cm,
    16 directions per cell (4.19M particles, 2.1 GB of state: larger than L2),
    per-cell densities and 3D flux vectors from a seeded generator, quadratic
    shape.  Autotuned grid, `steps` steps timed with CUDA events on the box's
    stream, the per-kernel launch times recorded by the library in the same
    window, and the dominant kernel's FP64 roofline."""
    import torch

    from paper_2101_02745_gb300 import emu as E
    from paper_2101_02745_gb300 import workloads as W

    n3 = args.n3 or 64
    wl = W.random_box3(n3, n3, n3, args.ndir3 or 16, seed=0)
    box = E.Box3D.from_workload(wl, device=device)
    dt = box.timestep()
    choice, cand_ms = box.autotune(trial_steps=2)
    box.step(args.warmup, dt)
    barrier(dist, device)
    torch.cuda.synchronize(device)
    E.emu_profile(box.box, True)
    n0 = box.launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(box.stream)
    box.step(steps, dt)
    ev1.record(box.stream)
    torch.cuda.synchronize(device)
    ms = max_over_ranks(dist, ev0.elapsed_time(ev1), device)
    launches = box.launches() - n0
    kt = E.emu_kernel_times(box.box)
    E.emu_profile(box.box, False)
    box.sync()
    per = {k: (t / n if n else 0.0, n, t) for k, (t, n) in kt.items()}
    total = sum(t for (_, _, t) in per.values()) or 1.0
    dominant = "rk_stage" if per["rk_stage"][2] >= per["deposit"][2] else "deposit"
    avg = per[dominant][0]
    flops = (FLOPS3_RK if dominant == "rk_stage" else FLOPS3_DEPOSIT) * wl.P
    achieved = flops / (avg * 1e-3) / 1e12
    peak = fp64_peak_tflops or PEAK_FP64_DERIVED_TFLOPS
    out = {"workload": wl.name, "particles_per_gpu": wl.P, "cells": [wl.nx, wl.ny, wl.nz], "ndir": wl.ndir,
           "steps": steps, "value": world * wl.P * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
           "note": "launches bracketed by the library's timing events (no graph replay) in this window",
           "autotune_choice": choice, "autotune_ms": [round(float(x), 4) for x in cand_ms],
           "gpu_launches": launches,
           "kernels": {k: {"launches": n, "avg_ms": a, "share": t / total} for k, (a, n, t) in per.items() if n},
           "roofline": {"bound": "alu", "kernel": f"k3_{dominant}", "achieved": achieved, "peak": peak,
                        "unit": "TFLOP/s", "frac": achieved / peak, "flops_per_launch": flops,
                        "avg_launch_ms": avg,
                        "peak_source": "measured in this run (DGEMM)" if fp64_peak_tflops else "derived"}}
    del box
    torch.cuda.empty_cache()
    return out


def run_box3d(args, rank, world, local_rank):
    """--workload box_3d: the 3D box's own line (value = its particle-updates/s)."""
    import torch

    from paper_2101_02745_gb300 import build as B

    if rank == 0:
        B.build()
    dist = dist_init(world, True)
    device = torch.device("cuda", local_rank)
    torch.cuda.set_device(device)
    barrier(dist, device)
    pk = fp64_peak(device) if not args.no_fp64_peak else None
    clocks = ClockSampler(device.index).start()
    r = measure_box3d(args, dist, device, world, args.steps, pk["tflops"] if pk else None)
    clk = clocks.stop()
    if rank == 0:
        line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": r["workload"], "cells": r["cells"], "ndir": r["ndir"],
                           "particles_per_gpu": r["particles_per_gpu"],
                           "l2": "inputs larger than L2 (particle state %.2f GB per GPU vs 129 MB L2)"
                                 % (r["particles_per_gpu"] * 496 / 1e9)},
                "roofline": r["roofline"], "box_3d": r, "gpu_launches": r["gpu_launches"], "clocks": clk,
                "fp64_peak": pk}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def measure_anywhere(args, dist, device, world, steps=20):
    """Particles anywhere: the paper's 1D run shape (1024 cells x 378
    directions, 387,072 particles) with every position moved by U(-0.45, 0.45)
    cells and every particle given its own random direction (numpy PCG64(0)),
    so no ring keeps the lattice contract and the box steps with the sorted
    path (per stage a stable radix sort by cell and a deposit by one warp per
    cell).  `steps` steps timed with CUDA events; the lattice path on the
    unscattered box beside it."""
    import numpy as np
    import torch

    from paper_2101_02745_gb300 import emu as E
    from paper_2101_02745_gb300 import workloads as W

    wl = W.paper_1d()
    rng = np.random.Generator(np.random.PCG64(0))
    out = {"workload": wl.name + "_anywhere", "particles_per_gpu": wl.P, "steps": steps,
           "scatter": "positions + U(-0.45, 0.45) cells, one random direction per particle"}
    for general in (True, False):
        box = E.Box.from_workload(wl, device=device)
        if general:
            h = box.get_host()
            z = h["z"] + rng.uniform(-0.45, 0.45, wl.P) * wl.dz
            z = z - wl.Lz * np.floor(z / wl.Lz)
            z = np.where(z >= wl.Lz, z - wl.Lz, z)   # (rounding can land a tiny negative on Lz)
            om = rng.normal(size=(wl.P, 3))
            om /= np.linalg.norm(om, axis=1, keepdims=True)
            box.set_host(z=z, ox=om[:, 0].copy(), oy=om[:, 1].copy(), oz=om[:, 2].copy())
            assert box.general()
        dt = box.timestep()
        box.step(args.warmup, dt)
        barrier(dist, device)
        torch.cuda.synchronize(device)
        n0 = box.launches()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(box.stream)
        box.step(steps, dt)
        ev1.record(box.stream)
        torch.cuda.synchronize(device)
        ms = max_over_ranks(dist, ev0.elapsed_time(ev1), device)
        box.sync()
        r = {"value": world * wl.P * steps / (ms * 1e-3), "ms_per_step": ms / steps,
             "launches_per_step": (box.launches() - n0) / steps}
        if general:
            out.update(r)
        else:
            out["lattice_path"] = r
        del box
    out["vs_lattice"] = out["value"] / out["lattice_path"]["value"]
    torch.cuda.empty_cache()
    return out


def run_anywhere(args, rank, world, local_rank):
    """--workload anywhere: the scattered paper-shaped box's own line."""
    import torch

    from paper_2101_02745_gb300 import build as B

    if rank == 0:
        B.build()
    dist = dist_init(world, True)
    device = torch.device("cuda", local_rank)
    torch.cuda.set_device(device)
    barrier(dist, device)
    clocks = ClockSampler(device.index).start()
    r = measure_anywhere(args, dist, device, world, args.steps)
    clk = clocks.stop()
    if rank == 0:
        line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": r["workload"], "particles_per_gpu": r["particles_per_gpu"],
                           "scatter": r["scatter"],
                           "l2": "inputs larger than L2 (particle state %.2f GB per GPU vs 129 MB L2)"
                                 % (r["particles_per_gpu"] * 480 / 1e9)},
                "anywhere": r, "gpu_launches": int(r["launches_per_step"] * args.steps), "clocks": clk}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def measure_paper_shape(args, dist, device, world, steps=100):
    """The paper's 1D run shape (1024 cells x 378 directions, 387,072 particles;
    the nubar flux along z, and tilted to normalize(0.1, 0, -1)): `steps` steps
    of each box on its autotuned grid, CUDA events on the box's stream.  The
    particle state (186 MB) is larger than L2."""
    import torch

    from paper_2101_02745_gb300 import emu as E
    from paper_2101_02745_gb300 import workloads as W

    out = {}
    for wl in (W.paper_1d(), W.paper_1d(True)):
        box = E.Box.from_workload(wl, device=device)
        dt = box.timestep()
        choice, cand_ms = box.autotune(trial_steps=2)
        box.step(args.warmup, dt)
        barrier(dist, device)
        torch.cuda.synchronize(device)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(box.stream)
        box.step(steps, dt)
        ev1.record(box.stream)
        torch.cuda.synchronize(device)
        ms = max_over_ranks(dist, ev0.elapsed_time(ev1), device)
        box.sync()
        out[wl.name] = {"particles_per_gpu": wl.P, "steps": steps, "value": world * wl.P * steps / (ms * 1e-3),
                        "ms_per_step": ms / steps, "autotune_choice": choice, "autotune_ms": list(cand_ms)}
        del box
    torch.cuda.empty_cache()
    return out


def measure_sweep(args, dist, device, rank, world, steps):
    """Batched sweep against the same boxes one at a time: the parameter sweep's
    independent boxes of uneven sizes advanced by one set of launches per step
    (CUDA graph replay, autotuned grid) and, for comparison, by the single-box
    calls box after box; both timed over `steps` steps with CUDA events."""
    import torch

    from paper_2101_02745_gb300 import emu as E
    from paper_2101_02745_gb300 import workloads as W

    wls = W.sweep(args.nbox, seed=rank)
    P = sum(w.P for w in wls)
    batch = E.Box.from_workloads(wls, device=device)
    dts = batch.batch_timestep()
    choice, cand_ms = batch.autotune(trial_steps=2)
    batch.batch_step(args.warmup)
    stream = batch.stream
    barrier(dist, device)
    torch.cuda.synchronize(device)
    n0 = batch.launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    batch.batch_step(steps)
    ev1.record(stream)
    torch.cuda.synchronize(device)
    batched_ms = max_over_ranks(dist, ev0.elapsed_time(ev1), device)
    launches = batch.launches() - n0
    batch.sync()
    del batch
    torch.cuda.empty_cache()
    singles = [E.Box.from_workload(w, device=device) for w in wls]
    for s_, dt in zip(singles, dts):
        s_.step(args.warmup, dt)
    torch.cuda.synchronize(device)
    ev0.record(stream)
    for _ in range(steps):
        for s_, dt in zip(singles, dts):
            s_.step(1, dt)
    ev1.record(stream)
    torch.cuda.synchronize(device)
    single_ms = max_over_ranks(dist, ev0.elapsed_time(ev1), device)
    for s_ in singles:
        s_.sync()
    del singles
    torch.cuda.empty_cache()
    return {"workload": f"sweep_{args.nbox}_boxes", "particles_per_gpu": P, "steps": steps,
            "value": world * P * steps / (batched_ms * 1e-3), "ms_per_step": batched_ms / steps,
            "launches_per_step": launches / steps, "autotune_choice": choice, "autotune_ms": list(cand_ms),
            "one_at_a_time": {"value": world * P * steps / (single_ms * 1e-3), "ms_per_step": single_ms / steps},
            "vs_plain": single_ms / batched_ms}


def measure_adjoint(dist, device, world, reps=1, nz=0, ndir=0, steps=0, record=None):
    """Gradient of log <|n_emu|> after the growth-phase run (256 cells x 96
    directions, 400 steps, checkpoints every 20 steps) through the adjoint's
    autograd Function, against the plain forward steps of the same run.
    Times (CUDA events): plain = the 400 steps alone; forward = initialisation,
    checkpointed steps and moments; backward = seed, checkpoint recomputation,
    400 adjoint steps and the chain rule through Eq. 8."""
    import torch

    from paper_2101_02745_gb300 import emu as E
    from paper_2101_02745_gb300 import workloads as W
    from paper_2101_02745_gb300.adjoint import Evolve, Simulation, objectives

    wl = W.adjoint_box()
    if nz or ndir or steps:
        wl = W.adjoint_box(nz=nz or wl.nz, ndir=ndir or wl.ndir, steps=steps or wl.steps)
    box = E.Box.from_workload(wl, device=device)
    dt = box.timestep()
    sim = Simulation(box, wl.steps, dt, every=wl.meta["checkpoint_every"], alpha=wl.alpha, seed=wl.seed,
                     record=record)
    stream = box.stream
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    best = None
    for r in range(reps + 1):            # the first pass is a warm-up
        box.init(wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar, wl.dirs, wl.alpha, wl.seed)
        torch.cuda.synchronize(device)
        ev[0].record(stream)
        box.step(wl.steps, dt)
        ev[1].record(stream)
        leaves = [torch.tensor(a, dtype=torch.float64, device=device, requires_grad=True)
                  for a in (wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar)]
        n0 = box.launches()
        ev[2].record(stream)
        L = objectives(Evolve.apply(*leaves, sim))
        ev[3].record(stream)
        L[1].backward()
        ev[4].record(stream)
        torch.cuda.synchronize(device)
        launches = box.launches() - n0
        t = [ev[i].elapsed_time(ev[i + 1]) for i in (0, 2, 3)]
        if r > 0 and (best is None or sum(t[1:]) < sum(best[1:])):
            best = t
    plain, fwd, bwd = (max_over_ranks(dist, x, device) for x in best)
    upd = wl.P * wl.steps
    return {"workload": wl.name, "particles": wl.P, "steps": wl.steps, "checkpoint_every": sim.every,
            "value": world * upd / ((fwd + bwd) * 1e-3), "unit": "differentiated particle-updates/s",
            "plain_value": world * upd / (plain * 1e-3),
            "plain_ms": plain, "forward_ms": fwd, "backward_ms": bwd,
            "backward_over_forward": bwd / fwd, "vs_plain": plain / (fwd + bwd), "recorded": sim.use_record(),
            "launches_per_gradient": launches}


def run_adjoint(args, rank, world, local_rank):
    """--workload adjoint: one line whose value is the gradient's throughput."""
    import torch

    from paper_2101_02745_gb300 import build as B

    if rank == 0:
        B.build()
    dist = dist_init(world, True)
    device = torch.device("cuda", local_rank)
    torch.cuda.set_device(device)
    barrier(dist, device)
    clocks = ClockSampler(device.index).start()
    record = {"auto": None, "on": True, "off": False}[args.adj_record]
    a = measure_adjoint(dist, device, world, reps=args.steps, nz=args.nz, ndir=args.ndir, steps=args.adj_steps,
                        record=record)
    clk = clocks.stop()
    if rank == 0:
        line = {"metric": METRIC, "value": a["value"], "unit": a["unit"], "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": (a["forward_ms"] + a["backward_ms"]) / a["steps"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": a["workload"], "particles_per_gpu": a["particles"], "steps": a["steps"],
                           "checkpoint_every": a["checkpoint_every"], "recorded": a["recorded"],
                           "l2": ("particle state %.2f GB %s L2 (129 MB)"
                                  % (a["particles"] * 480 / 1e9,
                                     "above" if a["particles"] * 480 > 129e6 else "below"))},
                "adjoint": a, "gpu_launches": a["launches_per_gradient"], "clocks": clk}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_sweep(args, rank, world, local_rank):
    """--workload sweep: the batched sweep's own line (value = batched rate)."""
    import torch

    from paper_2101_02745_gb300 import build as B

    if rank == 0:
        B.build()
    dist = dist_init(world, True)
    device = torch.device("cuda", local_rank)
    torch.cuda.set_device(device)
    barrier(dist, device)
    clocks = ClockSampler(device.index).start()
    r = measure_sweep(args, dist, device, rank, world, args.steps)
    clk = clocks.stop()
    if rank == 0:
        line = {
            "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": r["workload"], "boxes": args.nbox, "particles_per_gpu": r["particles_per_gpu"],
                       "nz_range": [64, 1024], "ndir_range": [48, 378],
                       "l2": "inputs larger than L2 (particle state %.1f GB per GPU)"
                             % (r["particles_per_gpu"] * 480 / 1e9)},
            "batched": r, "speedup": r["vs_plain"],
            "gpu_launches": int(r["launches_per_step"] * args.steps), "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="throughput_1d",
                    choices=["throughput_1d", "paper_1d", "paper_1d_asym", "tiny_fiducial", "sweep", "adjoint",
                             "box_3d", "anywhere"])
    ap.add_argument("--nbox", type=int, default=256, help="boxes of the sweep workload")
    ap.add_argument("--n3", type=int, default=0, help="cells per axis of the 3D box (default 64)")
    ap.add_argument("--ndir3", type=int, default=0, help="directions per cell of the 3D box (default 16)")
    ap.add_argument("--nz", type=int, default=0, help="cells of the throughput workload (profiling runs)")
    ap.add_argument("--ndir", type=int, default=0, help="directions of the throughput workload (profiling runs)")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--ref-cells", type=int, default=256, help="cells per oracle step in --impl reference")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--choice", type=int, default=-1,
                    help="launch configuration of the main box (autotuner candidate index; default: autotune)")
    ap.add_argument("--adj-steps", type=int, default=0, help="steps of the adjoint workload (default 400)")
    ap.add_argument("--adj-record", choices=["auto", "on", "off"], default="auto",
                    help="adjoint backward with per-step records (auto: large boxes)")
    ap.add_argument("--shape-order", type=int, default=2, choices=[0, 1, 2, 3], help="particle shape (Sec. 2.2.1)")
    ap.add_argument("--osc", action="store_true", help="add the vacuum and matter terms of Eq. 2")
    ap.add_argument("--no-fp64-peak", action="store_true", help="skip the in-run DGEMM measurement of the FP64 peak")
    ap.add_argument("--fp64-peak", action="store_true", help="only measure and print the FP64 peak (DGEMM)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched-sweep and adjoint comparisons of the default line")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local_rank = dist_env()
    if args.fp64_peak:
        import torch
        torch.cuda.set_device(local_rank)
        print(json.dumps({"fp64_peak": fp64_peak(torch.device("cuda", local_rank), reps=max(args.steps, 1))}))
        return 0
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "sweep":
        return run_sweep(args, rank, world, local_rank)
    if args.workload == "adjoint":
        return run_adjoint(args, rank, world, local_rank)
    if args.workload == "box_3d":
        return run_box3d(args, rank, world, local_rank)
    if args.workload == "anywhere":
        return run_anywhere(args, rank, world, local_rank)
    return run_gpu(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
