#!/usr/bin/env python
"""Benchmark of the IEWPF hot path on one GB300.

A step is one IEWPF cycle on the largest configuration: 1024 x 1024 cells,
1000 particles, 1521 moored buoys every 26 cells observing (u, v): 5 model
steps of 60 s (scheme steps from the CFL condition, model error after the
first 4) followed by one two-stage IEWPF analysis with the dense 3042 x 3042
HQH^T + R.  Throughput is particle.cell-steps/s (sum over particles of scheme
steps x 1024^2 cells per second); the cycle time is ms_per_step.  The state
(2 x 12.6 GB) exceeds the 129 MB L2, so no flush is needed between timed
steps.  e2e is the same work over the host's clock through the C ABI, the
observations copied from pinned host memory and the diagnostics read back
every cycle.

Further workloads follow on the same line (--legs selects them): "drifters"
(512^2, 100 particles, 64 drifters, with the bare scheme step and the
standard-particle-filter collapse experiment), "coupled" (624^2, 1000
particles, 1521 moorings every 16 cells whose HQH^T + R couples neighbours
and whose FP64 factor fills in), "batched" (32 independent
problems of 128^2-1024^2 cells advanced together as one CUDA graph per
cycle), "surrogate" (a 12 h drift forecast of 1000 particles x 64 drifters
on 256^2 cells with the plain stepper and with the learned surrogate),
"one_stage" and "rank_histogram".

--impl reference times the FP64 CPU oracle on a bounded sample of the
headline workload on the host cores (there is no other implementation to
run).  Under torchrun each rank runs an independent replica (own seed).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle·cell-steps/s"
UNIT = "particle*cell*step/s"
BYTES_PER_CELL_STEP = 24          # read (eta, hu, hv) + write (eta, hu, hv), float32
# FP32 operations of one scheme step per cell (adds, multiplies and fused
# multiply-adds, one each; no halo), counted from the kernel's arithmetic
SCHEME_OPS_PER_CELL_STEP = 260
# issue slots per cell and scheme step measured by ncu at 512^2 x 100
# (smsp__inst_executed.sum x 32 / cells), per stepper kind
ISSUE_PER_CELL_STEP = {1: 524.3, 2: 363.3}
WORKLOAD = "iewpf_cycle_1024x1024_ne1000_1521moorings"
LEGS = ("drifters", "coupled", "batched", "batched_small", "surrogate", "one_stage", "rank_histogram")


def measured_peak(key, default):
    """A peak from MEASURED_PEAKS.json (HBM copy, cuBLAS BF16 burst and
    sustained), else the stated fallback."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get(key, default))
    except Exception:
        return float(default)


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


def make_observations(cfg, n_cycles, rank):
    """Synthetic truth: one particle carrying 64 drifters, run with model
    error; drifter observations (eq. drifterObservation) every 5 minutes."""
    from paper_1910_01031_gb300 import iewpf, synth
    tcfg = synth.Config(**{**cfg.as_dict(), "n_particles": 1, "seed": cfg.seed + 7919 * (rank + 1)})
    truth = iewpf.Ensemble(iewpf.params_from_config(tcfg, n_drifters_max=cfg.n_obs))
    truth.set_state(synth.initial_state(tcfg, 1, seed=1000 + rank).astype(np.float32))
    xy = synth.drifter_positions(cfg)[None]
    truth.set_drifters(xy)
    obs = []
    dt = cfg.obs_every_steps * cfg.dt_model
    for k in range(n_cycles):
        prev = truth.get_drifters()[0].copy()
        truth.forecast(cfg.obs_every_steps, True)
        cur = truth.get_drifters()[0].copy()
        val = (cur - prev) / dt * cfg.H + synth.obs_noise(cfg, cfg.n_obs, k, seed=17 + rank)
        obs.append((cur, val))
    truth.close()
    return obs


def replica(rank):
    """Workload of one rank: an independent replica of the 1024 x 1024,
    1000-particle, 1521-mooring problem with its own seed and Philox
    instance id."""
    from paper_1910_01031_gb300 import synth
    cfg = synth.config4(seed=0x1910_01031 + 104729 * rank)
    return cfg, rank


def combine_ranks(dev_s, host_s, work, world, device="cuda"):
    """Job totals over the ranks: the slowest rank's device and host times,
    the sum of the work.  Collective only for world > 1."""
    import torch
    t = torch.tensor([dev_s, host_s, float(work)], dtype=torch.float64, device=device)
    if world > 1:
        tw = t.clone()
        torch.distributed.all_reduce(t[:2], op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(tw[2:], op=torch.distributed.ReduceOp.SUM)
        t[2] = tw[2]
    return float(t[0]), float(t[1]), float(t[2])


def device_ensemble(cfg, ne, seed):
    """The initial ensemble built on the device: the two-jet state of
    synth.initial_particle with N(0, noise_std^2) added to eta of every
    particle from torch's seeded generator (the particles are synthetic
    inputs only; the library never sees how they were drawn)."""
    import torch
    from paper_1910_01031_gb300 import synth
    eta_y, hu_y = synth._jet(cfg)
    g = torch.Generator(device="cuda").manual_seed(seed)
    U = torch.zeros((ne, 3, cfg.ny, cfg.nx), dtype=torch.float32, device="cuda")
    U[:, 0] = torch.as_tensor(eta_y, dtype=torch.float32, device="cuda")[None, :, None]
    U[:, 1] = torch.as_tensor(hu_y, dtype=torch.float32, device="cuda")[None, :, None]
    for a in range(0, ne, 100):
        b = min(ne, a + 100)
        U[a:b, 0] += cfg.noise_std * torch.randn((b - a, cfg.ny, cfg.nx), generator=g, device="cuda")
    return U


def scheme_step_roofline(ens, cfg, stream, local, n=13):
    """The dominant kernel alone: n bare scheme steps of the whole ensemble
    timed with CUDA events on the context's stream (the launching stream),
    against HBM (24 algorithmic bytes per cell and step) and against the FP32
    pipe (SCHEME_OPS_PER_CELL_STEP operations, a fused multiply-add counted
    once) and instruction issue."""
    import torch
    ne, N = cfg.n_particles, cfg.nx * cfg.ny
    dt = cfg.dt_model / 13.0
    ens.substeps(2, dt)           # warm
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("scheme_step_%dx%d" % (cfg.nx, cfg.ny))   # selects these launches for a profiler
    f0.record(stream)
    ens.substeps(n, dt)
    f1.record(stream)
    f1.synchronize()
    torch.cuda.nvtx.range_pop()
    launch_s = f0.elapsed_time(f1) / 1e3 / n
    cells = ne * N
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    fp32_ops_peak = n_sm * 128 * sm_mhz * 1e6 / 1e12         # T operations/s on the FP32 pipes
    issue_peak = n_sm * 4 * 32 * sm_mhz * 1e6 / 1e12         # T thread-instructions/s
    achieved_gbs = BYTES_PER_CELL_STEP * cells / launch_s / 1e9
    ops = SCHEME_OPS_PER_CELL_STEP * cells / launch_s / 1e12
    traffic = None
    try:
        prof = json.load(open(os.path.join(ROOT, "profiles", "rk2_march_traffic.json")))
        if prof.get("kernel_sha") == _kernel_sha():
            traffic = prof["bytes_per_cell_step"] * cells
    except Exception:
        pass
    shape = ens.stepper()
    return {"bound": "hbm", "achieved": round(achieved_gbs, 1), "peak": hbm_peak, "unit": "GB/s",
            "frac": round(achieved_gbs / hbm_peak, 4), "traffic": traffic,
            "kernel": "%s (SSP-RK2 scheme step, register march), shape (kind, nc, rows, warps) = %s"
                      % ("rk2_march2_kernel" if shape[0] == 2 else "rk2_march_kernel", shape,),
            "per_launch_ms": round(launch_s * 1e3, 4), "cells_per_launch": cells,
            "fp32": {"achieved": round(ops, 2), "peak": round(fp32_ops_peak, 1), "unit": "Top/s",
                     "frac": round(ops / fp32_ops_peak, 4), "ops_per_cell_step": SCHEME_OPS_PER_CELL_STEP},
            "issue": {"instructions_per_cell_step": ISSUE_PER_CELL_STEP.get(shape[0]),
                      "frac": (round(ISSUE_PER_CELL_STEP[shape[0]] * cells / launch_s / 1e12 / issue_peak, 4)
                               if shape[0] in ISSUE_PER_CELL_STEP else None)}}


def run_ours(args, rank, world, local):
    """The headline workload: IEWPF cycles on 1024 x 1024 cells, 1000
    particles, 1521 moorings observing (u, v) every 26 cells (dense 3042 x
    3042 HQH^T + R), end to end through the C ABI with the observations in
    pinned host memory and the diagnostics read back every cycle."""
    import torch
    from paper_1910_01031_gb300 import build, iewpf, synth

    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    cfg, instance = replica(rank)
    ne, N = cfg.n_particles, cfg.nx * cfg.ny
    cells = synth.mooring_cells(cfg)
    xy = synth.cell_positions(cfg, cells)
    P = iewpf.params_from_config(cfg)
    P.instance_id = instance
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ens = iewpf.Ensemble(P, mooring_xy=xy)
    create_s = time.perf_counter() - t0
    U = device_ensemble(cfg, ne, seed=7 + rank)
    ens.set_state(U)
    del U
    torch.cuda.empty_cache()
    # the truth and its observations (eq. buoyObservation), in pinned buffers
    truth = synth.initial_particle(cfg, ne + 1, seed=43 + rank)
    n_cyc = args.warmup + args.steps + 1
    pin_val = []
    for k in range(n_cyc):
        t = torch.empty((len(cells), 2), dtype=torch.float64, pin_memory=True)
        t.numpy()[:] = synth.obs_from_state(cfg, truth, cells, synth.obs_noise(cfg, len(cells), k, seed=17 + rank))
        pin_val.append(t)
    stream = torch.cuda.ExternalStream(ens.stream())

    def cycle(k):
        ens.forecast(cfg.obs_every_steps - 1, True)
        ens.forecast(1, False)
        return ens.assimilate(None, pin_val[k].numpy())

    for k in range(args.warmup):
        cycle(k)
    clocks = Clocks(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    w0, l0 = ens.work(), ens.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")     # lets a profiler capture only the timed cycles
    e0.record(stream)
    h0 = time.perf_counter()
    for k in range(args.warmup, args.warmup + args.steps):
        d = cycle(k)
    e1.record(stream)
    e1.synchronize()
    h1 = time.perf_counter()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    dev_s = e0.elapsed_time(e1) / 1e3
    host_s = h1 - h0
    work = ens.work() - w0
    launches = ens.launch_count() - l0
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    dev_s, host_s, work_all = combine_ranks(dev_s, host_s, work, world)
    value = work_all * N / dev_s
    e2e_value = work_all * N / host_s
    roofline = scheme_step_roofline(ens, cfg, stream, local)
    ens.close()
    torch.cuda.empty_cache()
    legs = set(LEGS) if args.legs == "all" else set(x for x in args.legs.split(",") if x and x != "none")
    side = {}
    for name, fn in (("drifters", run_drifters), ("coupled", run_coupled), ("batched", run_batched),
                     ("batched_small", run_batched_small), ("surrogate", run_surrogate),
                     ("one_stage", run_one_stage), ("rank_histogram", run_rank_histogram)):
        if name in legs:
            try:
                side[name] = fn(rank)
            except Exception as e:  # reported, the main number stands without it
                side[name] = {"error": str(e)}
    if rank != 0:
        return
    cpu = cpu_baseline(args) if world == 1 and not args.no_cpu_baseline else None
    h2d = len(cells) * 2 * 8
    d2h = 6 * ne * 8 + 2 * 8
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dev_s / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 state, f64 weights", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": cfg.nx, "ny": cfg.ny,
                   "particles": ne, "moorings": len(cells), "n_y": 2 * len(cells),
                   "model_steps_per_cycle": cfg.obs_every_steps, "dt_model_s": cfg.dt_model,
                   "c_omega": cfg.c_omega, "courant": cfg.courant, "hqht": "dense (couplings kept)",
                   "particle_substeps_timed": int(work_all),
                   "l2": "inputs larger than L2 (state 2 x %.1f GB)" % (ne * N * 12 / 1e9),
                   "parallelism": "replicas" if world > 1 else "single"},
        "iewpf_cycle_ms": round(dev_s / args.steps * 1e3, 3),
        "create_s": round(create_s, 3),
        "e2e": {"value": round(e2e_value, 1), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "timing": "host wall clock through the C ABI, pinned obs buffers"},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "clocks": clk,
        "last_cycle": {"beta": d["beta"], "c_bar": d["cbar"], "alpha_min": float(np.min(d["alpha"])),
                       "alpha_max": float(np.max(d["alpha"])),
                       "neglogw_spread": float(np.max(d["neglogw"]) - np.min(d["neglogw"]))} if d else None,
    }
    line.update(side)
    print(json.dumps(line), flush=True)


def run_drifters(rank, cycles=10, warm=3):
    """The 512 x 512, 100-particle, 64-drifter workload: IEWPF cycles timed
    with CUDA events on the context's stream (drifter observations from two
    GPS fixes of a truth run), the bare scheme step, and the collapse
    experiment of the standard particle filter on the same ensemble."""
    import torch
    from paper_1910_01031_gb300 import iewpf, synth
    cfg = synth.config2(seed=0x1910_01031 + 104729 * rank)
    ne, N = cfg.n_particles, cfg.nx * cfg.ny
    P = iewpf.params_from_config(cfg)
    P.instance_id = 100 + rank
    ens = iewpf.Ensemble(P)
    ens.set_state(synth.initial_state(cfg, ne, seed=7 + rank).astype(np.float32))
    obs = make_observations(cfg, warm + cycles + 1, rank)
    stream = torch.cuda.ExternalStream(ens.stream())

    def cycle(k):
        ens.forecast(cfg.obs_every_steps - 1, True)
        ens.forecast(1, False)
        return ens.assimilate(*obs[k])

    for k in range(warm):
        cycle(k)
    torch.cuda.synchronize()
    w0, l0 = ens.work(), ens.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("drifters_timed")
    e0.record(stream)
    for k in range(warm, warm + cycles):
        cycle(k)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.nvtx.range_pop()
    secs = e0.elapsed_time(e1) / 1e3
    work = ens.work() - w0
    out = {"workload": "iewpf_cycle_512x512_ne100_64drifters", "cycles_timed": cycles,
           "cycle_ms": round(secs / cycles * 1e3, 3), "value": round(work * N / secs, 1), "unit": UNIT,
           "gpu_launches_per_cycle": round((ens.launch_count() - l0) / cycles, 1)}
    out["scheme_step"] = scheme_step_roofline(ens, cfg, stream, torch.cuda.current_device(), n=26)
    try:
        out["sir_collapse"] = run_sir_collapse(ens, cfg, *obs[-1])
    except Exception as e:
        out["sir_collapse"] = {"error": str(e)}
    ens.close()
    torch.cuda.empty_cache()
    return out


def run_batched(rank):
    """The 32-problem batched workload (grids 128^2..1024^2, 20-500
    particles, 4-128 drifters): one CUDA-graph cycle per problem set, timed
    with CUDA events on the batch stream.  Each problem's particles start
    from one synthetic state (they diverge through the model error)."""
    import torch
    from paper_1910_01031_gb300 import iewpf, synth
    cfgs = synth.config3()
    params = []
    for i, c in enumerate(cfgs):
        p = iewpf.params_from_config(c)
        p.instance_id = i + 32 * rank
        params.append(p)
    batch = iewpf.Batch(params)
    for i, c in enumerate(cfgs):
        x = torch.from_numpy(synth.initial_particle(c, 0, seed=100 + i, dtype=np.float32)).cuda()
        U = x.unsqueeze(0).expand(c.n_particles, -1, -1, -1).contiguous()
        batch.instances[i].set_state(U)
        del U, x
    torch.cuda.synchronize()

    def obs(k):
        out = []
        for c in cfgs:
            xy = synth.drifter_positions(c) + 1000.0 * k
            cells = np.stack([np.floor(xy[:, 0] / c.dx) % c.nx, np.floor(xy[:, 1] / c.dy) % c.ny], 1).astype(int)
            truth = synth.initial_particle(c, 1, seed=300)
            out.append((xy, synth.obs_from_state(c, truth, cells, synth.obs_noise(c, len(cells), k))))
        return out

    warm, steps = 1, 2
    o = [obs(k) for k in range(warm + steps)]
    for k in range(warm):
        batch.cycle(5, o[k])
    torch.cuda.synchronize()
    stream = torch.cuda.ExternalStream(batch.stream())
    w0, l0 = batch.work()
    iw0 = [inst.work() for inst in batch.instances]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(warm, warm + steps):
        batch.cycle(5, o[k])
    e1.record(stream)
    e1.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    w1, l1 = batch.work()
    iw1 = [inst.work() for inst in batch.instances]
    pcs = sum((b - a) * c.nx * c.ny for a, b, c in zip(iw0, iw1, cfgs))
    total_pc = sum(c.n_particles * c.nx * c.ny for c in cfgs)
    out = {"workload": "32 problems, grids 128^2-1024^2, 20-500 particles, 4-128 drifters (seeded draw)",
           "particle_cells": total_pc, "cycles_timed": steps, "cycle_ms": round(secs / steps * 1e3, 2),
           "value": round(pcs / secs, 1), "unit": UNIT, "cuda_graph": True,
           "particle_substeps_timed": int(w1 - w0),
           "state_gb": round(sum(c.n_particles * c.nx * c.ny * 24 for c in cfgs) / 1e9, 1)}
    out["kernel_nodes_captured"] = int(l1)
    batch.close()
    torch.cuda.empty_cache()
    return out


def run_coupled(rank, cycles=3):
    """Moorings that interact: 1521 moorings every 16 cells on 624 x 624
    cells, 1000 particles.  Each mooring lies within the 21-cell pull stencil
    of its neighbours, so HQH^T + R (3042 x 3042, FP64) couples them and its
    Cholesky factor fills in.  Times the context creation (assembly and
    factorisation on the GPU), the analysis alone and the whole cycle with
    CUDA events, and reports the factor's fill."""
    import torch
    from paper_1910_01031_gb300 import iewpf, synth
    cfg = synth.coupled_moorings(seed=0x1910_01031 + 31 * rank)
    ne = cfg.n_particles
    cells = synth.mooring_cells(cfg, synth.COUPLED_SPACING)
    xy = synth.cell_positions(cfg, cells)
    P = iewpf.params_from_config(cfg)
    P.instance_id = 300 + rank
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ens = iewpf.Ensemble(P, mooring_xy=xy)
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t0
    n, nnz = ens.factor_info()
    ens.set_state(device_ensemble(cfg, ne, seed=51 + rank))
    torch.cuda.empty_cache()
    ens.tune()                  # the stepper's autotuner, outside the timed cycles
    truth = synth.initial_particle(cfg, ne + 1, seed=53 + rank)
    ys = [synth.obs_from_state(cfg, truth, cells, synth.obs_noise(cfg, len(cells), k)) for k in range(cycles + 1)]
    stream = torch.cuda.ExternalStream(ens.stream())
    ev = lambda: torch.cuda.Event(enable_timing=True)
    ana_ms = []
    e0, e1 = ev(), ev()
    torch.cuda.nvtx.range_push("coupled_timed")
    for k in range(cycles + 1):
        ens.forecast(cfg.obs_every_steps - 1, True)
        ens.forecast(1, False)
        if k == 1:
            e0.record(stream)
        a0, a1 = ev(), ev()
        a0.record(stream)
        ens.assimilate(None, ys[k], diag=False)
        a1.record(stream)
        a1.synchronize()
        if k >= 1:
            ana_ms.append(a0.elapsed_time(a1))
    e1.record(stream)
    e1.synchronize()
    torch.cuda.nvtx.range_pop()
    secs = e0.elapsed_time(e1) / 1e3
    ens.close()
    torch.cuda.empty_cache()
    solve_flops = 4.0 * nnz * ne + 2.0 * n * ne      # two triangular solves per particle
    ana_s = float(np.median(ana_ms)) / 1e3
    return {"workload": "iewpf_cycle_624x624_ne1000_1521moorings_every16 (coupled dense HQH^T + R)",
            "create_s": round(create_s, 3), "n_y": n, "factor_nnz_below_diag": nnz,
            "factor_fill": round(nnz / (n * (n - 1) / 2.0), 4), "cycles_timed": cycles,
            "cycle_ms": round(secs / cycles * 1e3, 2), "analysis_ms": round(ana_s * 1e3, 2),
            "solve_fp64_flops_per_analysis": solve_flops,
            "solve_fp64_gflops_lower_bound": round(solve_flops / ana_s / 1e9, 1)}


def run_batched_small(rank, n=64, cycles=4, warm=1):
    """Where batching pays: 64 independent problems of the 64 x 64,
    10-particle, 1-drifter configuration, each far too small to fill the GPU.
    The same cycles (5 model steps, model error on 4, one analysis) run once
    as one batched CUDA-graph cycle of all problems and once problem by
    problem through their own contexts; both are timed on the host's clock
    around whole cycles (the batch with its stream synchronised)."""
    import torch
    from paper_1910_01031_gb300 import iewpf, synth
    cfgs = [synth.config1(seed=0x1910_01031 + 7 * i + 1009 * rank) for i in range(n)]
    params = []
    for i, c in enumerate(cfgs):
        p = iewpf.params_from_config(c)
        p.instance_id = 400 + i + 64 * rank
        params.append(p)
    states = [synth.initial_state(c, c.n_particles, seed=61 + i).astype(np.float32) for i, c in enumerate(cfgs)]

    def obs(k):
        out = []
        for i, c in enumerate(cfgs):
            xy = synth.drifter_positions(c) + 500.0 * k
            cells = np.stack([np.floor(xy[:, 0] / c.dx) % c.nx, np.floor(xy[:, 1] / c.dy) % c.ny], 1).astype(int)
            truth = synth.initial_particle(c, 1000 + i, seed=71)
            out.append((xy, synth.obs_from_state(c, truth, cells, synth.obs_noise(c, len(cells), k))))
        return out

    o = [obs(k) for k in range(warm + cycles)]
    cells_total = sum(c.n_particles * c.nx * c.ny for c in cfgs)
    # batched
    batch = iewpf.Batch(params)
    for i in range(n):
        batch.instances[i].set_state(states[i])
    for k in range(warm):
        batch.cycle(5, o[k])
    bstream = torch.cuda.ExternalStream(batch.stream())
    torch.cuda.synchronize()
    iw0 = [inst.work() for inst in batch.instances]
    t0 = time.perf_counter()
    for k in range(warm, warm + cycles):
        batch.cycle(5, o[k])
    bstream.synchronize()
    b_s = time.perf_counter() - t0
    b_work = sum((inst.work() - a) * c.nx * c.ny for inst, a, c in zip(batch.instances, iw0, cfgs))
    batch.close()
    # one by one
    ens = [iewpf.Ensemble(p) for p in params]
    for e, U in zip(ens, states):
        e.set_state(U)

    def one_by_one(k):
        for i, e in enumerate(ens):
            e.forecast(4, True)
            e.forecast(1, False)
            e.assimilate(*o[k][i], diag=False)

    for k in range(warm):
        one_by_one(k)
    torch.cuda.synchronize()
    w0 = [e.work() for e in ens]
    t0 = time.perf_counter()
    for k in range(warm, warm + cycles):
        one_by_one(k)
    torch.cuda.synchronize()
    s_s = time.perf_counter() - t0
    s_work = sum((e.work() - a) * c.nx * c.ny for e, a, c in zip(ens, w0, cfgs))
    for e in ens:
        e.close()
    torch.cuda.empty_cache()
    return {"workload": "64 problems of 64x64 cells, 10 particles, 1 drifter (each too small to fill the GPU)",
            "particle_cells": cells_total, "cycles_timed": cycles,
            "batched": {"cycle_ms": round(b_s / cycles * 1e3, 2), "value": round(b_work / b_s, 1)},
            "one_by_one": {"cycle_ms": round(s_s / cycles * 1e3, 2), "value": round(s_work / s_s, 1)},
            "unit": UNIT, "speedup": round((b_work / b_s) / (s_work / s_s), 2)}


def run_sir_collapse(ens, cfg, xy, y):
    """The collapse experiment of the standard particle filter (Sec. 5.3) on
    the headline ensemble after its assimilation cycles, run on to the next
    observation time: every size 1..64 of drifter subsets, 50 random subsets
    each, with R and 10 R; the mean number of particles whose weight is above
    1/N_e per size.  Timed per call (host wall clock through the C ABI: the
    innovations, the weights of 3200 subsets, the copies)."""
    import torch
    from paper_1910_01031_gb300 import synth
    ens.forecast(cfg.obs_every_steps - 1, True)
    ens.forecast(1, False)
    out = {"workload": "SIR weights on the 512x512 ne100 ensemble, 64 drifters, sizes 1..64 x 50 subsets, R and 10R"}
    sets = [synth.observation_subsets(cfg.n_obs, k, 50) for k in range(1, cfg.n_obs + 1)]
    for r_scale in (1.0, 10.0):
        means = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for S in sets:
            _, kept = ens.sir_weights(xy, y, S, r_scale, weights=False)
            means.append(round(float(kept.mean()), 2))
        secs = time.perf_counter() - t0
        out["R" if r_scale == 1.0 else "10R"] = {"mean_kept_by_size": means, "seconds": round(secs, 4),
                                                 "subsets_per_s": round(len(sets) * 50 / secs, 1)}
    return out


def run_one_stage(rank, cycles=3):
    """The one-stage IEWPF (App. A) on the 512^2 drifter workload: cycle time
    with CUDA events, and per cycle its target max c_i against the two-stage
    target mean c_i.  The incomplete-gamma alpha (eq. numericalEqForAlpha) of
    the last cycle's particles is solved on the GPU as well and compared with
    the Lambert-W alpha the scheme used."""
    import torch
    from paper_1910_01031_gb300 import iewpf, synth
    cfg = synth.config2(seed=0x1910_01031 + 104729 * rank)
    P = iewpf.params_from_config(cfg, scheme=iewpf.ONE_STAGE)
    P.instance_id = 200 + rank
    ens = iewpf.Ensemble(P)
    ens.set_state(synth.initial_state(cfg, cfg.n_particles, seed=7 + rank).astype(np.float32))
    obs = make_observations(cfg, cycles + 1, rank)
    stream = torch.cuda.ExternalStream(ens.stream())

    def cycle(k):
        ens.forecast(cfg.obs_every_steps - 1, True)
        ens.forecast(1, False)
        return ens.assimilate(*obs[k])

    cycle(0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gaps = []
    e0.record(stream)
    for k in range(1, cycles + 1):
        d = cycle(k)
        gaps.append(round(d["w_target"] - d["cbar"], 3))
    e1.record(stream)
    e1.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    N = 3.0 * cfg.nx * cfg.ny
    cstar = d["w_target"] - d["c"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ag = iewpf.alpha_gamma(d["gamma"], cstar, N)
    g_s = time.perf_counter() - t0
    moved = cstar > 0
    ratio = (1.0 - ag[moved]) / (1.0 - d["alpha"][moved]) if moved.any() else np.array([1.0])
    out = {"workload": "iewpf_cycle_512x512_ne100_64drifters, one-stage scheme",
           "cycles_timed": cycles, "cycle_ms": round(secs / cycles * 1e3, 3),
           "w_target_minus_cbar": gaps,
           "alpha_gamma": {"particles": int(len(ag)), "N_psi": N, "seconds": round(g_s, 4),
                           "min_alpha": float(ag.min()),
                           "one_minus_alpha_ratio_gamma_over_lambert": {
                               "min": round(float(ratio.min()), 4), "median": round(float(np.median(ratio)), 4),
                               "max": round(float(ratio.max()), 4)}}}
    ens.close()
    return out


def run_rank_histogram(rank):
    """The rank-histogram experiment (Sec. 5.1) at a reduced count: 64
    experiments x 40 members on 500 x 300 cells, 120 moorings, 1 h of
    assimilation and a 1 h forecast (the paper: 1222 experiments, 6 h)."""
    from paper_1910_01031_gb300 import rank_histogram
    return rank_histogram.run(experiments=64, ne=40, hours_da=1.0, hours_fc=1.0, seed=2019 + 31 * rank)


SUR_FLOPS_PER_PIXEL = 2 * 9 * (3 * 64 + 4 * 64 * 64 + 64 * 3)   # algorithmic (unpadded) FLOPs of one network call


def run_surrogate(rank, n_pairs=20000, epochs=8, batch=32, lr=1e-3, hours=12.0, k=10, ne=1000, train_ne=500):
    """The learned-surrogate workload: the network is trained on n_pairs
    pairs (psi, 10 model steps of psi) of the 64 x 64 jet model (a 500-particle
    ensemble of it), its weights are moved to a 256 x 256 network, and a
    12 h drift forecast of 1000 particles x 64 drifters runs twice from the
    same ensemble and counters: with the plain stepper and with the
    surrogate (model error from the same Philox draws in both).  Reports the
    time of both, the RMS and largest drifter distance between the two
    forecasts at every hour, the forecast error E(t) of both against a truth
    run and its difference at 12 h, and the tensor-core rate of a network
    call."""
    import torch
    from paper_1910_01031_gb300 import iewpf, synth
    out = {"workload": "surrogate_256x256_ne%d_64drifters, %g h drift forecast, network 6 x conv3x3 (64 ch), "
                       "k = %d model steps per call" % (ne, hours, k)}
    cfg1 = synth.config1(n_particles=train_ne, seed=0x1910_01031 + 7 * rank)
    p1 = iewpf.params_from_config(cfg1)
    p1.instance_id = 2000 + rank
    ens1 = iewpf.Ensemble(p1)
    ens1.set_state(synth.initial_state(cfg1, train_ne, seed=21 + rank).astype(np.float32))
    net = iewpf.Surrogate(cfg1.nx, cfg1.ny, 64, 6, seed=rank)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = net.train(ens1, n_pairs=n_pairs, k_steps=k, epochs=epochs, batch=batch, lr=lr)
    train_s = time.perf_counter() - t0
    epochs_s = net.train_time()
    tc_train = net.uses_tcgen05_training()
    params, (si, so) = net.params(), net.scales()
    net.close()
    ens1.close()
    # tensor-core work of one optimizer step per pixel: forward, data passes
    # of layers 1..5 and weight gradients of all six layers (the 3 used
    # channels of the network's input and output)
    fwd = 2 * 9 * (3 * 64 + 4 * 64 * 64 + 64 * 3)
    flop_px = fwd + (fwd - 2 * 9 * 3 * 64) + fwd
    steps = epochs * (n_pairs // batch)
    flops = float(flop_px) * batch * cfg1.nx * cfg1.ny * steps
    out["train"] = {"pairs": n_pairs, "grid": "64x64", "epochs": epochs, "batch": batch, "lr": lr,
                    "seconds": round(train_s, 2), "epochs_device_s": round(epochs_s, 3),
                    "path": "tcgen05" if tc_train else "mma.sync", "optimizer_steps": steps,
                    "flops_per_pixel_step": flop_px,
                    "tflops": round(flops / epochs_s / 1e12, 1) if epochs_s > 0 else None,
                    "peak": measured_peak("bf16_tflops_sustained", 1700.0),
                    "frac": round(flops / epochs_s / 1e12 / measured_peak("bf16_tflops_sustained", 1700.0), 4)
                    if epochs_s > 0 else None,
                    "epoch_loss": [round(float(v), 5) for v in losses]}
    cfg = synth.config5(n_particles=ne, seed=0x1910_01031 + 11 * rank)
    P = iewpf.params_from_config(cfg, n_drifters_max=cfg.n_obs)
    P.instance_id = rank
    ens = iewpf.Ensemble(P)
    U0 = torch.empty((ne, 3, cfg.ny, cfg.nx), dtype=torch.float32, device="cuda")
    for a in range(0, ne, 100):
        b = min(ne, a + 100)
        U0[a:b] = torch.from_numpy(np.stack([synth.initial_particle(cfg, i, seed=31 + rank, dtype=np.float32)
                                             for i in range(a, b)]))
    sur = iewpf.Surrogate(cfg.nx, cfg.ny, 64, 6, seed=rank)
    sur.set_params(params)
    sur.set_scales(si, so)
    ens.set_surrogate(sur, k)
    xy0 = synth.drifter_positions(cfg)
    # the truth: one more draw of the initial state with its own model error,
    # its drifters advected by the plain stepper
    Pt = iewpf.params_from_config(synth.Config(**{**cfg.as_dict(), "n_particles": 1}), n_drifters_max=cfg.n_obs)
    Pt.instance_id = 9000 + rank
    truth_ens = iewpf.Ensemble(Pt)
    truth_ens.set_state(synth.initial_particle(cfg, ne + 17, seed=31 + rank, dtype=np.float32)[None])
    truth = truth_ens.drifter_forecast(xy0, hours, 3600.0)[:, 0]
    truth_ens.close()
    stream = torch.cuda.ExternalStream(ens.stream())
    res, errs = {}, {}
    for mode in ("plain", "surrogate"):
        ens.set_state(U0)
        ens.set_counters(0, 0)
        torch.cuda.synchronize()
        w0 = ens.work()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h0 = time.perf_counter()
        E, R, traj = ens.drifter_forecast_errors(xy0, hours, 3600.0, truth, want_traj=True,
                                                 use_surrogate=(mode == "surrogate"))
        e1.record(stream)
        e1.synchronize()
        res[mode] = (traj, time.perf_counter() - h0, e0.elapsed_time(e1) / 1e3, ens.work() - w0)
        errs[mode] = (E, R)
    calls, fallbacks = ens.surrogate_stats()
    d = np.sqrt(np.sum((res["surrogate"][0] - res["plain"][0]) ** 2, axis=-1)) / 1e3     # km, [hour][p][drifter]
    rms = np.sqrt(np.mean(d ** 2, axis=(1, 2)))
    model_steps = int(round(hours * 3600.0 / cfg.dt_model)) * ne
    out["plain"] = {"seconds": round(res["plain"][1], 3), "device_s": round(res["plain"][2], 3),
                    "particle_model_steps_per_s": round(model_steps / res["plain"][1], 1),
                    "particle_substeps": int(res["plain"][3])}
    out["surrogate"] = {"seconds": round(res["surrogate"][1], 3), "device_s": round(res["surrogate"][2], 3),
                        "particle_model_steps_per_s": round(model_steps / res["surrogate"][1], 1),
                        "network_calls": calls, "fallbacks": fallbacks,
                        "particle_substeps_of_fallbacks": int(res["surrogate"][3])}
    out["speedup"] = round(res["plain"][1] / res["surrogate"][1], 3)
    out["drift_distance_km"] = {"rms_by_hour": [round(float(v), 4) for v in rms],
                                "max_at_end": round(float(d[-1].max()), 4),
                                "median_at_end": round(float(np.median(d[-1])), 4)}
    out["within_1km"] = bool(rms[-1] <= 1.0)
    # forecast error against the truth (eqs. errorPerEnsembleDrifter, errorNorm), computed on the GPU
    e_p, e_s = float(errs["plain"][0][-1]) / 1e3, float(errs["surrogate"][0][-1]) / 1e3
    out["forecast_error_km"] = {"E_plain_by_hour": [round(float(v) / 1e3, 3) for v in errs["plain"][0]],
                                "E_surrogate_by_hour": [round(float(v) / 1e3, 3) for v in errs["surrogate"][0]],
                                "RMSE_plain_end": round(float(errs["plain"][1][-1]) / 1e3, 3),
                                "RMSE_surrogate_end": round(float(errs["surrogate"][1][-1]) / 1e3, 3),
                                "abs_E_difference_end": round(abs(e_s - e_p), 4)}
    out["within_1km_E"] = bool(abs(e_s - e_p) <= 1.0)
    pdh = ne * len(xy0) * hours
    out["particle_drifter_hours_per_s"] = {"plain": round(pdh / res["plain"][1], 1),
                                           "surrogate": round(pdh / res["surrogate"][1], 1)}
    # one network call over the whole ensemble, CUDA events on the surrogate stream
    s_stream = torch.cuda.ExternalStream(sur.stream())
    V = U0.clone()
    sur.apply_device(V, stream=ctypes_stream(s_stream))
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 2
    f0.record(s_stream)
    for _ in range(reps):
        sur.apply_device(V, stream=ctypes_stream(s_stream))
    f1.record(s_stream)
    f1.synchronize()
    call_s = f0.elapsed_time(f1) / 1e3 / reps
    flops = SUR_FLOPS_PER_PIXEL * ne * cfg.nx * cfg.ny
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("bf16_tflops", 1900.0))
    out["network_call"] = {"ms_per_ensemble_call": round(call_s * 1e3, 2), "bound": "tensor",
                           "achieved": round(flops / call_s / 1e12, 1), "peak": peak, "unit": "TFLOP/s",
                           "frac": round(flops / call_s / 1e12 / peak, 4),
                           "flops_per_pixel": SUR_FLOPS_PER_PIXEL}
    ens.set_surrogate(None, 0)
    sur.close()
    ens.close()
    del U0, V
    torch.cuda.empty_cache()
    return out


def ctypes_stream(torch_stream):
    import ctypes
    return ctypes.c_void_p(torch_stream.cuda_stream)


def _kernel_sha():
    import hashlib
    h = hashlib.sha1()
    for f in ("march.cu", "march_dev.cuh", "common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1910_01031_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


class OracleSample:
    """A bounded sample of the headline workload run by the FP64 CPU oracle
    (OpenMP over particles in its C scheme, numpy for the analysis):
    n_particles particles of the 1024 x 1024, 1521-mooring problem, stepped
    model step by model step with the cycle's cadence (model error after the
    first four model steps, the analysis after the fifth)."""

    def __init__(self, n_particles, seed_rank=0):
        from oracle import oracle as O
        from paper_1910_01031_gb300 import synth
        self.O = O
        cfg = self.cfg = synth.config4()
        self.P = O.Problem(nx=cfg.nx, ny=cfg.ny, dx=cfg.dx, dy=cfg.dy, g=cfg.g, f=cfg.f, H=cfg.H,
                           theta=cfg.theta, courant=cfg.courant, dt_model=cfg.dt_model, c_omega=cfg.c_omega,
                           q0=cfg.q0, L0=cfg.L0, seed=cfg.seed, obs_sigma=cfg.obs_sigma)
        self.U = np.stack([synth.initial_particle(cfg, i, seed=7 + seed_rank) for i in range(n_particles)])
        self.cells = [tuple(c) for c in synth.mooring_cells(cfg)]
        truth = synth.initial_particle(cfg, 100003, seed=43 + seed_rank)
        self.y = synth.obs_from_state(cfg, truth, np.array(self.cells), synth.obs_noise(cfg, len(self.cells), 0))
        self.K = O.pull_stencil(self.P)
        self.M = O.local_block_sqrt(self.P)
        self.step = 0
        threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        self.threads = min(threads, os.cpu_count() or 1, n_particles)

    def model_step(self):
        """One model step (the analysis too after every fifth); returns
        (particle.cell-steps, seconds)."""
        cfg = self.cfg
        k = self.step % cfg.obs_every_steps
        t0 = time.perf_counter()
        self.U, nsub, _ = self.O.forecast(self.P, self.U, 1, [int(k < cfg.obs_every_steps - 1)], t0=self.step)
        if k == cfg.obs_every_steps - 1:
            self.U, _ = self.O.assimilate(self.P, self.U, self.cells, self.y,
                                          t=self.step // cfg.obs_every_steps, K=self.K, Msq=self.M)
        secs = time.perf_counter() - t0
        self.step += 1
        return float(nsub.sum()) * cfg.nx * cfg.ny, secs


def cpu_baseline(args):
    try:
        from oracle import build as ob
        ob.build()
        n = min(1000, os.cpu_count() or 1)
        sample = OracleSample(n)
        work, secs = 0.0, 0.0
        for _ in range(sample.cfg.obs_every_steps):
            w, t = sample.model_step()
            work += w
            secs += t
        return {"value": round(work / secs, 1), "unit": UNIT, "cores": sample.threads, "kind": "oracle",
                "sample": "1 IEWPF cycle (5 model steps, model error on 4, analysis against 1521 moorings) of "
                          "%d of the 1000 particles of the 1024x1024 workload, FP64, OpenMP over particles" % n,
                "seconds": round(secs, 2)}
    except Exception as e:  # the GPU number stands without it
        return {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                "sample": "failed: %s" % e}


def run_reference(args, rank, world):
    if rank != 0:
        return
    from oracle import build as ob
    ob.build()
    n = min(1000, os.cpu_count() or 1)
    sample = OracleSample(n)
    total_work, total_s = 0.0, 0.0
    for k in range(args.warmup + args.steps):
        work, secs = sample.model_step()
        if k >= args.warmup:
            total_work += work
            total_s += secs
    value = total_work / total_s
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_s / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_particles": n},
        "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": sample.threads, "kind": "oracle",
                         "sample": "each step: one model step of %d of the 1000 particles of the 1024x1024, "
                                   "1521-mooring workload, with the analysis after every fifth (the cycle's "
                                   "cadence)" % n},
        "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="leave out the oracle's CPU timing (profiling runs)")
    ap.add_argument("--legs", default="all",
                    help="side workloads after the headline, comma-separated from %s, 'all' or 'none'"
                         % ",".join(LEGS))
    args = ap.parse_args()
    rank, world, local = _dist()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
