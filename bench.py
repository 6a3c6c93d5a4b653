#!/usr/bin/env python
"""Benchmark of the IEWPF hot path on one GB300.

A step is one IEWPF cycle on the 512 x 512, 100-particle, 64-drifter
workload: 5 model steps of 60 s (scheme steps from the CFL condition, model
error after the first 4) followed by one two-stage IEWPF analysis against
64 drifter observations.  Throughput is particle.cell-steps/s
(sum over particles of scheme steps x 512^2 cells per second); the cycle time
is ms_per_step.  The state (2 x 315 MB) exceeds the 129 MB L2, so no flush
is needed between timed steps.

The line also carries three further workloads, each with its own numbers:
"batched" (32 independent problems of 128^2-1024^2 cells advanced together
as one CUDA graph per cycle), "moorings" (1024^2 cells, 1000 particles, 1521
moored buoys: context creation with the dense FP64 factorisation, and the
cycle time) and "surrogate" (a 12 h drift forecast of 1000
particles x 64 drifters on 256^2 cells with the plain stepper and with the
learned surrogate, their times and the distance between the two forecasts).

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores (there is no other implementation to run).
Under torchrun each rank runs an independent replica (own seed).
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
FLOPS_PER_CELL_STEP = 490         # FP32 operations of one scheme step per cell, counted from the scheme


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
    """Workload of one rank: an independent replica of the 512 x 512,
    100-particle problem with its own seed and Philox instance id."""
    from paper_1910_01031_gb300 import synth
    cfg = synth.config2(seed=0x1910_01031 + 104729 * rank)
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


def run_ours(args, rank, world, local):
    import torch
    from paper_1910_01031_gb300 import build, iewpf, synth

    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    cfg, instance = replica(rank)
    ne, N = cfg.n_particles, cfg.nx * cfg.ny
    P = iewpf.params_from_config(cfg)
    P.instance_id = instance
    ens = iewpf.Ensemble(P)
    ens.set_state(synth.initial_state(cfg, ne, seed=7 + rank).astype(np.float32))
    obs = make_observations(cfg, args.warmup + args.steps + 1, rank)
    # pinned host buffers for the per-step inputs and outputs (end-to-end leg)
    pin_xy = [torch.empty((cfg.n_obs, 2), dtype=torch.float64, pin_memory=True) for _ in obs[:-1]]
    pin_val = [torch.empty((cfg.n_obs, 2), dtype=torch.float64, pin_memory=True) for _ in obs[:-1]]
    for k, (xy, val) in enumerate(obs[:-1]):
        pin_xy[k].numpy()[:] = xy
        pin_val[k].numpy()[:] = val
    stream = torch.cuda.ExternalStream(ens.stream())

    def cycle(k):
        ens.forecast(cfg.obs_every_steps - 1, True)
        ens.forecast(1, False)
        return ens.assimilate(pin_xy[k].numpy(), pin_val[k].numpy())

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
    # slowest rank sets the job time
    dev_s, host_s, work_all = combine_ranks(dev_s, host_s, work, world)
    value = work_all * N / dev_s
    e2e_value = work_all * N / host_s
    # the dominant kernel: bare scheme steps, CUDA events on the context stream
    nsub_probe = 26
    dt_probe = cfg.dt_model / 13.0
    ens.substeps(2, dt_probe)           # warm
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    ens.substeps(nsub_probe, dt_probe)
    f1.record(stream)
    f1.synchronize()
    launch_s = f0.elapsed_time(f1) / 1e3 / nsub_probe
    cells = ne * N
    achieved_gbs = BYTES_PER_CELL_STEP * cells / launch_s / 1e9
    achieved_tflops = FLOPS_PER_CELL_STEP * cells / launch_s / 1e12
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12        # TFLOP/s, FMA = 2
    traffic = None
    try:
        prof = json.load(open(os.path.join(ROOT, "profiles", "rk2_march_traffic.json")))
        if prof.get("kernel_sha") == _kernel_sha():
            traffic = prof["bytes_per_cell_step"] * cells
    except Exception:
        pass
    roofline = {"bound": "hbm", "achieved": round(achieved_gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(achieved_gbs / hbm_peak, 4), "traffic": traffic,
                "kernel": "rk2_march_kernel (register-marching SSP-RK2 scheme step), shape (kind, nc, rows, warps) = %s"
                          % (ens.stepper(),),
                "per_launch_ms": round(launch_s * 1e3, 4),
                "alu": {"achieved": round(achieved_tflops, 2), "peak": round(fp32_peak, 1), "unit": "TFLOP/s",
                        "frac": round(achieved_tflops / fp32_peak, 4)}}
    try:
        sir = run_sir_collapse(ens, cfg, *obs[-1])
    except Exception as e:  # reported, the main number stands without it
        sir = {"error": str(e)}
    ens.close()
    try:
        batched = run_batched(rank)
    except Exception as e:  # reported, the main number stands without it
        batched = {"error": str(e)}
    try:
        moorings = run_moorings(rank)
    except Exception as e:  # reported, the main number stands without it
        moorings = {"error": str(e)}
    try:
        surrogate = run_surrogate(rank, epochs=8)
    except Exception as e:  # reported, the main number stands without it
        surrogate = {"error": str(e)}
    try:
        one_stage = run_one_stage(rank)
    except Exception as e:  # reported, the main number stands without it
        one_stage = {"error": str(e)}
    try:
        ranks = run_rank_histogram(rank)
    except Exception as e:  # reported, the main number stands without it
        ranks = {"error": str(e)}
    if rank != 0:
        return
    cpu = cpu_baseline(args) if world == 1 else None
    h2d = 2 * cfg.n_obs * 2 * 8
    d2h = 6 * ne * 8 + 2 * 8
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dev_s / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 state, f64 weights", "data": "synthetic",
        "config": {"workload": "iewpf_cycle_512x512_ne100_64drifters", "nx": cfg.nx, "ny": cfg.ny,
                   "particles": ne, "drifters": cfg.n_obs, "model_steps_per_cycle": cfg.obs_every_steps,
                   "dt_model_s": cfg.dt_model, "c_omega": cfg.c_omega, "courant": cfg.courant,
                   "particle_substeps_timed": int(work_all), "l2": "inputs larger than L2 (state 2x315 MB)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "iewpf_cycle_ms": round(dev_s / args.steps * 1e3, 3),
        "e2e": {"value": round(e2e_value, 1), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "timing": "host wall clock through the C ABI, pinned obs buffers"},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "batched": batched,
        "moorings": moorings,
        "surrogate": surrogate,
        "one_stage": one_stage,
        "sir_collapse": sir,
        "rank_histogram": ranks,
        "cpu_baseline": cpu,
        "clocks": clk,
        "last_cycle": {"beta": d["beta"], "c_bar": d["cbar"], "alpha_min": float(np.min(d["alpha"])),
                       "alpha_max": float(np.max(d["alpha"])),
                       "neglogw_spread": float(np.max(d["neglogw"]) - np.min(d["neglogw"]))} if d else None,
    }
    print(json.dumps(line), flush=True)


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


def run_moorings(rank, cycles=2):
    """The moored-buoy workload: 1024 x 1024 cells, 1000 particles, 1521
    equidistant moorings observing (u, v).  Times the context creation (pull
    stencil, dense 3042 x 3042 HQH^T + R and its FP64 Cholesky on the GPU,
    the 49 x 49 block root) and IEWPF cycles (5 model steps, model error on 4,
    one analysis against the moorings) with CUDA events.  The particles start
    from one synthetic state (they diverge through the model error)."""
    import torch
    from paper_1910_01031_gb300 import iewpf, synth
    cfg = synth.config4(seed=0x1910_01031 + 13 * rank)
    cells = synth.mooring_cells(cfg)
    xy = synth.cell_positions(cfg, cells)
    P = iewpf.params_from_config(cfg)
    P.instance_id = rank
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ens = iewpf.Ensemble(P, mooring_xy=xy)
    create_s = time.perf_counter() - t0
    x = torch.from_numpy(synth.initial_particle(cfg, 0, seed=41 + rank, dtype=np.float32)).cuda()
    ens.set_state(x.unsqueeze(0).expand(cfg.n_particles, -1, -1, -1).contiguous())
    del x
    truth = synth.initial_particle(cfg, 1, seed=43 + rank)
    stream = torch.cuda.ExternalStream(ens.stream())

    def cycle(k):
        ens.forecast(cfg.obs_every_steps - 1, True)
        ens.forecast(1, False)
        y = synth.obs_from_state(cfg, truth, cells, synth.obs_noise(cfg, len(cells), k))
        return ens.assimilate(None, y, diag=False)

    cycle(0)
    torch.cuda.synchronize()
    w0 = ens.work()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(1, cycles + 1):
        cycle(k)
    e1.record(stream)
    e1.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    work = ens.work() - w0
    out = {"workload": "iewpf_1024x1024_ne1000_1521moorings (dense 3042 x 3042 HQH^T + R)",
           "create_s": round(create_s, 3), "cycles_timed": cycles, "cycle_ms": round(secs / cycles * 1e3, 2),
           "value": round(work * cfg.nx * cfg.ny / secs, 1), "unit": UNIT,
           "state_gb": round(2 * cfg.n_particles * cfg.nx * cfg.ny * 12 / 1e9, 1)}
    ens.close()
    torch.cuda.empty_cache()
    return out


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
    """The one-stage IEWPF (App. A) on the headline workload: cycle time
    with CUDA events, and per cycle its target max c_i against the two-stage
    target mean c_i.  The incomplete-gamma alpha (eq. numericalEqForAlpha) of
    the last cycle's particles is solved on the GPU as well and compared with
    the Lambert-W alpha the scheme used."""
    import torch
    from paper_1910_01031_gb300 import iewpf, synth
    cfg, instance = replica(rank)
    P = iewpf.params_from_config(cfg, scheme=iewpf.ONE_STAGE)
    P.instance_id = instance
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
    params, (si, so) = net.params(), net.scales()
    net.close()
    ens1.close()
    out["train"] = {"pairs": n_pairs, "grid": "64x64", "epochs": epochs, "batch": batch, "lr": lr,
                    "seconds": round(train_s, 2), "epoch_loss": [round(float(v), 5) for v in losses]}
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


def oracle_sample(n_particles=4, seed_rank=0):
    """One IEWPF cycle of the FP64 oracle on n_particles of the 512^2
    workload; returns (particle.cell-steps, seconds, threads)."""
    from oracle import oracle as O
    from paper_1910_01031_gb300 import synth
    cfg = synth.config2()
    P = O.Problem(nx=cfg.nx, ny=cfg.ny, dx=cfg.dx, dy=cfg.dy, g=cfg.g, f=cfg.f, H=cfg.H, theta=cfg.theta,
                  courant=cfg.courant, dt_model=cfg.dt_model, c_omega=cfg.c_omega, q0=cfg.q0, L0=cfg.L0,
                  seed=cfg.seed, obs_sigma=cfg.obs_sigma)
    U = synth.initial_state(cfg, n_particles, seed=7 + seed_rank)
    xy = synth.drifter_positions(cfg)
    cells = [O.obs_cell(P, *p) for p in xy]
    truth = synth.initial_state(cfg, 1, seed=3)[0]
    y = synth.obs_from_state(cfg, truth, np.array(cells), synth.obs_noise(cfg, len(cells), 0))
    K = O.pull_stencil(P)
    M = O.local_block_sqrt(P)
    t0 = time.perf_counter()
    U, nsub, _ = O.forecast(P, U, cfg.obs_every_steps, [1] * (cfg.obs_every_steps - 1) + [0], t0=0)
    U, _ = O.assimilate(P, U, cells, y, t=0, K=K, Msq=M)
    dt = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return float(nsub.sum()) * cfg.nx * cfg.ny, dt, min(threads, os.cpu_count() or 1, n_particles)


def cpu_baseline(args):
    try:
        from oracle import build as ob
        ob.build()
        n = min(100, 2 * (os.cpu_count() or 1))
        work, secs, threads = oracle_sample(n)
        return {"value": round(work / secs, 1), "unit": UNIT, "cores": threads, "kind": "oracle",
                "sample": "1 IEWPF cycle (5 model steps + analysis, 64 drifters) of %d of the 100 particles "
                          "of the 512x512 workload, FP64, OpenMP over particles" % n,
                "seconds": round(secs, 2)}
    except Exception as e:  # the GPU number stands without it
        return {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                "sample": "failed: %s" % e}


def run_reference(args, rank, world):
    if rank != 0:
        return
    from oracle import build as ob
    ob.build()
    total_work, total_s = 0.0, 0.0
    threads = 1
    for k in range(args.warmup + args.steps):
        work, secs, threads = oracle_sample(2, seed_rank=k)
        if k >= args.warmup:
            total_work += work
            total_s += secs
    value = total_work / total_s
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_s / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "iewpf_cycle_512x512_ne100_64drifters", "sample_particles_per_step": 2},
        "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "each step: 1 IEWPF cycle of 2 of the 100 particles of the 512x512 workload"},
        "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
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
