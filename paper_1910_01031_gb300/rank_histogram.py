"""Rank-histogram experiment (Sec. 5.1) on synthetic truths.

Many independent data-assimilation experiments run together as one batch of
problems (one persistent launch per phase, the cycle as a CUDA graph).
Experiment e has its own truth (particle e of a separate truth ensemble,
drawn from the same initial distribution and the same model error as the
members) and its own N_e-member ensemble.  Every five minutes the truth's
(hu, hv) at the moorings, plus observation error, is assimilated; after the
assimilation period the members and the truths run a free forecast, and the
rank of each observed value at the rank cells within the perturbed members is
taken on the GPU (iewpf_rank).  The accumulated histogram over all cells and
both components should be flat when the filter's spread is right.

    python -m paper_1910_01031_gb300.rank_histogram --experiments 1222 --hours-da 6

(the paper's size: 1222 experiments of 40 members, 6 h of assimilation, a
1 h forecast).  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import iewpf, synth


def _device_states(torch, cfg, n, seed, device):
    """n particles of the initial distribution (the jet of synth plus eta
    noise of noise_std), generated on the device."""
    eta_y, hu_y = synth._jet(cfg)
    g = torch.Generator(device=device).manual_seed(int(seed))
    U = torch.zeros((n, 3, cfg.ny, cfg.nx), dtype=torch.float32, device=device)
    U[:, 0] = torch.as_tensor(eta_y, dtype=torch.float32, device=device)[None, :, None]
    U[:, 1] = torch.as_tensor(hu_y, dtype=torch.float32, device=device)[None, :, None]
    U[:, 0] += cfg.noise_std * torch.randn((n, cfg.ny, cfg.nx), generator=g, device=device)
    return U


def _values_at(torch, U, cells):
    """(eta, hu, hv) of every particle of U at integer cells: [n][ncells][3]."""
    c = torch.as_tensor(np.asarray(cells), dtype=torch.long, device=U.device)
    return U[:, :, c[:, 1], c[:, 0]].permute(0, 2, 1).double().cpu().numpy()


def _observe(cfg, vals, noise):
    """Mooring-type observations (eq. buoyObservation) from (eta, hu, hv) at
    the cells: (hu, hv) H/(H + eta) plus the noise."""
    s = cfg.H / (cfg.H + vals[:, 0])
    return np.stack([vals[:, 1] * s, vals[:, 2] * s], axis=1) + noise


def run(experiments=64, ne=40, hours_da=1.0, hours_fc=1.0, scheme=iewpf.TWO_STAGE, seed=2019, nx=500, ny=300):
    import torch
    from scipy.stats import chisquare
    dev = torch.device("cuda")
    cfg = synth.config_rank(n_particles=ne)
    if (nx, ny) != (500, 300):
        cfg = synth.Config("rank_%dx%d" % (nx, ny), nx, ny, **{k: v for k, v in cfg.as_dict().items()
                                                                if k not in ("name", "nx", "ny")})
    moor = synth.rank_moorings(cfg)
    moor_xy = synth.cell_positions(cfg, moor)
    cells = synth.rank_cells(cfg)
    steps_per_obs = cfg.obs_every_steps
    n_cycles = int(round(hours_da * 3600.0 / (steps_per_obs * cfg.dt_model)))
    n_fc = int(round(hours_fc * 3600.0 / cfg.dt_model))
    params = []
    for e in range(experiments):
        p = iewpf.params_from_config(cfg, n_obs_max=len(moor), scheme=scheme)
        p.instance_id = e
        params.append(p)
    t_setup = time.perf_counter()
    batch = iewpf.Batch(params, [moor_xy] * experiments)
    tp = iewpf.params_from_config(cfg, n_obs_max=0)
    tp.obs_kind = synth.OBS_DRIFTER
    tp.n_particles = experiments
    tp.instance_id = experiments                 # draws independent of every experiment's
    truth = iewpf.Ensemble(tp)
    truth.set_state(_device_states(torch, cfg, experiments, seed, dev))
    for e, inst in enumerate(batch.instances):
        inst.set_state(_device_states(torch, cfg, ne, seed + 1 + e, dev))
    batch.tune()
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    TU = torch.empty((experiments, 3, cfg.ny, cfg.nx), dtype=torch.float32, device=dev)
    work0 = batch.work()[0]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in range(n_cycles):
        truth.forecast(steps_per_obs, True)
        truth.get_state(TU)
        vals = _values_at(torch, TU, moor)
        obs = [(None, _observe(cfg, vals[e], synth.obs_noise(cfg, len(moor), c, seed=seed + 7 * e)))
               for e in range(experiments)]
        batch.cycle(steps_per_obs, obs)
    da_s = time.perf_counter() - t0
    work_da = batch.work()[0] - work0
    t1 = time.perf_counter()
    truth.forecast(n_fc, True)
    before = batch.work()[0]
    batch.forecast(n_fc, True)
    fc_work = batch.work()[0] - before
    truth.get_state(TU)
    vals = _values_at(torch, TU, cells)
    ranks = np.zeros((experiments, len(cells), 2), np.int64)
    for e, inst in enumerate(batch.instances):
        y = _observe(cfg, vals[e], synth.obs_noise(cfg, len(cells), 10 ** 6, seed=seed + 7 * e))
        ranks[e] = inst.rank(cells, y, draw=e)
    torch.cuda.synchronize()
    fc_s = time.perf_counter() - t1
    hist = np.bincount(ranks.ravel(), minlength=ne + 1)
    per_cell = [[np.bincount(ranks[:, m, comp], minlength=ne + 1).tolist() for comp in (0, 1)]
                for m in range(len(cells))]
    out = {
        "workload": "rank histograms: %d experiments x %d members, %dx%d, %d moorings, %.3g h DA + %.3g h forecast"
                    % (experiments, ne, cfg.nx, cfg.ny, len(moor), hours_da, hours_fc),
        "scheme": "one-stage" if scheme == iewpf.ONE_STAGE else "two-stage",
        "experiments": experiments, "members": ne, "cycles": n_cycles, "forecast_steps": n_fc,
        "setup_s": round(setup_s, 3), "da_s": round(da_s, 3), "forecast_and_rank_s": round(fc_s, 3),
        "particle_substeps": int(work_da + fc_work),
        "value": (work_da + fc_work) * cfg.nx * cfg.ny / (da_s + fc_s), "unit": "particle*cell*step/s",
        "rank_cells": cells.tolist(), "histogram": hist.tolist(), "per_cell": per_cell,
        "chi2_pvalue": float(chisquare(hist).pvalue),
        "rank_mean": float(ranks.mean()), "rank_mean_expected": ne / 2.0,
        "edge_fraction": float((hist[0] + hist[-1]) / hist.sum()), "edge_fraction_flat": 2.0 / (ne + 1),
    }
    batch.close()
    truth.close()
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--experiments", type=int, default=64)
    ap.add_argument("--members", type=int, default=40)
    ap.add_argument("--hours-da", type=float, default=1.0)
    ap.add_argument("--hours-fc", type=float, default=1.0)
    ap.add_argument("--scheme", type=int, default=0, choices=[0, 1], help="0 two-stage, 1 one-stage")
    ap.add_argument("--seed", type=int, default=2019)
    args = ap.parse_args()
    print(json.dumps(run(args.experiments, args.members, args.hours_da, args.hours_fc, args.scheme, args.seed)),
          flush=True)


if __name__ == "__main__":
    main()
