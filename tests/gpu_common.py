"""Helpers shared by the GPU parity tests: configurations, the oracle Problem
matching a synth.Config, and error metrics."""
import numpy as np

from oracle import oracle as O
from paper_1910_01031_gb300 import iewpf, synth


def oracle_problem(cfg):
    return O.Problem(nx=cfg.nx, ny=cfg.ny, dx=cfg.dx, dy=cfg.dy, g=cfg.g, f=cfg.f, H=cfg.H, theta=cfg.theta,
                     courant=cfg.courant, dt_model=cfg.dt_model, c_omega=cfg.c_omega, q0=cfg.q0, L0=cfg.L0,
                     seed=cfg.seed, obs_sigma=cfg.obs_sigma)


def ensemble(cfg, mooring_xy=None, n_drifters_max=0, n_obs_max=None):
    return iewpf.Ensemble(iewpf.params_from_config(cfg, n_drifters_max=n_drifters_max, n_obs_max=n_obs_max),
                          mooring_xy=mooring_xy)


def start_state(cfg, ne, seed=7):
    """float32 initial ensemble and the same values in float64 for the oracle."""
    U32 = synth.initial_state(cfg, ne, seed=seed).astype(np.float32)
    return U32, U32.astype(np.float64)


def rel_l2(a, b):
    """Relative L2 error of a state against the reference, the largest over
    particles of two norms: the surface elevation eta alone, and the
    momentum (hu, hv) together (the two carry different units; hv alone can
    be nearly zero in a zonal jet)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if a.ndim == 3:
        a, b = a[None], b[None]
    out = 0.0
    for sl in (slice(0, 1), slice(1, 3)):
        num = np.sqrt(np.sum((a[:, sl] - b[:, sl]) ** 2, axis=(1, 2, 3)))
        den = np.sqrt(np.sum(b[:, sl] ** 2, axis=(1, 2, 3)))
        out = max(out, float(np.max(num / np.maximum(den, 1e-30))))
    return out


def ragged_config(**kw):
    """72 x 50 cells: partial tiles in x and y and a 2-cell seam of the
    coarse grid in y."""
    args = {"n_particles": 4, "n_obs": 3}
    args.update(kw)
    return synth.Config("ragged_72x50", 72, 50, **args)
