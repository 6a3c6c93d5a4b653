"""Seeded synthetic inputs shaped like the paper's twin experiments.

This module holds no arithmetic of the method itself: it only produces
problem parameters, initial states, observation layouts and observation noise.
Both the CUDA path and the oracle receive identical arrays from it.

Workloads (sizes as in the experiment configurations of this library):
  * ``config1``: periodic 64x64 grid, dx = dy = 2 km, 10 particles, 1 drifter.
  * ``config2``: periodic 512x512 grid, 100 particles, 64 drifters (8x8).
  * ``config3``: 32 independent problems of uneven size (batched mode).
  * ``config4``: periodic 1024x1024 grid, 1000 particles, 1521 moorings
    every 26 cells (39 x 39).
  * ``config5``: 256x256 tiles for the learned surrogate.
Physics for all: H = 230 m, g = 9.81, f = 1.2e-4 1/s, model step 60 s,
Courant number 0.45 on top of the 1/4 of eq. swecfl, model error on a coarse
grid of every 3rd cell with L0 = 0.75 coarse cells and q0 = 5e-4 m,
observations of (hu, hv) with sigma = 0.01 m/s * H every 5 minutes.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field, asdict

import numpy as np

OBS_DRIFTER, OBS_MOORING = 0, 1


@dataclass
class Config:
    name: str
    nx: int
    ny: int
    dx: float = 2000.0
    dy: float = 2000.0
    g: float = 9.81
    f: float = 1.2e-4
    H: float = 230.0
    theta: float = 1.3
    courant: float = 0.45
    dt_model: float = 60.0
    c_omega: int = 3
    q0: float = 5e-4
    L0: float = 0.0
    seed: int = 0x1910_01031
    n_particles: int = 10
    obs_kind: int = OBS_DRIFTER
    n_obs: int = 1
    obs_sigma_vel: float = 0.01
    obs_every_steps: int = 5
    jet_amp: float = 0.1
    jet_width_cells: float = 8.0
    noise_std: float = 1e-3
    dense_S: int = 1

    def __post_init__(self):
        if self.L0 <= 0.0:
            self.L0 = 0.75 * self.c_omega * self.dx

    @property
    def obs_sigma(self):
        """observation standard deviation in hu/hv units (m^2/s)"""
        return self.obs_sigma_vel * self.H

    def as_dict(self):
        return asdict(self)


def _cfg(name, n, defaults, kw):
    args = dict(defaults)
    args.update(kw)
    return Config(name, n, n, **args)


def config1(**kw):
    return _cfg("iewpf_64x64_ne10_1drifter", 64, {"n_particles": 10, "n_obs": 1}, kw)


def config2(**kw):
    return _cfg("iewpf_512x512_ne100_64drifters", 512, {"n_particles": 100, "n_obs": 64}, kw)


def config4(**kw):
    return _cfg("iewpf_1024x1024_ne1000_1521moorings", 1024,
                {"n_particles": 1000, "obs_kind": OBS_MOORING, "n_obs": 1521}, kw)


def coupled_moorings(**kw):
    """1521 moorings every 16 cells on 624 x 624 cells, 1000 particles: the
    moorings sit closer than the 21-cell radius of the pull stencil, so the
    dense 3042 x 3042 HQH^T + R couples neighbouring moorings and its
    Cholesky factor fills in (the moorings of config4, 26 cells apart, do not
    interact).  Use mooring_cells(cfg, COUPLED_SPACING)."""
    return _cfg("iewpf_624x624_ne1000_1521moorings_every16", 624,
                {"n_particles": 1000, "obs_kind": OBS_MOORING, "n_obs": 1521}, kw)


COUPLED_SPACING = 16


def config5(**kw):
    return _cfg("surrogate_256x256_ne1000_64drifters", 256, {"n_particles": 1000, "n_obs": 64}, kw)


def config3(seed: int = 3, **kw):
    """32 independent problems with grids from {128,256,512,1024}^2,
    20-500 particles and 4-128 drifters (drawn with a seeded generator)."""
    rng = np.random.Generator(np.random.Philox(seed))
    out = []
    sizes = [128, 256, 512, 1024]
    for i in range(32):
        n = int(sizes[rng.integers(0, 4)])
        ne = int(rng.integers(20, 501))
        nd = int(rng.integers(4, 129))
        out.append(Config("batch%02d_%dx%d_ne%d_%ddrifters" % (i, n, n, ne, nd), n, n,
                          n_particles=ne, n_obs=nd, seed=0x1910_01031 + i, **kw))
    return out


def config_rank(**kw):
    """The rank-histogram setup of Sec. 5.1 with the domain of Sec. 5: 500 x
    300 cells of 2220 m, g = 9.806, f = 1.405e-4 1/s, Courant number 0.8,
    q0 = 2.5e-4 m, c_omega = 5, L0 = 3/4 coarse cell; 40 particles, the
    120 moorings of the western half."""
    base = dict(dx=2220.0, dy=2220.0, g=9.806, f=1.405e-4, courant=0.8, q0=2.5e-4, c_omega=5,
                n_particles=40, obs_kind=OBS_MOORING, n_obs=120)
    base.update(kw)
    return Config("rank_500x300", 500, 300, **base)


def rank_moorings(cfg: Config):
    """The western half of a 20 x 12 mooring lattice (240 moorings, Sec. 5):
    10 x 12 = 120 cells, every nx/20 cells in x and ny/12 in y."""
    sx, sy = cfg.nx // 20, cfg.ny // 12
    return np.array([(sx // 2 + sx * p, sy // 2 + sy * q) for q in range(12) for p in range(10)], dtype=np.int32)


def rank_cells(cfg: Config):
    """Cells (100, y), y = 0, 50, ..., 250 (scaled to the grid), where the
    ranks are taken (Sec. 5.1)."""
    x = min(100, cfg.nx - 1)
    return np.array([(x, y) for y in range(0, cfg.ny - 49, 50)], dtype=np.int32)


def _jet(cfg: Config):
    Ly = cfg.ny * cfg.dy
    w = cfg.jet_width_cells * cfg.dy
    y = (np.arange(cfg.ny) + 0.5) * cfg.dy
    a1, a2 = (y - Ly / 4) / w, (y - 3 * Ly / 4) / w
    eta_y = 0.5 * cfg.jet_amp * (np.tanh(a1) - np.tanh(a2))
    eta_y -= eta_y.mean()
    deta_dy = 0.5 * cfg.jet_amp / w * (1.0 / np.cosh(a1) ** 2 - 1.0 / np.cosh(a2) ** 2)
    hu_y = -(cfg.g * cfg.H / cfg.f) * deta_dy
    return eta_y, hu_y


def initial_particle(cfg: Config, i: int, seed: int = 7, dtype=np.float64):
    """Particle i of the initial ensemble: [3][ny][nx] (see initial_state);
    its noise comes from its own generator, so any subset of a large
    ensemble can be produced on its own."""
    eta_y, hu_y = _jet(cfg)
    rng = np.random.Generator(np.random.Philox(key=seed, counter=[0, 0, 0, i]))
    U = np.zeros((3, cfg.ny, cfg.nx), dtype=np.float64)
    U[0] = eta_y[:, None]
    U[1] = hu_y[:, None]
    U[0] += cfg.noise_std * rng.standard_normal((cfg.ny, cfg.nx))
    return U.astype(dtype)


def initial_state(cfg: Config, ne: int, seed: int = 7, dtype=np.float64):
    """Two opposite zonal jets: eta(y) = A/2 [tanh((y - Ly/4)/w) -
    tanh((y - 3Ly/4)/w)] minus its mean, with (hu, hv) from the continuous
    geostrophic balance hu = -(g H / f) d eta/dy evaluated analytically, and
    i.i.d. N(0, noise_std^2) added to eta of every particle (numpy's Philox
    bit generator, one counter per particle).  Returns [ne][3][ny][nx]."""
    return np.stack([initial_particle(cfg, i, seed, dtype) for i in range(ne)])


def drifter_positions(cfg: Config, n: int | None = None):
    """Drifter start positions (metres): a centred k x k lattice (8 x 8 for
    64 drifters, Sec. 5.2); a single drifter sits at the centre cell."""
    n = cfg.n_obs if n is None else n
    Lx, Ly = cfg.nx * cfg.dx, cfg.ny * cfg.dy
    if n == 1:
        return np.array([[0.5 * Lx + 0.3 * cfg.dx, 0.5 * Ly + 0.6 * cfg.dy]])
    k = int(math.ceil(math.sqrt(n)))
    pts = []
    for q in range(k):
        for p in range(k):
            if len(pts) < n:
                pts.append([(p + 0.5) * Lx / k + 0.3 * cfg.dx, (q + 0.5) * Ly / k + 0.6 * cfg.dy])
    return np.array(pts, dtype=np.float64)


def mooring_cells(cfg: Config, spacing: int = 26):
    """Equidistant moorings every `spacing` cells (39 x 39 = 1521 on 1024^2)."""
    m = int(math.isqrt(cfg.n_obs))
    off = (cfg.nx - spacing * (m - 1)) // 2
    cells = [(off + spacing * p, off + spacing * q) for q in range(m) for p in range(m)]
    return np.array(cells, dtype=np.int32)


def cell_positions(cfg: Config, cells):
    """Cell-centre coordinates (metres) of integer cells."""
    cells = np.asarray(cells, dtype=np.float64)
    return np.stack([(cells[:, 0] + 0.5) * cfg.dx, (cells[:, 1] + 0.5) * cfg.dy], axis=1)


def obs_noise(cfg: Config, n_obs: int, cycle: int, seed: int = 11):
    """Observation errors epsilon ~ N(0, obs_sigma^2 I), one draw per cycle."""
    rng = np.random.Generator(np.random.Philox(seed + 1000003 * cycle))
    return cfg.obs_sigma * rng.standard_normal((n_obs, 2))


def obs_from_state(cfg: Config, U, cells, noise):
    """Synthetic mooring-type observations read from a state [3][ny][nx]:
    (hu, hv) scaled by H/(H + eta) at the cells, plus the given noise
    (eq. buoyObservation)."""
    U = np.asarray(U, dtype=np.float64)
    cells = np.asarray(cells)
    eta = U[0][cells[:, 1], cells[:, 0]]
    s = cfg.H / (cfg.H + eta)
    return np.stack([U[1][cells[:, 1], cells[:, 0]] * s, U[2][cells[:, 1], cells[:, 0]] * s],
                    axis=1) + noise


def observation_subsets(n_obs: int, size: int, n_subsets: int, seed: int = 13):
    """n_subsets random subsets of `size` distinct observation indices out of
    n_obs ([n_subsets][size] int32), as drawn for the collapse experiment of
    the standard particle filter (Sec. 5.3: 50 subsets per size)."""
    rng = np.random.Generator(np.random.Philox(seed + 7919 * size))
    return np.stack([np.sort(rng.choice(n_obs, size, replace=False)) for _ in range(n_subsets)]).astype(np.int32)


CONFIG_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "configs")


def workloads():
    """The named workloads of this library: name -> Config or list of Config."""
    return {"plain_64x64": config1(), "plain_512x512": config2(), "batched_32": config3(),
            "moorings_1024x1024": config4(), "surrogate_256x256": config5(), "rank_500x300": config_rank()}


def config_to_json(cfg):
    """A Config (or a list of them) as JSON text."""
    obj = [c.as_dict() for c in cfg] if isinstance(cfg, list) else cfg.as_dict()
    return json.dumps(obj, indent=1, sort_keys=True) + "\n"


def load_config(path_or_name):
    """A Config (or a list of them, for batched workloads) from a JSON file,
    or from the name of one of configs/*.json."""
    path = path_or_name
    if not os.path.exists(path):
        path = os.path.join(CONFIG_DIR, path_or_name + ".json")
    with open(path) as f:
        obj = json.load(f)
    return [Config(**o) for o in obj] if isinstance(obj, list) else Config(**obj)


def write_configs(directory=CONFIG_DIR):
    """Writes configs/<workload>.json for every named workload."""
    os.makedirs(directory, exist_ok=True)
    for name, cfg in workloads().items():
        with open(os.path.join(directory, name + ".json"), "w") as f:
            f.write(config_to_json(cfg))
