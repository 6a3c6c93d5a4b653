"""The synthetic inputs (stand-ins for the paper's twin experiments, Sec. 5):
layouts, initial jets, observation errors and subsets, pinned on the CPU to
the properties their recipe states."""
import math

import numpy as np

from paper_1910_01031_gb300 import synth


def _torus_dist(a, b, n):
    d = abs(int(a) - int(b)) % n
    return min(d, n - d)


def test_headline_moorings_are_a_centred_uncoupled_lattice():
    cfg = synth.config4()
    cells = synth.mooring_cells(cfg)
    assert cells.shape == (1521, 2)
    xs, ys = np.unique(cells[:, 0]), np.unique(cells[:, 1])
    assert len(xs) == len(ys) == 39
    assert np.all(np.diff(xs) == 26) and np.all(np.diff(ys) == 26)
    # centred: the margins on both sides differ by at most one cell
    assert abs(int(xs[0]) - (cfg.nx - 1 - int(xs[-1]))) <= 1
    # the pull stencil reaches 7 c_Omega = 21 cells: no two moorings within it
    # (the seam gap 1024 - 26 * 38 = 36 is wider than the spacing)
    reach = 7 * cfg.c_omega
    gap = cfg.nx - (int(xs[-1]) - int(xs[0]))
    assert gap > reach and 26 > reach


def test_coupled_moorings_couple_each_to_its_eight_neighbours():
    cfg = synth.coupled_moorings()
    cells = synth.mooring_cells(cfg, synth.COUPLED_SPACING)
    assert cells.shape == (1521, 2) and cfg.nx == cfg.ny == 624
    reach = 7 * cfg.c_omega
    n = len(cells)
    near = np.zeros(n, int)
    for k in range(n):
        dx = [_torus_dist(cells[k, 0], c, cfg.nx) for c in cells[:, 0]]
        dy = [_torus_dist(cells[k, 1], c, cfg.ny) for c in cells[:, 1]]
        near[k] = sum(1 for l in range(n) if l != k and dx[l] <= reach and dy[l] <= reach)
    # 16 <= 21 < 32: the 3 x 3 neighbourhood on the torus, across the seam too
    assert np.all(near == 8)


def test_rank_layout():
    cfg = synth.config_rank()
    moor = synth.rank_moorings(cfg)
    assert moor.shape == (120, 2)
    assert np.all(moor[:, 0] < cfg.nx // 2) and np.all(moor[:, 1] < cfg.ny)
    assert len(np.unique(moor[:, 0])) == 10 and len(np.unique(moor[:, 1])) == 12
    assert len({tuple(c) for c in moor}) == 120
    cells = synth.rank_cells(cfg)
    assert cells.tolist() == [[100, y] for y in (0, 50, 100, 150, 200, 250)]


def test_drifter_lattice():
    cfg = synth.config2()
    xy = synth.drifter_positions(cfg)
    assert xy.shape == (64, 2)
    Lx, Ly = cfg.nx * cfg.dx, cfg.ny * cfg.dy
    assert np.all((xy[:, 0] > 0) & (xy[:, 0] < Lx) & (xy[:, 1] > 0) & (xy[:, 1] < Ly))
    assert len(np.unique(np.round(xy[:, 0], 6))) == 8 and len(np.unique(np.round(xy[:, 1], 6))) == 8
    one = synth.drifter_positions(cfg, 1)
    assert one.shape == (1, 2)
    assert abs(one[0, 0] - 0.5 * Lx) < cfg.dx and abs(one[0, 1] - 0.5 * Ly) < cfg.dy


def test_jets_are_geostrophic_and_opposite():
    cfg = synth.config2()
    eta, hu = synth._jet(cfg)
    assert abs(eta.mean()) < 1e-15
    # hu = -(g H / f) d eta / dy: against centred differences, O(dy^2)
    d = (np.roll(eta, -1) - np.roll(eta, 1)) / (2 * cfg.dy)
    inner = slice(2, cfg.ny - 2)
    ref = -(cfg.g * cfg.H / cfg.f) * d
    assert np.max(np.abs(hu[inner] - ref[inner])) < 1e-2 * np.max(np.abs(hu))
    # two jets of opposite direction at y = Ly / 4 and 3 Ly / 4
    q1, q3 = cfg.ny // 4, 3 * cfg.ny // 4
    assert hu[q1] * hu[q3] < 0 and abs(abs(hu[q1]) - abs(hu[q3])) < 1e-3 * abs(hu[q1])


def test_particles_are_reproducible_one_by_one():
    cfg = synth.config1()
    U = synth.initial_state(cfg, 4, seed=5)
    for i in (0, 3):
        assert np.array_equal(U[i], synth.initial_particle(cfg, i, seed=5))
    eta, _ = synth._jet(cfg)
    noise = U[:, 0] - eta[None, :, None]
    assert abs(noise.std() - cfg.noise_std) < 0.05 * cfg.noise_std
    assert np.all(U[:, 2] == 0.0)
    assert not np.array_equal(U[0], U[1])


def test_observation_errors_and_observations():
    cfg = synth.config4()
    e0 = synth.obs_noise(cfg, 1521, 0)
    e1 = synth.obs_noise(cfg, 1521, 1)
    assert e0.shape == (1521, 2)
    assert abs(e0.std() - cfg.obs_sigma) < 0.05 * cfg.obs_sigma
    assert not np.array_equal(e0, e1)
    assert np.array_equal(e0, synth.obs_noise(cfg, 1521, 0))
    # eq. buoyObservation on a hand-made state
    small = synth.config1()
    U = np.zeros((3, small.ny, small.nx))
    U[0, 3, 2], U[1, 3, 2], U[2, 3, 2] = small.H, 4.0, -2.0     # (x, y) = (2, 3)
    y = synth.obs_from_state(small, U, np.array([[2, 3], [0, 0]]), np.zeros((2, 2)))
    np.testing.assert_allclose(y, [[2.0, -1.0], [0.0, 0.0]], rtol=0, atol=1e-14)


def test_observation_subsets():
    s = synth.observation_subsets(64, 10, 50)
    assert s.shape == (50, 10) and s.dtype == np.int32
    for row in s:
        assert np.all(np.diff(row) > 0) and row[0] >= 0 and row[-1] < 64
    assert not np.array_equal(s, synth.observation_subsets(64, 10, 50, seed=14))
    assert math.comb(64, 10) > 50
