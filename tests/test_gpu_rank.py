"""GPU parity of the ranks of observed values within the ensemble (Sec.
5.1) against the oracle, through the C ABI, and a small run of the
rank-histogram experiment.  Ranks are integers: equal, except where a
perturbed member lies within 1e-9 of the observed value (the two sides
round the perturbation differently; either count is correct there)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_01031_gb300 import iewpf, synth

from gpu_common import ensemble, oracle_problem

pytestmark = pytest.mark.gpu


def test_ranks_match_oracle():
    cfg = synth.config1(n_particles=40, n_obs=1)
    P = oracle_problem(cfg)
    ens = ensemble(cfg)
    ens.set_state(synth.initial_state(cfg, cfg.n_particles, seed=4).astype(np.float32))
    ens.forecast(5, True)
    U = ens.get_state().astype(np.float64)
    rng = np.random.default_rng(0)
    cells = np.stack([rng.integers(0, cfg.nx, 25), rng.integers(0, cfg.ny, 25)], axis=1).astype(np.int32)
    cells[0] = (0, 0)
    cells[1] = (cfg.nx - 1, cfg.ny - 1)
    truth = synth.initial_particle(cfg, 77, seed=1)
    y = synth.obs_from_state(cfg, truth, cells, synth.obs_noise(cfg, len(cells), 3))
    y[2] = (-1e6, 1e6)                                   # below and above every member
    for draw in (0, 9):
        rg = ens.rank(cells, y, draw)
        ro = O.ranks(P, U, cells, y, t=draw)
        eps = np.stack([O.normals(P.seed, i, draw, O.STREAM_RANK, 2 * len(cells)) for i in range(cfg.n_particles)])
        for m, (j, k) in enumerate(cells):
            for c in (0, 1):
                v = U[:, 1 + c, k, j] + P.obs_sigma * eps[:, 2 * m + c]
                if np.min(np.abs(v - y[m, c])) < 1e-9 * max(1.0, abs(y[m, c])):
                    continue
                assert rg[m, c] == ro[m, c], (draw, m, c)
        assert rg[2, 0] == 0 and rg[2, 1] == cfg.n_particles
    # the state is not touched
    assert np.array_equal(ens.get_state(), U.astype(np.float32))


def test_rank_rejects_points_outside_the_grid():
    cfg = synth.config1(n_particles=4)
    ens = ensemble(cfg)
    ens.set_state(synth.initial_state(cfg, 4).astype(np.float32))
    for cell in ((-1, 0), (0, cfg.ny), (cfg.nx, 3)):
        with pytest.raises(iewpf.IewpfError) as e:
            ens.rank(np.array([cell]), np.zeros((1, 2)), 0)
        assert e.value.name == "EINVAL"
    with pytest.raises(iewpf.IewpfError):
        ens.rank(np.array([(1, 1)]), np.array([[np.nan, 0.0]]), 0)


def test_small_rank_histogram_experiment():
    pytest.importorskip("torch")
    from paper_1910_01031_gb300 import rank_histogram
    for scheme in (iewpf.TWO_STAGE, iewpf.ONE_STAGE):
        out = rank_histogram.run(experiments=3, ne=6, hours_da=10 / 60, hours_fc=5 / 60, scheme=scheme,
                                 nx=200, ny=150)
        assert out["cycles"] == 2 and out["forecast_steps"] == 5
        assert sum(out["histogram"]) == 3 * len(out["rank_cells"]) * 2
        assert len(out["histogram"]) == 7 and out["particle_substeps"] > 0
