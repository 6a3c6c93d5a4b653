"""GPU parity of the standard particle filter weights (Sec. 2.1) and the
count of sure survivors of residual resampling (Sec. 5.3) against the FP64
oracle, through the C ABI.  Weights 1e-9 relative (FP64 on both sides; the
innovations differ by one rounding of a fused multiply-add); the counts
exactly, except for subsets where an oracle weight lies within 1e-9 of
1/N_e, where either answer is correct."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_01031_gb300 import iewpf, synth

from gpu_common import ensemble, oracle_problem, ragged_config

pytestmark = pytest.mark.gpu


def _compare(wg, kg, wo, ko, ne):
    assert np.allclose(wg, wo, rtol=1e-9, atol=1e-300)
    assert np.allclose(wg.sum(axis=1), 1.0, rtol=1e-12)
    for s in range(len(ko)):
        if np.any(np.abs(wo[s] * ne - 1.0) < 1e-9):
            continue
        assert kg[s] == ko[s], s


@pytest.mark.parametrize("r_scale", [1.0, 10.0])
def test_sir_weights_match_oracle_drifters(r_scale):
    cfg = synth.config1(n_particles=20, n_obs=16)
    P = oracle_problem(cfg)
    ens = ensemble(cfg)
    ens.set_state(synth.initial_state(cfg, cfg.n_particles, seed=3).astype(np.float32))
    ens.forecast(5, True)                       # spread the ensemble
    U = ens.get_state()
    xy = synth.drifter_positions(cfg)
    cells = np.array([O.obs_cell(P, *p) for p in xy])
    truth = synth.initial_particle(cfg, 40, seed=9)
    y = synth.obs_from_state(cfg, truth, cells, synth.obs_noise(cfg, len(cells), 0))
    for k in (1, 4, 16):
        sets = synth.observation_subsets(16, k, 6)
        wg, kg = ens.sir_weights(xy, y, sets, r_scale)
        d = O.innovations(P, U.astype(np.float64), cells, y)
        wo, ko = O.sir_weights(d, sets, cfg.obs_sigma ** 2, r_scale)
        _compare(wg, kg, wo, ko, cfg.n_particles)
    # the state is not touched
    assert np.array_equal(ens.get_state(), U)


def test_sir_weights_match_oracle_moorings_ragged_and_repeated_indices():
    cfg = ragged_config(obs_kind=synth.OBS_MOORING, n_obs=4, n_particles=7)
    cells = np.array([[5, 7], [36, 9], [60, 30], [20, 44]], dtype=np.int32)
    ens = ensemble(cfg, mooring_xy=synth.cell_positions(cfg, cells))
    ens.set_state(synth.initial_state(cfg, cfg.n_particles, seed=6).astype(np.float32))
    ens.forecast(3, True)
    U = ens.get_state()
    y = synth.obs_from_state(cfg, synth.initial_particle(cfg, 30, seed=2), cells, synth.obs_noise(cfg, 4, 1))
    sets = np.array([[0, 1, 2, 3], [3, 3, 3, 3], [2, 0, 2, 1]], dtype=np.int32)
    wg, kg = ens.sir_weights(None, y, sets)
    P = oracle_problem(cfg)
    wo, ko = O.sir_weights(O.innovations(P, U.astype(np.float64), cells, y), sets, cfg.obs_sigma ** 2)
    _compare(wg, kg, wo, ko, cfg.n_particles)


def test_sir_weights_reject_bad_subsets():
    cfg = synth.config1(n_particles=4, n_obs=3)
    ens = ensemble(cfg)
    ens.set_state(synth.initial_state(cfg, 4).astype(np.float32))
    xy = synth.drifter_positions(cfg)
    y = np.zeros((3, 2))
    for sets, r in ((np.array([[0, 3]]), 1.0), (np.array([[-1]]), 1.0), (np.zeros((1, 0)), 1.0),
                    (np.array([[0, 1, 2, 0]]), 1.0), (np.array([[0]]), 0.0)):
        with pytest.raises(iewpf.IewpfError) as e:
            ens.sir_weights(xy, y, sets, r)
        assert e.value.name == "EINVAL"
    # the context stays usable
    w, k = ens.sir_weights(xy, y, np.array([[0, 1, 2]]))
    assert w.shape == (1, 4) and np.isclose(w.sum(), 1.0)


def test_collapse_experiment_full_size_sampled():
    """Sec. 5.3 on the 512 x 512, 100-particle, 64-drifter workload: every
    size 1..64 with 50 subsets and R, 10 R in one call each; the oracle checks
    three sizes at both scales on 5 subsets each."""
    cfg = synth.config2()
    P = oracle_problem(cfg)
    ens = ensemble(cfg)
    ens.set_state(synth.initial_state(cfg, cfg.n_particles, seed=12).astype(np.float32))
    ens.forecast(1, True)
    U = ens.get_state()
    xy = synth.drifter_positions(cfg)
    cells = np.array([O.obs_cell(P, *p) for p in xy])
    y = synth.obs_from_state(cfg, synth.initial_particle(cfg, 500, seed=12), cells, synth.obs_noise(cfg, 64, 0))
    d = O.innovations(P, U.astype(np.float64), cells, y)
    for r_scale in (1.0, 10.0):
        means = []
        for k in range(1, 65):
            sets = synth.observation_subsets(64, k, 50)
            wg, kg = ens.sir_weights(xy, y, sets, r_scale)
            means.append(kg.mean())
            if k in (1, 8, 64):
                wo, ko = O.sir_weights(d, sets[:5], cfg.obs_sigma ** 2, r_scale)
                _compare(wg[:5], kg[:5], wo, ko, cfg.n_particles)
        assert all(1 <= m <= cfg.n_particles for m in means)
