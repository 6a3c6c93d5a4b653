"""GPU parity of the IEWPF analysis against the FP64 oracle, through the C
ABI.  Tolerances: FP64 weights 1e-10 relative on shared inputs; gamma and
zeta (no state dependence) 1e-10; state after the analysis 1e-5 relative L2
(FP32 state); phi and c 1e-4 relative (they inherit the FP32 state's
rounding through innovations of a few m^2/s)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_01031_gb300 import iewpf, synth

from gpu_common import ensemble, oracle_problem, ragged_config, rel_l2, start_state

pytestmark = pytest.mark.gpu


def test_pull_stencil_and_block_root_match_oracle():
    for cfg in (synth.config1(), ragged_config(dy=2500.0)):
        ens = ensemble(cfg)
        P = oracle_problem(cfg)
        K = O.pull_stencil(P)
        Kg = ens.pull_stencil()
        assert Kg.shape == K.shape
        assert np.max(np.abs(Kg - K)) <= 1e-12 * np.max(np.abs(K))
        M = O.local_block_sqrt(P)
        assert np.max(np.abs(ens.local_block() - M)) <= 1e-10


def _scalars_inputs(seed, ne, N, Ny):
    rng = np.random.default_rng(seed)
    c = rng.chisquare(Ny, ne) + math.log(ne)
    gamma = N + math.sqrt(2 * N) * rng.standard_normal(ne)
    zeta = N + math.sqrt(2 * N) * rng.standard_normal(ne)
    return c, gamma, zeta


@pytest.mark.parametrize("ne,N,Ny", [(10, 12288, 2), (100, 786432, 128), (1000, 3145728, 3042), (3, 60.0, 2)])
def test_weights_stage_matches_oracle_to_1e10(ne, N, Ny):
    c, gamma, zeta = _scalars_inputs(ne + Ny, ne, N, Ny)
    if N < 100:        # tiny state: gamma far from N, alpha far from 1
        gamma = np.array([40.0, 75.0, 61.0])
        zeta = np.array([55.0, 70.0, 64.0])
        c = np.array([3.0, 4.5, 3.7])
    g = iewpf.weights(c, gamma, zeta, N)
    o = O.iewpf_scalars(c, gamma, zeta, N)
    assert math.isclose(g["cbar"], o["cbar"], rel_tol=1e-12)
    assert math.isclose(g["beta"], o["beta"], rel_tol=1e-10)
    assert np.allclose(g["alpha"], o["alpha"], rtol=1e-10, atol=0)
    assert np.allclose(g["neglogw"], o["neglogw"], rtol=1e-10, atol=0)
    # every particle reaches the target weight on the GPU as well
    assert np.allclose(g["neglogw"], g["cbar"], rtol=1e-10, atol=0)


@pytest.mark.parametrize("ne,N,Ny", [(10, 12288, 2), (100, 786432, 128), (1000, 3145728, 3042), (5, 50.0, 2)])
def test_one_stage_weights_match_oracle_to_1e10(ne, N, Ny):
    c, gamma, _ = _scalars_inputs(ne + Ny + 1, ne, N, Ny)
    if N < 100:        # tiny state: the Lambert-W argument away from -1/e
        gamma = np.array([20.0, 35.0, 49.0, 60.0, 80.0])
        c = np.array([4.0, 9.5, 1.0, 6.0, 2.5])
    g = iewpf.weights_one_stage(c, gamma, N)
    o = O.iewpf_scalars_one_stage(c, gamma, N)
    assert g["w_target"] == o["w_target"] == c.max()
    assert g["beta"] == 0.0
    assert np.array_equal(g["cstar"], o["cstar"])
    assert np.allclose(g["alpha"], o["alpha"], rtol=1e-10, atol=0)
    assert np.allclose(g["neglogw"], o["neglogw"], rtol=1e-10, atol=0)
    assert np.allclose(g["neglogw"], g["w_target"], rtol=1e-10, atol=0)


@pytest.mark.parametrize("N", [2.0, 4.0, 60.0, 1e4, 786432.0, 3145728.0])
def test_incomplete_gamma_alpha_matches_oracle(N):
    rng = np.random.default_rng(int(N) % 1000)
    ne = 24
    gamma = np.abs(N + math.sqrt(2 * N) * rng.standard_normal(ne)) + 0.05
    cstar = np.concatenate([[0.0, 1e-6, 0.5, 300.0], rng.uniform(0.0, 60.0, ne - 4)])
    g = iewpf.alpha_gamma(gamma, cstar, N)
    o = O.alpha_incomplete_gamma(gamma, cstar, N)
    assert g[0] == 1.0
    assert np.all(g > 0.0) and np.all(g <= 1.0)
    assert np.allclose(g, o, rtol=1e-9, atol=0)


def test_incomplete_gamma_alpha_rejects_bad_arguments():
    for gamma, cstar in (([1.0], [-0.1]), ([0.0], [1.0]), ([float("nan")], [1.0])):
        with pytest.raises(iewpf.IewpfError) as e:
            iewpf.alpha_gamma(gamma, cstar, 10.0)
        assert e.value.name == "EINVAL"


def test_weights_stage_reports_negative_beta():
    # c_bar - c_i very negative against zeta: beta < 0
    with pytest.raises(iewpf.IewpfError) as e:
        iewpf.weights(np.array([0.0, 1000.0, 0.0]), np.array([50.0, 50, 50]), np.array([50.0, 50, 50]), 60.0)
    assert e.value.name == "EBETA"


def _obs_for(cfg, U, cells, cycle=0):
    noise = synth.obs_noise(cfg, len(cells), cycle)
    return synth.obs_from_state(cfg, U, cells, noise)


@pytest.mark.parametrize("dense", [1, 0])
def test_assimilate_matches_oracle_drifters(dense):
    cfg = synth.config1(dense_S=dense, n_obs=3)
    ne = cfg.n_particles
    U32, U64 = start_state(cfg, ne)
    P = oracle_problem(cfg)
    ens = ensemble(cfg)
    ens.set_state(U32)
    xy = np.array([[20.3e3, 30.1e3], [26.9e3, 34.5e3], [90.2e3, 100.7e3]])   # two close, one far
    cells = [O.obs_cell(P, *p) for p in xy]
    truth = synth.initial_state(cfg, 1, seed=99)[0]
    y = _obs_for(cfg, truth, np.array(cells))
    dg = ens.assimilate(xy, y)
    ref, do = O.assimilate(P, U64, cells, y, t=0, dense=bool(dense))
    assert np.allclose(dg["gamma"], do["gamma"], rtol=1e-10, atol=0)
    assert np.allclose(dg["zeta"], do["zeta"], rtol=1e-10, atol=0)
    assert np.allclose(dg["phi"], do["phi"], rtol=1e-4, atol=0)
    assert np.allclose(dg["c"], do["c"], rtol=1e-4, atol=0)
    assert math.isclose(dg["beta"], do["beta"], rel_tol=1e-6)
    assert np.allclose(dg["alpha"], do["alpha"], rtol=1e-6, atol=0)
    assert np.allclose(dg["neglogw"], dg["cbar"], rtol=1e-10, atol=0)
    e = rel_l2(ens.get_state(), ref)
    assert e < 1e-5, e
    assert ens.counters() == (0, 1)


def test_one_stage_assimilate_matches_oracle():
    cfg = ragged_config(n_obs=3, n_particles=6)
    ne = cfg.n_particles
    U32, U64 = start_state(cfg, ne, seed=8)
    P = oracle_problem(cfg)
    ens = iewpf.Ensemble(iewpf.params_from_config(cfg, scheme=iewpf.ONE_STAGE))
    ens.set_state(U32)
    xy = np.array([[20.3e3, 30.1e3], [26.9e3, 34.5e3], [90.2e3, 60.7e3]])
    cells = [O.obs_cell(P, *p) for p in xy]
    truth = synth.initial_state(cfg, 1, seed=99)[0]
    ref = U64
    for cycle in range(2):
        y = _obs_for(cfg, truth, np.array(cells), cycle)
        dg = ens.assimilate(xy, y)
        ref, do = O.assimilate(P, ref, cells, y, t=cycle, one_stage=True)
        assert dg["beta"] == 0.0
        assert dg["w_target"] == dg["c"].max()
        assert math.isclose(dg["cbar"], np.mean(dg["c"]), rel_tol=1e-12)
        assert np.allclose(dg["c"], do["c"], rtol=1e-4, atol=0)
        assert np.allclose(dg["alpha"], do["alpha"], rtol=1e-6, atol=0)
        assert np.allclose(dg["neglogw"], dg["w_target"], rtol=1e-10, atol=0)
        e = rel_l2(ens.get_state(), ref)
        assert e < 1e-5, (cycle, e)


def test_assimilate_matches_oracle_moorings_ragged():
    cfg = ragged_config(obs_kind=synth.OBS_MOORING, n_obs=4)
    ne = cfg.n_particles
    cells = np.array([[5, 7], [36, 9], [60, 30], [20, 44]], dtype=np.int32)
    xy = synth.cell_positions(cfg, cells)
    U32, U64 = start_state(cfg, ne)
    P = oracle_problem(cfg)
    ens = ensemble(cfg, mooring_xy=xy)
    ens.set_state(U32)
    truth = synth.initial_state(cfg, 1, seed=5)[0]
    ref = U64
    for cycle in range(2):
        y = _obs_for(cfg, truth, cells, cycle)
        dg = ens.assimilate(None, y)
        ref, do = O.assimilate(P, ref, [tuple(c) for c in cells], y, t=cycle, dense=True)
        assert np.allclose(dg["gamma"], do["gamma"], rtol=1e-10, atol=0)
        assert np.allclose(dg["phi"], do["phi"], rtol=1e-4, atol=0)
        e = rel_l2(ens.get_state(), ref)
        assert e < 1e-5, (cycle, e)


def test_full_cycle_matches_oracle():
    """Forecast 5 model steps (model error on the first 4) then assimilate,
    twice, on the 64 x 64 ten-particle one-drifter problem."""
    cfg = synth.config1()
    ne = cfg.n_particles
    U32, U64 = start_state(cfg, ne)
    P = oracle_problem(cfg)
    ens = ensemble(cfg)
    ens.set_state(U32)
    ref = U64
    truth = synth.initial_state(cfg, 1, seed=3)[0]
    xy = synth.drifter_positions(cfg)
    cells = [O.obs_cell(P, *p) for p in xy]
    step = 0
    for cycle in range(2):
        ens.forecast(4, True)
        ens.forecast(1, False)
        ref, _, _ = O.forecast(P, ref, 5, [1, 1, 1, 1, 0], t0=step)
        step += 5
        y = _obs_for(cfg, truth, np.array(cells), cycle)
        ens.assimilate(xy, y)
        ref, _ = O.assimilate(P, ref, cells, y, t=cycle)
        e = rel_l2(ens.get_state(), ref)
        assert e < 1e-5, (cycle, e)


def test_fifty_model_steps_match_oracle_every_step():
    """Ten assimilation cycles, 50 model steps, on the 64 x 64 ten-particle
    one-drifter problem: model error after the first four model steps of a
    cycle, none on the fifth, then the analysis (Sec. 4).  The state is
    compared with the oracle after every model step and every analysis at the
    1e-5 relative bound; each particle's scheme-step count is the oracle's."""
    cfg = synth.config1()
    ne = cfg.n_particles
    U32, U64 = start_state(cfg, ne)
    P = oracle_problem(cfg)
    ens = ensemble(cfg)
    ens.set_state(U32)
    ref = U64
    truth = synth.initial_state(cfg, 1, seed=3)[0]
    xy = synth.drifter_positions(cfg)
    cells = [O.obs_cell(P, *p) for p in xy]
    step = 0
    worst = 0.0
    for cycle in range(10):
        for k in range(cfg.obs_every_steps):
            err = k < cfg.obs_every_steps - 1
            ens.forecast(1, err)
            ref, ns, _ = O.forecast(P, ref, 1, [int(err)], t0=step)
            assert np.array_equal(ens.last_nsub(), ns[:, 0]), (cycle, k)
            step += 1
            e = rel_l2(ens.get_state(), ref)
            worst = max(worst, e)
            assert e < 1e-5, (cycle, k, e)
        y = _obs_for(cfg, truth, np.array(cells), cycle)
        ens.assimilate(xy, y)
        ref, _ = O.assimilate(P, ref, cells, y, t=cycle)
        e = rel_l2(ens.get_state(), ref)
        worst = max(worst, e)
        assert e < 1e-5, (cycle, e)
    assert step == 50


def test_assimilate_rejects_bad_observations():
    cfg = synth.config1()
    ens = ensemble(cfg)
    with pytest.raises(iewpf.IewpfError):
        ens.assimilate(np.zeros((2, 2)), np.zeros((2, 2)))     # more than n_obs_max


def test_cfl_rates_left_by_the_updates_match_a_fresh_pass():
    """The model-error and analysis updates leave the CFL rates of the state
    they wrote; a context that recomputes them from a copy of the same state
    must step identically."""
    cfg = synth.config1(n_particles=4, n_obs=2)
    U32, _ = start_state(cfg, 4)
    xy = synth.drifter_positions(cfg, 2)
    a, b = ensemble(cfg), ensemble(cfg)
    for e in (a, b):
        e.set_state(U32)
        e.forecast(2, True)
    truth = synth.initial_particle(cfg, 9, seed=5)
    cells = np.stack([np.floor(xy[:, 0] / cfg.dx) % cfg.nx, np.floor(xy[:, 1] / cfg.dy) % cfg.ny], 1).astype(int)
    y = synth.obs_from_state(cfg, truth, cells, synth.obs_noise(cfg, 2, 0))
    a.assimilate(xy, y)
    b.assimilate(xy, y)
    # b forgets its rates: a copy of its own state goes back in
    b.set_state(b.get_state())
    b.set_counters(*a.counters())
    a.forecast(3, True)
    b.forecast(3, True)
    assert np.array_equal(a.last_nsub(), b.last_nsub())
    assert np.array_equal(a.get_state(), b.get_state())


def test_corrupted_observations_are_refused_and_leave_the_state():
    cfg = synth.config1(n_particles=4, n_obs=2)
    ens = ensemble(cfg)
    U = synth.initial_state(cfg, 4, seed=2).astype(np.float32)
    ens.set_state(U)
    xy = synth.drifter_positions(cfg)
    y = np.ones((2, 2))
    for bad_xy, bad_y in ((xy, np.array([[1.0, np.nan], [0.0, 0.0]])),
                          (np.array([[np.inf, 3e4], [5e4, 5e4]]), y)):
        with pytest.raises(iewpf.IewpfError) as e:
            ens.assimilate(bad_xy, bad_y)
        assert e.value.name == "EINVAL"
        assert np.array_equal(ens.get_state(), U)
        assert ens.counters() == (0, 0)
    ens.assimilate(xy, y)                      # still usable
    assert ens.counters() == (0, 1)


def test_weights_step_reports_domain_and_nonfinite_inputs():
    c = np.array([3.0, 4.0, 5.0])
    z = np.array([60.0, 60.0, 60.0])
    with pytest.raises(iewpf.IewpfError) as e:       # gamma < 0: Lambert-W argument out of its domain
        iewpf.weights(c, np.array([50.0, -5.0, 55.0]), z, 60.0)
    assert e.value.name == "EDOMAIN"
    with pytest.raises(iewpf.IewpfError) as e:
        iewpf.weights(np.array([3.0, np.nan, 5.0]), np.array([50.0, 52.0, 55.0]), z, 60.0)
    assert e.value.name == "ENONFINITE"
    with pytest.raises(iewpf.IewpfError) as e:
        iewpf.weights_one_stage(c, np.array([50.0, -5.0, 55.0]), 60.0)
    assert e.value.name == "EDOMAIN"


def test_device_allocation_failure_is_reported():
    # about 13 TB of state: cudaMalloc refuses it, create returns ENOMEM
    cfg = synth.Config("huge", 16384, 16384, n_particles=2000)
    with pytest.raises(iewpf.IewpfError) as e:
        iewpf.Ensemble(iewpf.params_from_config(cfg))
    assert e.value.name == "ENOMEM"
    # the device is still usable afterwards
    small = ensemble(synth.config1(n_particles=2))
    small.set_state(synth.initial_state(synth.config1(), 2).astype(np.float32))
    small.forecast(1, True)


@pytest.mark.parametrize("scheme", [iewpf.TWO_STAGE, iewpf.ONE_STAGE])
def test_single_particle_analysis_matches_oracle(scheme):
    # N_e = 1: the target is the particle's own c, beta = 1 (two-stage) or 0
    # (one-stage), c* = 0
    cfg = synth.config1(n_particles=1, n_obs=2)
    P = oracle_problem(cfg)
    U32, U64 = start_state(cfg, 1, seed=3)
    ens = iewpf.Ensemble(iewpf.params_from_config(cfg, scheme=scheme))
    ens.set_state(U32)
    xy = synth.drifter_positions(cfg)
    cells = [O.obs_cell(P, *p) for p in xy]
    y = _obs_for(cfg, synth.initial_state(cfg, 1, seed=99)[0], np.array(cells))
    dg = ens.assimilate(xy, y)
    ref, do = O.assimilate(P, U64, cells, y, t=0, one_stage=scheme == iewpf.ONE_STAGE)
    assert dg["beta"] == (1.0 if scheme == iewpf.TWO_STAGE else 0.0)
    assert dg["w_target"] == dg["c"][0] == dg["cbar"]
    assert math.isclose(dg["alpha"][0], do["alpha"][0], rel_tol=1e-6)
    assert rel_l2(ens.get_state(), ref) < 1e-5


def test_drifter_values_formed_from_two_fixes():
    # value = NULL with the previous fixes: the library forms eq.
    # drifterObservation itself; the analysis equals one given those values
    cfg = synth.config1(n_particles=5, n_obs=2)
    U = synth.initial_state(cfg, 5, seed=6).astype(np.float32)
    xy = synth.drifter_positions(cfg)
    xy_prev = xy - np.array([[120.0, -40.0], [-30.0, 85.0]])
    a, b = ensemble(cfg), ensemble(cfg)
    a.set_state(U)
    b.set_state(U)
    da = a.assimilate(xy, None, xy_prev=xy_prev, dt=300.0)
    db = b.assimilate(xy, iewpf.drifter_obs(iewpf.params_from_config(cfg), xy, xy_prev, 300.0))
    assert np.array_equal(a.get_state(), b.get_state())
    assert np.array_equal(da["phi"], db["phi"])
    with pytest.raises(iewpf.IewpfError) as e:      # neither values nor usable fixes
        a.assimilate(xy, None, xy_prev=xy_prev, dt=0.0)
    assert e.value.name == "EINVAL"


def test_mooring_block_levels_equal_the_in_order_walk_bitwise():
    """A fixed mooring layout applies its overlapping 7 x 7 blocks level by
    level (Sec. 4.6, blocks in observation order); a drifter context with the
    same observation cells and values walks them in order.  Everything else
    of the two analyses is the same arithmetic, so the posterior states and
    diagnostics agree bit for bit."""
    kw = dict(n_particles=16, n_obs=100)
    cm = synth.Config("moorings_192_every16", 192, 192, obs_kind=synth.OBS_MOORING, **kw)
    cd = synth.Config("drifters_192_every16", 192, 192, obs_kind=synth.OBS_DRIFTER, **kw)
    cells = synth.mooring_cells(cm, synth.COUPLED_SPACING)
    xy = synth.cell_positions(cm, cells)
    c = cm.c_omega
    nR = -(-cm.nx // c)
    b0 = [[O.nearest_coarse(cm.nx, nR, c, int(x)), O.nearest_coarse(cm.ny, nR, c, int(y))] for x, y in cells]
    assert iewpf.block_levels(b0, nR, nR).max() >= 1          # the blocks overlap: several levels
    U32, _ = start_state(cm, cm.n_particles)
    truth = synth.initial_particle(cm, 999, seed=5)
    y = synth.obs_from_state(cm, truth, cells, synth.obs_noise(cm, len(cells), 0))
    em, ed = ensemble(cm, mooring_xy=xy), ensemble(cd)
    em.set_state(U32)
    ed.set_state(U32)
    dm = em.assimilate(None, y)
    dd = ed.assimilate(xy, y)
    for k in ("phi", "gamma", "zeta", "alpha", "neglogw"):
        assert np.array_equal(dm[k], dd[k]), k
    assert np.array_equal(em.get_state(), ed.get_state())
