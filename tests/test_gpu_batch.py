"""Batched problems (one persistent launch per phase, the whole cycle as a
CUDA graph with a conditional while-node for the CFL-chosen scheme steps)
against the same problems run one by one through the C ABI: the results
must be identical, including after a graph replay."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_01031_gb300 import iewpf, synth

from gpu_common import oracle_problem, rel_l2

pytestmark = pytest.mark.gpu


def _problems():
    cfgs = [
        synth.config1(n_particles=4),
        synth.Config("ragged_72x50", 72, 50, n_particles=3, n_obs=3),
        synth.Config("grid_96x64_block", 96, 64, n_particles=5, n_obs=2, dense_S=0),
        synth.Config("moor_72x50", 72, 50, n_particles=2, n_obs=4, obs_kind=synth.OBS_MOORING),
    ]
    moor = [None, None, None, synth.cell_positions(cfgs[3], np.array([[5, 7], [36, 9], [60, 30], [20, 44]]))]
    params = []
    for i, c in enumerate(cfgs):
        p = iewpf.params_from_config(c)
        p.instance_id = i
        params.append(p)
    params[2].scheme = iewpf.ONE_STAGE       # one problem runs the one-stage IEWPF
    return cfgs, params, moor


def _obs(cfg, cycle):
    if cfg.obs_kind == synth.OBS_MOORING:
        cells = np.array([[5, 7], [36, 9], [60, 30], [20, 44]])
        xy = None
    else:
        xy = synth.drifter_positions(cfg) + 1500.0 * cycle
        P = oracle_problem(cfg)
        cells = np.array([O.obs_cell(P, *p) for p in xy])
    truth = synth.initial_particle(cfg, 77, seed=5)
    return xy, synth.obs_from_state(cfg, truth, cells, synth.obs_noise(cfg, len(cells), cycle))


def test_batched_cycles_equal_one_by_one():
    cfgs, params, moor = _problems()
    batch = iewpf.Batch(params, moor)
    singles = [iewpf.Ensemble(p, mooring_xy=m) for p, m in zip(params, moor)]
    for i, c in enumerate(cfgs):
        U = synth.initial_state(c, c.n_particles, seed=20 + i).astype(np.float32)
        batch.instances[i].set_state(U)
        singles[i].set_state(U)
    for cycle in range(2):           # the second cycle replays the captured graph
        obs = [_obs(c, cycle) for c in cfgs]
        diag = batch.cycle(5, obs)
        for i, s in enumerate(singles):
            s.forecast(4, True)
            s.forecast(1, False)
            d = s.assimilate(obs[i][0], obs[i][1])
            assert diag[i, 0] == d["w_target"] and diag[i, 1] == d["beta"], (cycle, i)
            if i == 2:
                assert d["beta"] == 0.0 and d["w_target"] == d["c"].max()
            assert diag[i, 2] == 0
            a, b = batch.instances[i].get_state(), s.get_state()
            assert np.array_equal(a, b), (cycle, i, np.abs(a - b).max())
            assert batch.instances[i].counters() == s.counters()
    work, launches = batch.work()
    assert work > 0 and launches > 0


def test_batched_forecast_equals_one_by_one():
    cfgs, params, moor = _problems()
    batch = iewpf.Batch(params, moor)
    singles = [iewpf.Ensemble(p, mooring_xy=m) for p, m in zip(params, moor)]
    for i, c in enumerate(cfgs):
        U = synth.initial_state(c, c.n_particles, seed=50 + i).astype(np.float32)
        batch.instances[i].set_state(U)
        singles[i].set_state(U)
    obs = [_obs(c, 0) for c in cfgs]
    batch.cycle(5, obs)
    for i, s in enumerate(singles):
        s.forecast(4, True)
        s.forecast(1, False)
        s.assimilate(obs[i][0], obs[i][1])
    for err, steps in ((True, 7), (True, 7), (False, 3)):     # the second call replays the graph
        batch.forecast(steps, err)
        for i, s in enumerate(singles):
            s.forecast(steps, err)
            a, b = batch.instances[i].get_state(), s.get_state()
            assert np.array_equal(a, b), (err, i, np.abs(a - b).max())
            assert batch.instances[i].counters() == s.counters()


def test_batched_cycle_matches_oracle():
    """Instance 0 draws from the oracle's streams (0, 1, 2)."""
    cfgs, params, moor = _problems()
    c0 = cfgs[0]
    batch = iewpf.Batch([params[0]], None)
    U0 = synth.initial_state(c0, c0.n_particles, seed=4).astype(np.float32)
    batch.instances[0].set_state(U0)
    xy0, y0 = _obs(c0, 0)
    batch.cycle(5, [(xy0, y0)])
    P0 = oracle_problem(c0)
    ref, _, _ = O.forecast(P0, U0.astype(np.float64), 5, [1, 1, 1, 1, 0], t0=0)
    cells = [O.obs_cell(P0, *p) for p in xy0]
    ref, _ = O.assimilate(P0, ref, cells, y0, t=0)
    assert rel_l2(batch.instances[0].get_state(), ref) < 1e-5


def test_batch_rejects_short_observation_sets():
    cfgs, params, moor = _problems()
    batch = iewpf.Batch(params[:1], None)
    with pytest.raises(iewpf.IewpfError):
        batch.cycle(5, [(np.zeros((2, 2)), np.zeros((2, 2)))])


def test_full_size_batched_workload_sampled():
    """The 32-problem batched workload (grids 128^2..1024^2, 20-500
    particles, 4-128 drifters, 73 GB of state) through one CUDA-graph cycle,
    as the bench runs it; the two smallest problems run one by one as well
    and must agree bitwise."""
    torch = pytest.importorskip("torch")
    cfgs = synth.config3()
    params = []
    for i, c in enumerate(cfgs):
        p = iewpf.params_from_config(c)
        p.instance_id = i
        params.append(p)
    batch = iewpf.Batch(params)
    starts = {}
    for i, c in enumerate(cfgs):
        x = synth.initial_particle(c, 0, seed=100 + i, dtype=np.float32)
        U = torch.from_numpy(x).cuda().unsqueeze(0).expand(c.n_particles, -1, -1, -1).contiguous()
        batch.instances[i].set_state(U)
        starts[i] = x
        del U
    obs = []
    for c in cfgs:
        xy = synth.drifter_positions(c)
        cells = np.stack([np.floor(xy[:, 0] / c.dx) % c.nx, np.floor(xy[:, 1] / c.dy) % c.ny], 1).astype(int)
        obs.append((xy, synth.obs_from_state(c, synth.initial_particle(c, 1, seed=300), cells,
                                             synth.obs_noise(c, len(cells), 0))))
    diag = batch.cycle(5, obs)
    assert np.all(diag[:, 2] == 0)
    small = sorted(range(len(cfgs)), key=lambda i: cfgs[i].n_particles * cfgs[i].nx * cfgs[i].ny)[:2]
    for i in small:
        c = cfgs[i]
        s = iewpf.Ensemble(params[i])
        s.set_state(np.broadcast_to(starts[i], (c.n_particles,) + starts[i].shape).copy())
        s.forecast(4, True)
        s.forecast(1, False)
        d = s.assimilate(*obs[i])
        assert diag[i, 0] == d["w_target"] and diag[i, 1] == d["beta"], i
        assert np.array_equal(batch.instances[i].get_state(), s.get_state()), i
        s.close()
    batch.close()
