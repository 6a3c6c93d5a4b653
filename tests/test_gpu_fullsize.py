"""Parity at the full sizes of the experiment configurations, in the launch
configuration bench.py uses (autotuned marching stepper), on outputs the
oracle can afford: sampled particles for the state, all particles for the
FP64 weights.

* 512 x 512, 100 particles: one model step with model error, two sampled
  particles against the oracle.
* 512 x 512, 100 particles, 64 drifters: one two-stage and one one-stage
  analysis of the initial ensemble, every particle's FP64 scalars and two
  sampled states.
* 1024 x 1024, 1000 particles, 1521 moorings every 26 cells, and 624 x 624,
  1000 particles, 1521 moorings every 16 cells (coupled through HQH^T): one
  analysis from the initial ensemble.  phi_i of every particle, gamma_i and
  zeta_i, beta and alpha_i from the oracle's own inputs, the fill of the
  factor, and the updated state of two sampled particles."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_01031_gb300 import iewpf, synth

from gpu_common import ensemble, oracle_problem, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _device_ensemble(cfg, ne, keep=(), cells=None, seed=7):
    """The initial ensemble on the GPU, built particle by particle; returns
    the device tensor, the float64 states of the `keep` particles and the
    (eta, hu, hv) values of every particle at `cells`."""
    U = torch.empty((ne, 3, cfg.ny, cfg.nx), dtype=torch.float32, device="cuda")
    kept = {}
    at = None if cells is None else np.zeros((ne, len(cells), 3))
    for i in range(ne):
        x = synth.initial_particle(cfg, i, seed=seed, dtype=np.float32)
        U[i].copy_(torch.from_numpy(x))
        if i in keep:
            kept[i] = x.astype(np.float64)
        if cells is not None:
            at[i] = x[:, cells[:, 1], cells[:, 0]].T.astype(np.float64)
    torch.cuda.synchronize()
    return U, kept, at


def test_config2_forecast_sampled_particles():
    cfg = synth.config2()
    P = oracle_problem(cfg)
    sample = (0, 57)
    U, kept, _ = _device_ensemble(cfg, cfg.n_particles, keep=sample)
    ens = ensemble(cfg)
    ens.set_state(U)
    ens.forecast(1, True)
    nsub = ens.last_nsub()
    out = torch.empty_like(U)
    ens.get_state(out)
    torch.cuda.synchronize()
    for i in sample:
        # particle i draws its model error with its own index
        ref, ns, _ = _forecast_as_particle(P, kept[i], i)
        assert ns[0, 0] == nsub[i]
        assert rel_l2(out[i].cpu().numpy(), ref[0]) < 1e-5


def _forecast_as_particle(P, U, i):
    """One model step of particle i alone (its model error uses stream 0 of
    particle i)."""
    n = O.n_sub(P, U)
    V = U.copy()
    dt = P.dt_model / n
    for _ in range(n):
        V = O.swe_substep(P, V, dt)
    V = O.model_error(P, V, i, 0)
    return V[None], np.array([[n]]), None


def _mooring_analysis_full_size(cfg, cells, sample, coupled):
    ne = cfg.n_particles
    P = oracle_problem(cfg)
    xy = synth.cell_positions(cfg, cells)
    U, kept, at = _device_ensemble(cfg, ne, keep=sample, cells=cells)
    truth = synth.initial_particle(cfg, 123456, seed=99)
    y = synth.obs_from_state(cfg, truth, cells, synth.obs_noise(cfg, len(cells), 0))
    ens = ensemble(cfg, mooring_xy=xy)
    n, nnz = ens.factor_info()
    assert n == 2 * len(cells)
    if coupled:
        assert nnz > 20 * n         # the factor fills in between neighbouring moorings
    else:
        assert nnz == n // 2        # 2 x 2 blocks: the moorings do not interact
    ens.set_state(U)
    dg = ens.assimilate(None, y)
    # the oracle's own innovations, S d and phi for every particle
    s = (cfg.H + at[:, :, 0]) / cfg.H
    d = np.stack([y[None, :, 0] * s - at[:, :, 1], y[None, :, 1] * s - at[:, :, 2]], axis=2).reshape(ne, -1)
    K = O.pull_stencil(P)
    A = O.s_matrix(P, K, [tuple(c) for c in cells], dense=True)
    Sd = O.cholesky_solve(A, d.T).T
    phi = np.einsum("ij,ij->i", d, Sd)
    assert np.allclose(dg["phi"], phi, rtol=1e-9, atol=0)
    c = phi + math.log(ne)
    rv = O.rand_vectors(P, ne, t=0)
    assert np.allclose(dg["gamma"], rv["gamma"], rtol=1e-10, atol=0)
    assert np.allclose(dg["zeta"], rv["zeta"], rtol=1e-10, atol=0)
    sc = O.iewpf_scalars(c, rv["gamma"], rv["zeta"], P.N_psi)
    assert math.isclose(dg["beta"], sc["beta"], rel_tol=1e-9)
    assert np.allclose(dg["alpha"], sc["alpha"], rtol=1e-9, atol=0)
    assert np.allclose(dg["neglogw"], dg["cbar"], rtol=1e-10, atol=0)
    # updated state of the sampled particles
    out = torch.empty_like(U)
    ens.get_state(out)
    torch.cuda.synchronize()
    Msq = O.local_block_sqrt(P)
    for i in sample:
        r = math.sqrt(sc["beta"]) * rv["nu"][i] + math.sqrt(sc["alpha"][i]) * rv["xi"][i]
        for cl in cells:
            idx = O.block_indices(P, cl)
            r[idx] = Msq @ r[idx]
        ref = O.add_pull(P, K, cells, Sd[i].reshape(-1, 2), kept[i])
        ref = O.add_qhalf(P, r, ref)
        assert rel_l2(out[i].cpu().numpy(), ref) < 1e-5


def test_config4_analysis_full_size():
    cfg = synth.config4()
    cells = synth.mooring_cells(cfg)
    assert len(cells) == 1521
    _mooring_analysis_full_size(cfg, cells, (3, 998), coupled=False)


def test_coupled_moorings_analysis_full_size():
    """1521 moorings every 16 cells on 624 x 624, 1000 particles: each
    mooring lies within the 21-cell pull stencil of its neighbours, so the
    3042 x 3042 HQH^T + R couples them and its FP64 Cholesky factor fills in
    (Sec. 4.2, eq. S_extended, with the cross-covariances kept)."""
    cfg = synth.coupled_moorings()
    cells = synth.mooring_cells(cfg, synth.COUPLED_SPACING)
    assert len(cells) == 1521
    _mooring_analysis_full_size(cfg, cells, (1, 999), coupled=True)


def test_largest_ensemble_sampled():
    """65 535 particles, the largest ensemble (N_e spans a grid dimension of
    several launches), on 48 x 48 cells: one model step with model error and
    one analysis against two drifters.  Sampled particles against the oracle
    (forecast; gamma, zeta, phi, alpha; the updated state), the ensemble-wide
    step on all particles."""
    cfg = synth.Config("max_ne_48x48", 48, 48, n_particles=65535, n_obs=2)
    P = oracle_problem(cfg)
    ne = cfg.n_particles
    sample = (0, 32768, 65534)
    eta_y, hu_y = synth._jet(cfg)
    g = torch.Generator(device="cuda").manual_seed(5)
    U = torch.zeros((ne, 3, cfg.ny, cfg.nx), dtype=torch.float32, device="cuda")
    U[:, 0] = torch.as_tensor(eta_y, dtype=torch.float32, device="cuda")[None, :, None]
    U[:, 1] = torch.as_tensor(hu_y, dtype=torch.float32, device="cuda")[None, :, None]
    U[:, 0] += cfg.noise_std * torch.randn((ne, cfg.ny, cfg.nx), generator=g, device="cuda")
    U0 = {i: U[i].double().cpu().numpy() for i in sample}
    ens = ensemble(cfg)
    ens.set_state(U)
    ens.forecast(1, True)
    nsub = ens.last_nsub()
    out = torch.empty_like(U)
    ens.get_state(out)
    torch.cuda.synchronize()
    F = {i: out[i].double().cpu().numpy() for i in sample}
    for i in sample:
        ref, ns, _ = _forecast_as_particle(P, U0[i], i)
        assert ns[0, 0] == nsub[i]
        assert rel_l2(F[i], ref[0]) < 1e-5, i
    xy = synth.drifter_positions(cfg)
    cells = [O.obs_cell(P, *p) for p in xy]
    y = synth.obs_from_state(cfg, synth.initial_particle(cfg, 3, seed=8), np.array(cells), synth.obs_noise(cfg, 2, 0))
    dg = ens.assimilate(xy, y)
    ens.get_state(out)
    torch.cuda.synchronize()
    o = O.iewpf_scalars(dg["c"], dg["gamma"], dg["zeta"], P.N_psi, only=sample)
    assert math.isclose(dg["cbar"], o["cbar"], rel_tol=1e-12)
    assert math.isclose(dg["beta"], o["beta"], rel_tol=1e-10)
    assert np.allclose(dg["neglogw"], dg["cbar"], rtol=1e-10, atol=0)
    for i in sample:
        post, do = O.assimilate(P, F[i][None], cells, y, t=0, p0=i,
                                scalars={"beta": dg["beta"], "alpha": [o["alpha"][i]]})
        assert math.isclose(dg["gamma"][i], do["gamma"][0], rel_tol=1e-10)
        assert math.isclose(dg["zeta"][i], do["zeta"][0], rel_tol=1e-10)
        assert math.isclose(dg["phi"][i], do["phi"][0], rel_tol=1e-4)
        assert math.isclose(dg["alpha"][i], o["alpha"][i], rel_tol=1e-10)
        assert rel_l2(out[i].cpu().numpy(), post[0]) < 1e-5, i


def test_config2_one_stage_analysis_full_size():
    """512 x 512, 100 particles, 64 drifters, the one-stage scheme (App. A):
    one analysis of the initial ensemble.  phi, gamma, zeta and alpha of every
    particle against the oracle's own, w_target = max c, and the updated
    state of two sampled particles."""
    cfg = synth.config2()
    ne = cfg.n_particles
    P = oracle_problem(cfg)
    sample = (0, 77)
    xy = synth.drifter_positions(cfg)
    cells = np.array([O.obs_cell(P, *p) for p in xy])
    U, kept, at = _device_ensemble(cfg, ne, keep=sample, cells=cells)
    truth = synth.initial_particle(cfg, 4242, seed=5)
    y = synth.obs_from_state(cfg, truth, cells, synth.obs_noise(cfg, len(cells), 0))
    ens = iewpf.Ensemble(iewpf.params_from_config(cfg, scheme=iewpf.ONE_STAGE))
    ens.set_state(U)
    dg = ens.assimilate(xy, y)
    s = (cfg.H + at[:, :, 0]) / cfg.H
    d = np.stack([y[None, :, 0] * s - at[:, :, 1], y[None, :, 1] * s - at[:, :, 2]], axis=2).reshape(ne, -1)
    cl = [tuple(c) for c in cells]
    K = O.pull_stencil(P)
    Sd = O.cholesky_solve(O.s_matrix(P, K, cl, dense=True), d.T).T
    phi = np.einsum("ij,ij->i", d, Sd)
    assert np.allclose(dg["phi"], phi, rtol=1e-9, atol=0)
    rv = O.rand_vectors(P, ne, t=0)
    assert np.allclose(dg["gamma"], rv["gamma"], rtol=1e-10, atol=0)
    sc = O.iewpf_scalars_one_stage(phi + math.log(ne), rv["gamma"], P.N_psi)
    assert dg["beta"] == 0.0 and dg["w_target"] == dg["c"].max()
    assert math.isclose(dg["w_target"], sc["w_target"], rel_tol=1e-9)
    assert np.allclose(dg["alpha"], sc["alpha"], rtol=1e-9, atol=0)
    assert np.allclose(dg["neglogw"], dg["w_target"], rtol=1e-10, atol=0)
    out = torch.empty_like(U)
    ens.get_state(out)
    torch.cuda.synchronize()
    Msq = O.local_block_sqrt(P)
    for i in sample:
        post, _ = O.assimilate(P, kept[i][None], cl, y, t=0, K=K, Msq=Msq, p0=i,
                               scalars={"beta": 0.0, "alpha": [sc["alpha"][i]]})
        assert rel_l2(out[i].cpu().numpy(), post[0]) < 1e-5, i


def test_config2_two_stage_analysis_full_size():
    """512 x 512, 100 particles, 64 drifters, the two-stage scheme (Sec. 4):
    one analysis of the initial ensemble.  phi, gamma, zeta, beta and alpha
    of every particle against the oracle's own, every particle at the common
    target weight, and the updated state of two sampled particles."""
    cfg = synth.config2()
    ne = cfg.n_particles
    P = oracle_problem(cfg)
    sample = (5, 96)
    xy = synth.drifter_positions(cfg)
    cells = np.array([O.obs_cell(P, *p) for p in xy])
    U, kept, at = _device_ensemble(cfg, ne, keep=sample, cells=cells)
    truth = synth.initial_particle(cfg, 31337, seed=6)
    y = synth.obs_from_state(cfg, truth, cells, synth.obs_noise(cfg, len(cells), 0))
    ens = ensemble(cfg)
    ens.set_state(U)
    dg = ens.assimilate(xy, y)
    s = (cfg.H + at[:, :, 0]) / cfg.H
    d = np.stack([y[None, :, 0] * s - at[:, :, 1], y[None, :, 1] * s - at[:, :, 2]], axis=2).reshape(ne, -1)
    cl = [tuple(c) for c in cells]
    K = O.pull_stencil(P)
    Sd = O.cholesky_solve(O.s_matrix(P, K, cl, dense=True), d.T).T
    phi = np.einsum("ij,ij->i", d, Sd)
    assert np.allclose(dg["phi"], phi, rtol=1e-9, atol=0)
    rv = O.rand_vectors(P, ne, t=0)
    assert np.allclose(dg["gamma"], rv["gamma"], rtol=1e-10, atol=0)
    assert np.allclose(dg["zeta"], rv["zeta"], rtol=1e-10, atol=0)
    sc = O.iewpf_scalars(phi + math.log(ne), rv["gamma"], rv["zeta"], P.N_psi)
    assert math.isclose(dg["cbar"], sc["cbar"], rel_tol=1e-9)
    assert math.isclose(dg["beta"], sc["beta"], rel_tol=1e-9)
    assert np.allclose(dg["alpha"], sc["alpha"], rtol=1e-9, atol=0)
    assert np.allclose(dg["neglogw"], dg["cbar"], rtol=1e-10, atol=0)
    out = torch.empty_like(U)
    ens.get_state(out)
    torch.cuda.synchronize()
    Msq = O.local_block_sqrt(P)
    for i in sample:
        post, _ = O.assimilate(P, kept[i][None], cl, y, t=0, K=K, Msq=Msq, p0=i,
                               scalars={"beta": sc["beta"], "alpha": [sc["alpha"][i]]})
        assert rel_l2(out[i].cpu().numpy(), post[0]) < 1e-5, i
