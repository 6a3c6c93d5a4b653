"""Pins of the oracle's one-stage IEWPF (App. A: eqs. iewpf_targetWeight,
iewpfCStar, iewpfAlphaSol, iewpfUpdateAgain): the target is the largest c_i,
the particle that sets it keeps alpha = 1, alpha equals the explicit Lambert-W
formula evaluated by scipy, every particle reaches the target, the target
moves away from the mean as N_e grows (the weakness App. A names), and for one
particle the two schemes differ by exactly the P^{1/2} nu term."""
import math

import numpy as np
import pytest

from oracle import oracle as O


def _case(seed=3, ne=40, N=786432.0, Ny=128):
    rng = np.random.default_rng(seed)
    c = rng.chisquare(Ny, ne) + math.log(ne)
    gamma = N + math.sqrt(2 * N) * rng.standard_normal(ne)
    return c, gamma, N


def test_target_is_the_largest_c_and_its_particle_keeps_alpha_one():
    c, gamma, N = _case()
    gamma = np.minimum(gamma, N)            # x <= 1: c* = 0 gives alpha = 1 exactly
    sc = O.iewpf_scalars_one_stage(c, gamma, N)
    i = int(np.argmax(c))
    assert sc["w_target"] == c[i]
    assert sc["beta"] == 0.0
    assert sc["cstar"][i] == 0.0 and np.all(sc["cstar"] >= 0.0)
    assert math.isclose(sc["alpha"][i], 1.0, rel_tol=1e-13)
    others = np.arange(len(c)) != i
    assert np.all(sc["alpha"][others] < 1.0) and np.all(sc["alpha"] > 0.0)


def test_alpha_is_the_lambert_w_formula():
    # eq. iewpfAlphaSol evaluated directly with scipy's W_0, on inputs whose
    # argument stays away from the branch point -1/e (small N_psi, spread gamma)
    from scipy.special import lambertw
    N = 50.0
    gamma = np.array([20.0, 35.0, 49.0, 60.0, 80.0])
    c = np.array([4.0, 9.5, 1.0, 6.0, 2.5])
    sc = O.iewpf_scalars_one_stage(c, gamma, N)
    cstar = c.max() - c
    ref = -(N / gamma) * lambertw(-(gamma / N) * np.exp(-gamma / N) * np.exp(-cstar / N), 0).real
    assert np.allclose(sc["alpha"], ref, rtol=1e-11, atol=0)


def test_every_particle_reaches_the_target_weight():
    c, gamma, N = _case(seed=11, ne=100)
    sc = O.iewpf_scalars_one_stage(c, gamma, N)
    # eq. implicitEquation (large-N_psi form) with -log w_i = w_target
    res = (sc["alpha"] - 1.0) * gamma - N * np.log(sc["alpha"]) - (c.max() - c)
    assert np.all(np.abs(res) <= 1e-12 * N)
    assert np.allclose(sc["neglogw"], sc["w_target"], rtol=1e-12, atol=0)


def test_one_stage_target_moves_away_from_the_mean_as_the_ensemble_grows():
    # App. A: max c_i grows with N_e while mean c_i (less the common log N_e)
    # stays; the two-stage target is the mean
    gaps = []
    for ne in (10, 100, 1000):
        c, gamma, N = _case(seed=5, ne=ne)
        one = O.iewpf_scalars_one_stage(c, gamma, N)
        gaps.append(one["w_target"] - one["cbar"])
    assert gaps[0] < gaps[1] < gaps[2]
    # and the particles move further: the smallest alpha shrinks
    a_min = [O.iewpf_scalars_one_stage(*_case(seed=5, ne=ne))["alpha"].min() for ne in (10, 1000)]
    assert a_min[1] < a_min[0]


def test_one_particle_schemes_differ_by_the_nu_term():
    # N_e = 1: the two-stage beta is 1 and both schemes have c* = 0, so both
    # use the same alpha; the posteriors differ by P^{1/2} nu (eqs.
    # iewpfUpdateAgain, updateEquationTwoStageAgain), P^{1/2} being the
    # block roots followed by Q^{1/2}
    P = O.Problem(nx=64, ny=64, dx=2000.0, dy=2000.0)
    rng = np.random.default_rng(2)
    ens = (rng.normal(0, 1, (1, 3, 64, 64)) * np.array([0.01, 20, 20])[None, :, None, None])
    cells = [(20, 20), (45, 40)]
    y = np.array([[3.0, -2.0], [1.0, 4.0]])
    two, d2 = O.assimilate(P, ens, cells, y, t=1)
    one, d1 = O.assimilate(P, ens, cells, y, t=1, one_stage=True)
    assert d2["beta"] == 1.0 and d1["beta"] == 0.0
    assert d1["alpha"][0] == d2["alpha"][0]
    nu = d2["nu"].copy()
    Msq = O.local_block_sqrt(P)
    for cl in cells:
        idx = O.block_indices(P, cl)
        nu[:, idx] = nu[:, idx] @ Msq.T
    diff = O.add_qhalf(P, nu[0], np.zeros((3, 64, 64)))
    assert np.max(np.abs((two - one)[0] - diff)) <= 1e-9 * np.max(np.abs(diff))


def test_one_stage_analysis_equalises_weights_and_pulls_toward_observations():
    P = O.Problem(nx=64, ny=64, dx=2000.0, dy=2000.0)
    rng = np.random.default_rng(9)
    ne = 8
    base = rng.normal(0, 1, (3, 64, 64)) * np.array([0.01, 20, 20])[:, None, None]
    ens = np.stack([base + rng.normal(0, 1, (3, 64, 64)) * np.array([0.005, 10, 10])[:, None, None]
                    for _ in range(ne)])
    cells = [(20, 20), (45, 40)]
    y = np.array([[base[1, 20, 20], base[2, 20, 20]], [base[1, 40, 45], base[2, 40, 45]]])
    out, dg = O.assimilate(P, ens, cells, y, t=2, one_stage=True)
    assert dg["w_target"] == dg["c"].max()
    assert np.allclose(dg["neglogw"], dg["w_target"], rtol=1e-10, atol=0)
    d_after = O.innovations(P, out, cells, y).reshape(ne, -1)
    assert np.mean(d_after ** 2) < np.mean(dg["d"] ** 2)
