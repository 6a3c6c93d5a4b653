"""Pins of the oracle's standard particle filter weights (Sec. 2.1, eqs.
standardParticleFilter, standardParticleFilterWeight) and the count of
particles above 1/N_e (Sec. 5.3): the two-particle logistic form, scipy's
softmax, equal innovations, the power law of a scaled R and extreme
innovations that underflow a plain exp."""
import math

import numpy as np
from scipy.special import expit, softmax

from oracle import oracle as O
from paper_1910_01031_gb300 import synth


def _d(seed, ne, nobs, scale=1.0):
    return scale * np.random.default_rng(seed).standard_normal((ne, nobs, 2))


def test_two_particles_follow_the_logistic_form():
    d = _d(1, 2, 3)
    sigma2 = 0.7
    w, kept = O.sir_weights(d, [[0, 2]], sigma2)
    l = 0.5 * np.sum(d[:, [0, 2], :] ** 2, axis=(1, 2)) / sigma2
    assert math.isclose(w[0, 0], expit(l[1] - l[0]), rel_tol=1e-14)
    assert math.isclose(w[0, 0] + w[0, 1], 1.0, rel_tol=1e-15)
    assert kept[0] == 1                    # one of two is above 1/2 (no tie here)


def test_weights_are_the_softmax_of_minus_half_the_misfit():
    d = _d(2, 30, 8, scale=2.0)
    sets = synth.observation_subsets(8, 3, 5)
    w, kept = O.sir_weights(d, sets, sigma2=1.5, r_scale=10.0)
    for s, S in enumerate(sets):
        x = -0.5 * np.sum(d[:, S, :] ** 2, axis=(1, 2)) / 15.0
        ref = softmax(x)
        assert np.allclose(w[s], ref, rtol=1e-12, atol=0)
        assert kept[s] == int(np.sum(ref > 1.0 / 30))


def test_equal_innovations_give_equal_weights_and_no_sure_survivor():
    d = np.tile(_d(3, 1, 4), (10, 1, 1))
    w, kept = O.sir_weights(d, [[0, 1, 2, 3]], 1.0)
    assert np.all(w == 0.1)
    assert kept[0] == 0                    # 1/N_e is not above 1/N_e


def test_scaling_r_takes_the_weights_to_a_power():
    # w_i(r R) is proportional to w_i(R)^(1/r)
    d = _d(4, 12, 5)
    w1, _ = O.sir_weights(d, [[0, 1, 2, 3, 4]], 0.8, r_scale=1.0)
    w10, _ = O.sir_weights(d, [[0, 1, 2, 3, 4]], 0.8, r_scale=10.0)
    p = w1[0] ** 0.1
    assert np.allclose(w10[0], p / p.sum(), rtol=1e-12, atol=0)


def test_extreme_innovations_do_not_underflow():
    # misfits of order 1e4: exp(-l) underflows for every particle, the
    # normalised weights do not; the best particle takes everything
    d = _d(5, 6, 2, scale=150.0)
    d[3] *= 1e-3
    w, kept = O.sir_weights(d, [[0, 1]], 1.0)
    assert np.isfinite(w).all() and w[0, 3] == 1.0 and kept[0] == 1


def test_subsets_are_distinct_sorted_and_seeded():
    a = synth.observation_subsets(64, 7, 50)
    b = synth.observation_subsets(64, 7, 50)
    assert a.shape == (50, 7) and np.array_equal(a, b)
    for row in a:
        assert len(set(row.tolist())) == 7 and np.all(np.diff(row) > 0) and row.max() < 64
