"""Pins of the oracle's rank of an observed value within the ensemble
(Sec. 5.1): the insertion position into the sorted perturbed members, the
extremes 0 and N_e, the unperturbed limit, and a flat histogram when truth
and members are exchangeable, which fails if the members' perturbation by
the observation error is left out."""
import numpy as np
from scipy.stats import chisquare

from oracle import oracle as O


def _problem(n, sigma):
    # obs_sigma is sigma_vel * H in the oracle's Problem
    return O.Problem(nx=n, ny=n, dx=1.0, dy=1.0, obs_sigma=sigma)


def test_rank_is_the_insertion_position_in_the_sorted_perturbed_members():
    P = _problem(16, 0.4)
    rng = np.random.default_rng(1)
    ens = rng.standard_normal((9, 3, 16, 16))
    cells = np.array([[3, 4], [15, 0], [7, 11]])
    y = rng.standard_normal((3, 2))
    r = O.ranks(P, ens, cells, y, t=5)
    eps = np.stack([O.normals(P.seed, i, 5, O.STREAM_RANK, 6) for i in range(9)])
    for m, (j, k) in enumerate(cells):
        for c in (0, 1):
            vals = np.sort(ens[:, 1 + c, k, j] + P.obs_sigma * eps[:, 2 * m + c])
            assert r[m, c] == np.searchsorted(vals, y[m, c])


def test_extremes_and_the_unperturbed_limit():
    P = _problem(8, 1e-12)
    ens = np.random.default_rng(2).standard_normal((7, 3, 8, 8))
    cells = np.array([[1, 1], [2, 5]])
    lo = np.full((2, 2), -100.0)
    hi = np.full((2, 2), 100.0)
    assert np.all(O.ranks(P, ens, cells, lo, t=0) == 0)
    assert np.all(O.ranks(P, ens, cells, hi, t=0) == 7)
    # no observation error: plain count of members below
    y = np.array([[0.1, -0.2], [0.3, 0.0]])
    r = O.ranks(P, ens, cells, y, t=0)
    for m, (j, k) in enumerate(cells):
        for c in (0, 1):
            assert r[m, c] == int(np.sum(ens[:, 1 + c, k, j] < y[m, c]))


def _histogram(perturb_members):
    n, ne, sigma = 40, 9, 1.0
    P = _problem(n, sigma if perturb_members else 1e-300)
    rng = np.random.default_rng(3)
    ens = rng.standard_normal((ne, 3, n, n))
    truth = rng.standard_normal((3, n, n))
    jj, kk = np.meshgrid(np.arange(n), np.arange(n))
    cells = np.stack([jj.ravel(), kk.ravel()], axis=1)
    y = np.stack([truth[1, cells[:, 1], cells[:, 0]], truth[2, cells[:, 1], cells[:, 0]]], axis=1)
    y = y + sigma * rng.standard_normal(y.shape)          # observations carry the error
    r = O.ranks(P, ens, cells, y, t=1)
    return np.bincount(r.ravel(), minlength=ne + 1)


def test_exchangeable_truth_gives_a_flat_histogram():
    h = _histogram(True)
    assert h.sum() == 2 * 40 * 40
    assert chisquare(h).pvalue > 1e-3


def test_leaving_members_unperturbed_gives_a_u_shape():
    h = _histogram(False)
    assert chisquare(h).pvalue < 1e-6
    assert h[0] + h[-1] > 2.5 * h.sum() / len(h)
