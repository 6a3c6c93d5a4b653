"""iewpf_weights_noalloc, the weights step for callers that cannot allocate
device memory (pooling allocators, latency-bound loops): it must give the
results of iewpf_weights on the same inputs, on consecutive calls that share
its fixed scratch array, and refuse ensembles above its stated maximum.
This file is collected last on purpose."""
import math

import numpy as np
import pytest

from paper_1910_01031_gb300 import iewpf

pytestmark = pytest.mark.gpu


def _inputs(seed, ne, N, Ny):
    rng = np.random.default_rng(seed)
    c = rng.chisquare(Ny, ne) + math.log(ne)
    gamma = N + math.sqrt(2 * N) * rng.standard_normal(ne)
    zeta = N + math.sqrt(2 * N) * rng.standard_normal(ne)
    return c, gamma, zeta


def test_noalloc_weights_match_allocating_entry_point_on_consecutive_calls():
    # two calls in a row with different sizes: the second reuses the scratch
    for seed, ne, N, Ny in [(1, 1000, 3145728.0, 3042), (2, 37, 786432.0, 128)]:
        c, gamma, zeta = _inputs(seed, ne, N, Ny)
        ref = iewpf.weights(c, gamma, zeta, N)
        got = iewpf.weights(c, gamma, zeta, N, noalloc=True)
        assert math.isclose(got["cbar"], ref["cbar"], rel_tol=1e-10)
        assert math.isclose(got["beta"], ref["beta"], rel_tol=1e-10)
        for k in ("alpha", "cstar", "neglogw"):
            assert np.allclose(got[k], ref[k], rtol=1e-10, atol=1e-12), k
        assert np.allclose(got["neglogw"], got["cbar"], rtol=1e-10, atol=0)


def test_noalloc_weights_error_flag_is_cleared_between_calls():
    bad = (np.array([0.0, 1000.0, 0.0]), np.array([50.0, 50, 50]), np.array([50.0, 50, 50]))
    with pytest.raises(iewpf.IewpfError) as e:
        iewpf.weights(*bad, 60.0, noalloc=True)
    assert e.value.name == "EBETA"
    c, gamma, zeta = _inputs(3, 64, 12288.0, 2)
    got = iewpf.weights(c, gamma, zeta, 12288.0, noalloc=True)
    ref = iewpf.weights(c, gamma, zeta, 12288.0)
    assert np.allclose(got["alpha"], ref["alpha"], rtol=1e-10, atol=0)


def test_noalloc_weights_reject_ensembles_above_the_maximum():
    n = iewpf.WEIGHTS_NOALLOC_MAX_NE + 1
    c, gamma, zeta = _inputs(4, n, 12288.0, 2)
    with pytest.raises(iewpf.IewpfError) as e:
        iewpf.weights(c, gamma, zeta, 12288.0, noalloc=True)
    assert e.value.name == "EINVAL"


def test_noalloc_weights_at_the_largest_accepted_ensemble_then_a_smaller_call():
    # ne = maximum fills the -log w slice up to the c_bar/beta slot and the
    # flag that follow it; a smaller call afterwards must be unaffected
    ne = iewpf.WEIGHTS_NOALLOC_MAX_NE
    c, gamma, zeta = _inputs(5, ne, 3145728.0, 3042)
    ref = iewpf.weights(c, gamma, zeta, 3145728.0)
    got = iewpf.weights(c, gamma, zeta, 3145728.0, noalloc=True)
    assert math.isclose(got["cbar"], ref["cbar"], rel_tol=1e-10)
    assert math.isclose(got["beta"], ref["beta"], rel_tol=1e-10)
    for k in ("alpha", "cstar", "neglogw"):
        assert np.allclose(got[k], ref[k], rtol=1e-10, atol=1e-12), k
    c, gamma, zeta = _inputs(6, 10, 12288.0, 2)
    ref = iewpf.weights(c, gamma, zeta, 12288.0)
    got = iewpf.weights(c, gamma, zeta, 12288.0, noalloc=True)
    assert math.isclose(got["beta"], ref["beta"], rel_tol=1e-10)
    for k in ("alpha", "cstar", "neglogw"):
        assert np.allclose(got[k], ref[k], rtol=1e-10, atol=1e-12), k
