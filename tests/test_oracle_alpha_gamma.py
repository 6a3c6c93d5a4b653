"""Pins of the oracle's incomplete-gamma alpha (App. A, eq.
numericalEqForAlpha) and of its log P: closed forms of the incomplete gamma
function for N_psi = 2 and 4, scipy's gammainc at moderate s, a 40-digit
series at s = 1.57e6 (where scipy's gammainc is off by 1e-4 relative in the
tail), a 50-digit solve with mpmath, alpha = 1 at c* = 0, monotonicity in c*,
and agreement with the Lambert-W solution (eq. iewpfAlphaSol) once c* is
large enough for the derivative term that the Lambert-W form drops to be
negligible."""
import math

import numpy as np
import pytest

from oracle import oracle as O


def test_log_p_closed_form_and_library_at_moderate_s():
    from scipy.special import gammainc
    # log P is a difference of terms of size s log x: it carries an absolute
    # error of a few ulp of those (relative error of P itself)
    for x in (1e-8, 0.3, 2.0, 17.0):
        assert math.isclose(O.log_gamma_p(1.0, x), math.log(-math.expm1(-x)), rel_tol=1e-13, abs_tol=1e-13)
    for s, x in ((5.0, 3.0), (30.0, 31.5), (500.0, 440.0), (500.0, 560.0)):
        assert math.isclose(O.log_gamma_p(s, x), math.log(gammainc(s, x)), rel_tol=1e-12, abs_tol=1e-12)


def test_log_p_at_large_s_against_a_forty_digit_series():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    s = mpmath.mpf(1572864)

    def logp(x):
        x = mpmath.mpf(x)
        term = sm = mpmath.mpf(1)
        n = 1
        while term >= sm * mpmath.mpf(10) ** -45:
            term *= x / (s + n)
            sm += term
            n += 1
        return s * mpmath.log(x) - x - mpmath.loggamma(s + 1) + mpmath.log(sm)

    # the median region and 6.3 standard deviations below it
    for x in (1574639.7957679094, 1566766.59678907):
        assert abs(O.log_gamma_p(1572864.0, x) - float(logp(x))) < 1e-8


def test_two_dimensions_closed_form():
    # P(1, x) = 1 - exp(-x): alpha = -(2/gamma) log(1 - exp(-c*/2)(1 - exp(-gamma/2)))
    g = np.array([0.3, 1.5, 3.0, 9.0, 2.2])
    cs = np.array([0.1, 0.7, 2.0, 30.0, 300.0])         # the last: alpha near 1e-66
    ref = -(2.0 / g) * np.log1p(-np.exp(-cs / 2) * -np.expm1(-g / 2))
    assert np.allclose(O.alpha_incomplete_gamma(g, cs, 2.0), ref, rtol=1e-12, atol=0)


def test_four_dimensions_residual():
    # P(2, x) = 1 - (1 + x) exp(-x)
    P2 = lambda x: -math.expm1(-x) - x * math.exp(-x)
    g = np.array([1.0, 4.0, 7.5])
    cs = np.array([0.5, 3.0, 12.0])
    a = O.alpha_incomplete_gamma(g, cs, 4.0)
    for ai, gi, ci in zip(a, g, cs):
        assert math.isclose(P2(0.5 * ai * gi), math.exp(-ci / 2) * P2(0.5 * gi), rel_tol=1e-12)


@pytest.mark.parametrize("N,g,cs", [(60.0, 55.0, 3.0), (60.0, 70.0, 0.2), (1000.0, 1030.0, 25.0)])
def test_against_a_fifty_digit_solve(N, g, cs):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    s = mpmath.mpf(N) / 2
    rhs = mpmath.exp(-mpmath.mpf(cs) / 2) * mpmath.gammainc(s, 0, mpmath.mpf(g) / 2, regularized=True)
    f = lambda a: mpmath.gammainc(s, 0, a * mpmath.mpf(g) / 2, regularized=True) - rhs
    lo, hi = mpmath.mpf("0.01"), mpmath.mpf(1)      # f(lo) < 0 < f(hi): bisection in 50 digits
    assert f(lo) < 0 < f(hi)
    for _ in range(120):
        mid = (lo + hi) / 2
        lo, hi = (mid, hi) if f(mid) < 0 else (lo, mid)
    ref = (lo + hi) / 2
    assert math.isclose(O.alpha_incomplete_gamma([g], [cs], N)[0], float(ref), rel_tol=1e-11)


def test_on_target_and_monotone():
    N = 5000.0
    g = np.full(6, 5050.0)
    cs = np.array([0.0, 0.5, 2.0, 10.0, 50.0, 400.0])
    a = O.alpha_incomplete_gamma(g, cs, N)
    assert a[0] == 1.0
    assert np.all(np.diff(a) < 0.0) and a[-1] > 0.0


def test_approaches_the_lambert_w_solution_for_large_cstar():
    N = 10000.0
    ratios = []
    for cs in (1.0, 10.0, 100.0, 1000.0):
        ag = O.alpha_incomplete_gamma([N], [cs], N)[0]
        al = O.iewpf_scalars_one_stage([cs, 0.0], [N, N], N)["alpha"][1]
        ratios.append((1.0 - ag) / (1.0 - al))
    assert all(r < 1.0 for r in ratios)
    assert np.all(np.diff(ratios) > 0.0) and ratios[-1] > 0.99
