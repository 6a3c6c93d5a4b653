"""Pins of the oracle's shallow-water stepper (Sec. 3.1) against exact
properties: lake at rest, mass conservation, discrete geostrophic balance
(well-balancing), translation and transpose symmetry, and the closed-form
linear geostrophic adjustment of a cosine bump."""
import math

import numpy as np
import pytest

from oracle import oracle as O


def problem(nx=32, ny=24, **kw):
    return O.Problem(nx=nx, ny=ny, dx=2000.0, dy=2000.0, **kw)


def smooth_state(P, seed=0, amp=0.05):
    rng = np.random.default_rng(seed)
    x = (np.arange(P.nx) + 0.5) / P.nx
    y = (np.arange(P.ny) + 0.5) / P.ny
    X, Y = np.meshgrid(x, y)
    U = np.zeros((3, P.ny, P.nx))
    for q in range(3):
        for _ in range(4):
            a, b = rng.integers(1, 4, 2)
            ph = rng.uniform(0, 2 * np.pi)
            scale = amp if q == 0 else 40.0
            U[q] += scale * rng.uniform(0.2, 1.0) * np.sin(2 * np.pi * (a * X + b * Y) + ph)
    U[0] += 1e-3 * rng.standard_normal((P.ny, P.nx))
    return U


def run(P, U, n, dt=None):
    dt = O.cfl_dt(P, U) if dt is None else dt
    for _ in range(n):
        U = O.swe_substep(P, U, dt)
    return U


def test_lake_at_rest_is_exactly_steady():
    P = problem()
    U = np.zeros((3, P.ny, P.nx))
    out = run(P, U, 25, dt=5.0)
    assert np.array_equal(out, U)


def test_mass_is_conserved():
    P = problem()
    U = smooth_state(P, 1)
    out = run(P, U, 30)
    scale = np.abs(U[0]).sum()
    assert abs(out[0].sum() - U[0].sum()) <= 1e-11 * scale
    assert np.abs(out - U).max() > 1e-6          # the state did evolve


def _x_jet(P, V0=0.3):
    """A discrete geostrophic jet along y: K-differences vanish on every
    x-face, i.e. g (eta_{j+1} - eta_j) = f dx (v_j + v_{j+1}) / 2."""
    j = np.arange(P.nx)
    v = V0 * np.sin(2 * np.pi * j / P.nx)
    eta = np.zeros(P.nx)
    for i in range(P.nx - 1):
        eta[i + 1] = eta[i] + P.f * P.dx / (2 * P.g) * (v[i] + v[i + 1])
    eta -= eta.mean()
    U = np.zeros((3, P.ny, P.nx))
    U[0] = eta[None, :]
    U[2] = (v * (P.H + eta))[None, :]
    return U


def _y_jet(P, U0=0.3):
    k = np.arange(P.ny)
    u = U0 * np.sin(2 * np.pi * k / P.ny)
    eta = np.zeros(P.ny)
    for i in range(P.ny - 1):
        eta[i + 1] = eta[i] - P.f * P.dy / (2 * P.g) * (u[i] + u[i + 1])
    eta -= eta.mean()
    U = np.zeros((3, P.ny, P.nx))
    U[0] = eta[:, None]
    U[1] = (u * (P.H + eta))[:, None]
    return U


@pytest.mark.parametrize("maker", [_x_jet, _y_jet])
def test_discrete_geostrophic_jet_is_steady(maker):
    """Well-balancing (eq. geostrophic_balance_cont): a jet in discrete
    geostrophic balance stays put to rounding, while the same jet with its
    momentum from plain central differences (not the scheme's balance) moves
    by orders of magnitude more."""
    P = problem(nx=48, ny=40)
    U = maker(P)
    out = run(P, U, 40)
    ref = np.abs(U).max(axis=(1, 2))
    drift = np.abs(out - U).max(axis=(1, 2))
    assert np.all(drift <= 1e-11 * np.maximum(ref, 1.0))
    # control: momentum from the central differences of eq. geostrophic_balance_disc
    W = U.copy()
    s = P.g * P.H / P.f
    W[1] = -s * (np.roll(U[0], -1, 0) - np.roll(U[0], 1, 0)) / (2 * P.dy)
    W[2] = s * (np.roll(U[0], -1, 1) - np.roll(U[0], 1, 1)) / (2 * P.dx)
    out2 = run(P, W, 40)
    assert np.abs(out2 - W).max(axis=(1, 2)).max() > 1e4 * drift.max()


def test_translation_invariance_is_bitwise():
    P = problem()
    U = smooth_state(P, 2)
    sh = (5, 7)
    a = np.roll(run(P, U, 3, dt=4.0), sh, axis=(1, 2))
    b = run(P, np.roll(U, sh, axis=(1, 2)), 3, dt=4.0)
    assert np.array_equal(a, b)


def test_transpose_symmetry_with_reversed_rotation():
    """Swapping x and y (and hu with hv) mirrors the domain, which reverses
    the sense of rotation: the mirrored state under -f must evolve into the
    mirror of the original evolution."""
    P = problem(nx=32, ny=24)
    Pt = O.Problem(nx=24, ny=32, dx=P.dy, dy=P.dx, f=-P.f)
    U = smooth_state(P, 3)
    Ut = np.stack([U[0].T, U[2].T, U[1].T])
    a = run(P, U, 5, dt=4.0)
    b = run(Pt, Ut, 5, dt=4.0)
    at = np.stack([a[0].T, a[2].T, a[1].T])
    scale = np.abs(a).max(axis=(1, 2))[:, None, None]
    assert np.all(np.abs(at - b) <= 1e-12 * scale)


def _adjustment_error(nx):
    """Linear geostrophic adjustment of eta = A cos(kx), hu = hv = 0: with
    omega^2 = f^2 + g H k^2 the exact linear solution is
    eta = A [f^2/omega^2 + (g H k^2/omega^2) cos(omega t)] cos(kx) and
    hv = -H (A f g k / omega^2)(1 - cos(omega t)) sin(kx)."""
    Lx = 128e3
    P = O.Problem(nx=nx, ny=4, dx=Lx / nx, dy=Lx / nx, f=2e-3, H=230.0)
    A = 1e-4
    kx = 2 * np.pi / Lx
    x = (np.arange(nx) + 0.5) * P.dx
    U = np.zeros((3, P.ny, nx))
    U[0] = (A * np.cos(kx * x))[None, :]
    om = math.sqrt(P.f ** 2 + P.g * P.H * kx ** 2)
    T = math.pi / om
    n = int(math.ceil(T / O.cfl_dt(P, U)))
    out = run(P, U, n, dt=T / n)
    E = A * (P.f ** 2 / om ** 2 + P.g * P.H * kx ** 2 / om ** 2 * math.cos(om * T))
    V = -P.H * A * P.f * P.g * kx / om ** 2 * (1 - math.cos(om * T))
    err_eta = np.abs(out[0] - E * np.cos(kx * x)[None, :]).max() / A
    err_hv = np.abs(out[2] - V * np.sin(kx * x)[None, :]).max() / abs(V)
    return err_eta, err_hv


def test_linear_geostrophic_adjustment_converges():
    """The limiter clips the cosine's extrema, so the max-norm order is
    between one and two; over two refinements the error must fall by more
    than 6x (order > 1.3) and end below 5e-4 of the amplitude."""
    e = [_adjustment_error(n) for n in (32, 64, 128)]
    for q in range(2):
        assert e[0][q] > e[1][q] > e[2][q]
        assert e[0][q] / e[2][q] > 6.0
        assert e[2][q] < 5e-4


def test_cfl_and_substeps():
    P = problem()
    U = smooth_state(P, 4)
    h = P.H + U[0]
    c = np.sqrt(P.g * h)
    ax = (np.abs(U[1] / h) + c).max()
    ay = (np.abs(U[2] / h) + c).max()
    dt = P.courant * 0.25 * min(P.dx / ax, P.dy / ay)
    assert math.isclose(O.cfl_dt(P, U), dt, rel_tol=1e-14)
    assert O.n_sub(P, U) == math.ceil(P.dt_model / dt)


def test_forecast_matches_manual_steps():
    P = problem()
    U = smooth_state(P, 5)
    ens = np.stack([U, U * 0.5])
    out, nsub, _ = O.forecast(P, ens, 2, [True, False], t0=3)
    for i in range(2):
        V = ens[i].copy()
        for s, err in enumerate([True, False]):
            ns = O.n_sub(P, V)
            assert nsub[i, s] == ns
            V = run(P, V, ns, dt=P.dt_model / ns)
            if err:
                V = O.model_error(P, V, i, 3 + s)
        assert np.array_equal(out[i], V)
