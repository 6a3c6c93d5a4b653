"""Pins of the oracle's model-error operators (Sec. 3.2):
Q_SOAR^{1/2} (closed-form weights, 25 nonzeros per row, symmetry, empirical
covariance), I_Omega (interpolating, exact for quadratics, partition of
unity), Q_GB^{1/2} (closed form on a sine) and the composition."""
import math

import numpy as np
import pytest

from oracle import oracle as O


def prob(nx, ny, c=3, **kw):
    return O.Problem(nx=nx, ny=ny, dx=2000.0, dy=2500.0, c_omega=c, **kw)


def soar_matrix(P):
    NR = P.N_R
    W = np.zeros((NR, NR))
    for m in range(NR):
        e = np.zeros(NR)
        e[m] = 1.0
        W[:, m] = O.soar(P, e).ravel()
    return W


def test_coarse_grid_layout():
    # points at o + c a while inside the domain (o = floor(c/2))
    assert O.Problem(nx=64, ny=64, dx=1, dy=1).nRx == 21        # 1, 4, ..., 61
    assert O.Problem(nx=63, ny=63, dx=1, dy=1).nRx == 21        # divisible
    assert O.Problem(nx=512, ny=512, dx=1, dy=1).nRx == 171
    assert O.Problem(nx=1024, ny=1024, dx=1, dy=1).nRx == 341
    assert O.Problem(nx=10, ny=10, dx=1, dy=1, c_omega=1).nRx == 10


def test_soar_weights_and_nonzeros():
    """Each column of Q_SOAR^{1/2} holds the 5x5 block of SOAR values
    q0 (1 + d/L0) exp(-d/L0) at the coarse distances (eq. soar_function)."""
    P = prob(45, 36)                       # divisible: uniform 15 x 12 coarse grid
    W = soar_matrix(P)
    assert np.all((W != 0).sum(axis=0) == 25)
    assert np.all((W != 0).sum(axis=1) == 25)
    m = 6 * P.nRx + 7
    col = W[:, m].reshape(P.nRy, P.nRx)
    for db in range(-2, 3):
        for da in range(-2, 3):
            d = math.hypot(3 * 2000.0 * da, 3 * 2500.0 * db)
            expect = P.q0 * (1 + d / P.L0) * math.exp(-d / P.L0)
            assert math.isclose(col[6 + db, 7 + da], expect, rel_tol=1e-14)


def test_soar_is_symmetric_across_the_seam():
    P = prob(20, 23)                       # gaps of 2 and 2 cells at the seams
    W = soar_matrix(P)
    assert np.allclose(W, W.T, rtol=0, atol=1e-18)
    assert np.all(np.linalg.eigvalsh(W @ W.T) > -1e-18)


def test_soar_empirical_covariance():
    """Cov(delta eta) = Q_SOAR^{1/2} Q_SOAR^{1/2,T}: the sample covariance over
    20000 draws must match q0^2 sum_k K(a - k) K(b - k) within 5 standard
    errors at several separations."""
    P = prob(30, 30)                       # 10 x 10 coarse points
    n = 20000
    NR = P.N_R
    Z = np.stack([O.normals(P.seed, p, 0, 0, NR) for p in range(n)])
    W = soar_matrix(P)
    E = Z @ W.T                            # rows: samples of delta eta
    a = 4 * P.nRx + 4
    K = lambda da, db: P.q0 * (1 + math.hypot(6000.0 * da, 7500.0 * db) / P.L0) * \
        math.exp(-math.hypot(6000.0 * da, 7500.0 * db) / P.L0)
    for (oa, ob) in [(0, 0), (1, 0), (0, 1), (2, 1), (3, 3), (4, 0)]:
        b = (4 + ob) * P.nRx + (4 + oa)
        exact = 0.0
        for kb in range(-2, 3):
            for ka in range(-2, 3):
                # point k at offset (ka,kb) from a; need |offset from b| <= 2
                rb, ra = kb - ob, ka - oa
                if abs(ra) <= 2 and abs(rb) <= 2:
                    exact += K(ka, kb) * K(ra, rb)
        emp = np.mean(E[:, a] * E[:, b])
        se = math.sqrt((np.var(E[:, a]) * np.var(E[:, b]) + exact ** 2) / n)
        assert abs(emp - exact) < 5 * se + 1e-20, (oa, ob, emp, exact, se)


def test_bicubic_interpolates_and_reproduces_quadratics():
    P = prob(45, 36)
    rng = np.random.default_rng(0)
    C = rng.standard_normal((P.nRy, P.nRx))
    F = O.bicubic(P, C)
    o = P.c_omega // 2
    for b in range(P.nRy):
        for a in range(P.nRx):
            assert F[o + 3 * b, o + 3 * a] == C[b, a]
    # quadratic in the fine coordinates, sampled at the coarse points
    q = lambda x, y: 0.3 + 0.02 * x - 0.05 * y + 1e-3 * x * x + 2e-3 * x * y - 7e-4 * y * y
    Xc = o + 3 * np.arange(P.nRx)
    Yc = o + 3 * np.arange(P.nRy)
    Cq = q(Xc[None, :], Yc[:, None])
    Fq = O.bicubic(P, Cq)
    # fine cells whose 4x4 coarse taps do not wrap around the domain
    for k in range(o + 3, o + 3 * (P.nRy - 2)):
        for j in range(o + 3, o + 3 * (P.nRx - 2)):
            assert math.isclose(Fq[k, j], q(j, k), rel_tol=1e-12, abs_tol=1e-12)


def test_bicubic_partition_of_unity_with_seam():
    P = prob(64, 50)
    F = O.bicubic(P, np.ones((P.nRy, P.nRx)))
    assert np.allclose(F, 1.0, rtol=0, atol=1e-14)


def test_geostrophic_balance_closed_form():
    """Central differences of a sine are exact up to sin(k dx)/dx:
    hv = (g H / f) A sin(k dx)/dx cos(k x), hu = -(g H/f) B sin(l dy)/dy cos(l y)."""
    P = prob(40, 30)
    s = P.g * P.H / P.f
    j = np.arange(P.nx)
    k = np.arange(P.ny)
    A, m = 0.01, 3
    eta = np.tile(A * np.sin(2 * np.pi * m * j / P.nx), (P.ny, 1))
    hu, hv = O.gb(P, eta)
    kx = 2 * np.pi * m / (P.nx * P.dx)
    expect = s * A * math.sin(kx * P.dx) / P.dx * np.cos(2 * np.pi * m * j / P.nx)
    assert np.allclose(hv, expect[None, :], rtol=0, atol=1e-12 * abs(expect).max())
    assert np.abs(hu).max() < 1e-12 * abs(expect).max()
    B, l = 0.02, 2
    eta = np.tile((B * np.sin(2 * np.pi * l * k / P.ny))[:, None], (1, P.nx))
    hu, hv = O.gb(P, eta)
    ky = 2 * np.pi * l / (P.ny * P.dy)
    expect = -s * B * math.sin(ky * P.dy) / P.dy * np.cos(2 * np.pi * l * k / P.ny)
    assert np.allclose(hu, expect[:, None], rtol=0, atol=1e-12 * abs(expect).max())
    assert np.abs(hv).max() < 1e-12 * abs(expect).max()


def test_qhalf_is_linear_and_model_error_uses_stream_zero():
    P = prob(64, 64)
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal((2, P.N_R))
    Z = np.zeros((3, P.ny, P.nx))
    lin = O.add_qhalf(P, 2.0 * x - 3.0 * y, Z)
    sep = 2.0 * O.add_qhalf(P, x, Z) - 3.0 * O.add_qhalf(P, y, Z)
    scale = np.abs(lin).max(axis=(1, 2))[:, None, None]
    assert np.all(np.abs(lin - sep) <= 1e-13 * scale)
    U = rng.standard_normal((3, P.ny, P.nx))
    me = O.model_error(P, U, 7, 11)
    ref = O.add_qhalf(P, O.normals(P.seed, 7, 11, 0, P.N_R), U)
    assert np.array_equal(me, ref)
    assert 1e-5 < np.abs(me[0] - U[0]).max() < 1e-1
