"""Pins of oracle parts that earlier pins could not tell from plausible
mistakes, each against a closed form, brute force or an exact invariant:

* the drift-forecast error E(t) and RMSE(t) of eqs. errorPerEnsembleDrifter
  and errorNorm on a hand-computed case;
* the CFL time step of eq. swecfl on states whose wave speeds are known in
  closed form;
* every entry of the dense H Q H^T of eq. S_extended (close observations and
  a pair straddling the periodic seam) against H Q^{1/2} (Q^{1/2})^T H^T
  from dense matrices, and the Kalman identity of the pull with those
  observations;
* the tangential momentum flux of the scheme (Sec. 3.1; carried by the mass
  flux with the upwind tangential velocity): passive transport of a
  tangential velocity by a uniform flow, whose exact solution is a
  translation, with the maximum principle that upwinding gives;
* the full nonlinear scheme on an axisymmetric vortex in gradient-wind
  balance, an exact steady state of eq. swe_full;
* one whole two-stage analysis (Sec. 4, eq. optUpdateEquationTwoStage) in
  the linear-Gaussian case: ensemble mean against the exact Kalman pull and
  ensemble covariance against (beta + E[alpha gamma / N_psi]) P, with P the
  dense Q - Q H^T S H Q."""
import math

import numpy as np
import pytest

from oracle import oracle as O


# --------------------------------------------------------------------------
# eqs. errorPerEnsembleDrifter, errorNorm
# --------------------------------------------------------------------------
def test_forecast_errors_on_a_hand_computed_case():
    # truth: drifter 1 at (0, 0), drifter 2 at (10, 0)
    # particle 1: (3, 4) and (10, 6); particle 2: (0, 0) and (13, 4)
    traj = np.array([[[[3.0, 4.0], [10.0, 6.0]],
                      [[0.0, 0.0], [13.0, 4.0]]]])          # [n_out=1][N_e=2][N_D=2][2]
    truth = np.array([[[0.0, 0.0], [10.0, 0.0]]])
    E, R = O.forecast_errors(traj, truth)
    # E_1 = (25 + 0) / 2 = 12.5, E_2 = (36 + 25) / 2 = 30.5, E = sqrt(21.5)
    assert E[0] == pytest.approx(math.sqrt(21.5), rel=1e-15)
    # ensemble means (1.5, 2) and (11.5, 5): every squared deviation of
    # drifter 1 is 6.25 and of drifter 2 is 3.25, RMSE = sqrt(4.75)
    assert R[0] == pytest.approx(math.sqrt(4.75), rel=1e-15)
    # a second output time: everything shifted by (7, -2) keeps both errors
    E2, R2 = O.forecast_errors(np.concatenate([traj, traj + [7.0, -2.0]]),
                               np.concatenate([truth, truth + [7.0, -2.0]]))
    assert np.allclose(E2, math.sqrt(21.5), rtol=1e-15) and np.allclose(R2, math.sqrt(4.75), rtol=1e-15)


# --------------------------------------------------------------------------
# eq. swecfl
# --------------------------------------------------------------------------
def test_cfl_step_of_the_lake_at_rest():
    # c = sqrt(9.81 * 230) = 47.500526... m/s; dt = 0.45 / 4 * 2000 / c
    P = O.Problem(nx=20, ny=16, dx=2000.0, dy=2500.0)
    U = np.zeros((3, 16, 20))
    assert O.cfl_dt(P, U) == pytest.approx(4.7367896204, rel=1e-10)
    assert O.n_sub(P, U) == 13               # 60 / 4.7368 = 12.67


def test_cfl_step_of_uniform_flows_and_a_single_fast_cell():
    # eta = 0.1 m, u = 0.5, v = -0.3 m/s everywhere: h = 230.1,
    # c = sqrt(9.81 * 230.1) = 47.510851...; x limits with dx = 2000,
    # dy = 2500: dt = 0.1125 * 2000 / (0.5 + c)
    P = O.Problem(nx=20, ny=16, dx=2000.0, dy=2500.0)
    h = 230.1
    U = np.zeros((3, 16, 20))
    U[0] = 0.1
    U[1] = 0.5 * h
    U[2] = -0.3 * h
    assert O.cfl_dt(P, U) == pytest.approx(4.6864405333, rel=1e-10)
    # dy small enough for the y direction to limit: 0.1125 * 500 / (0.3 + c)
    Py = O.Problem(nx=20, ny=16, dx=2000.0, dy=500.0)
    assert O.cfl_dt(Py, U) == pytest.approx(1.1765111552, rel=1e-10)
    # one cell with u = 20 m/s sets the step for the whole field
    V = U.copy()
    V[1, 7, 3] = 20.0 * h
    assert O.cfl_dt(P, V) == pytest.approx(3.3327975483, rel=1e-10)
    assert O.n_sub(P, V) == 19


# --------------------------------------------------------------------------
# eq. S_extended: dense H Q H^T with couplings, against brute force
# --------------------------------------------------------------------------
def _dense_qhalf(P):
    N, NR = P.nx * P.ny, P.N_R
    Qh = np.zeros((3 * N, NR))
    Z = np.zeros((3, P.ny, P.nx))
    for m in range(NR):
        e = np.zeros(NR)
        e[m] = 1.0
        Qh[:, m] = O.add_qhalf(P, e, Z).ravel()
    return Qh


def _obs_rows(P, cells):
    N = P.nx * P.ny
    Hm = np.zeros((2 * len(cells), 3 * N))
    for m, (j, k) in enumerate(cells):
        Hm[2 * m, N + k * P.nx + j] = 1.0          # hu
        Hm[2 * m + 1, 2 * N + k * P.nx + j] = 1.0  # hv
    return Hm


# close pairs (1-3 cells apart), a pair straddling the seam in x and y, and a
# far one; with c_Omega = 1 the pull chain is exactly Q^{1/2} (Q^{1/2})^T
SEAM_CELLS = [(6, 9), (8, 10), (5, 7), (17, 2), (1, 15), (11, 4)]


def test_dense_hqht_equals_brute_force_with_close_and_seam_observations():
    P = O.Problem(nx=18, ny=17, dx=2000.0, dy=2500.0, c_omega=1)
    K = O.pull_stencil(P)
    Qh = _dense_qhalf(P)
    Hm = _obs_rows(P, SEAM_CELLS)
    ref = Hm @ Qh @ Qh.T @ Hm.T
    got = O.hqht(P, K, SEAM_CELLS)
    scale = np.abs(ref).max()
    # the seam pair (17, 2)-(1, 15) is 2 cells apart in x and 4 in y across
    # the boundaries: its coupling is well away from zero
    assert np.abs(ref[6:8, 8:10]).max() > 1e-3 * scale
    assert np.allclose(got, ref, rtol=0, atol=1e-12 * scale)
    # the paper's block form keeps exactly the 2 x 2 diagonal blocks
    blk = O.hqht(P, K, SEAM_CELLS, dense=False)
    mask = np.kron(np.eye(len(SEAM_CELLS)), np.ones((2, 2))).astype(bool)
    assert np.allclose(blk[mask], ref[mask], rtol=0, atol=1e-12 * scale) and np.all(blk[~mask] == 0)


def test_dense_hqht_is_the_symmetrised_pull_response_with_coarse_model_error():
    """With c_Omega = 3 the pull of eq. detailedOPDUpdate (on a coarse
    lattice centred on each observation) is not exactly symmetric between
    two observations, so H Q H^T is the symmetrised matrix of responses:
    entry ((l, a), (k, b)) is field a of the pull of a unit b observation at
    obs k read at obs l's cell.  Built here by applying the pull one unit
    observation at a time, for close, seam-straddling and far pairs."""
    P = O.Problem(nx=48, ny=45, dx=2000.0, dy=2500.0, c_omega=3)
    K = O.pull_stencil(P)
    cells = [(10, 12), (13, 13), (11, 17), (46, 3), (2, 41), (30, 30)]
    N = P.nx * P.ny
    n = len(cells)
    Rm = np.zeros((2 * n, 2 * n))
    for k, ck in enumerate(cells):
        for b in range(2):
            Sd = np.zeros((n, 2))
            Sd[k, b] = 1.0
            resp = O.add_pull(P, K, cells, Sd, np.zeros((3, P.ny, P.nx))).ravel()
            for l, cl in enumerate(cells):
                for a in range(2):
                    Rm[2 * l + a, 2 * k + b] = resp[(1 + a) * N + cl[1] * P.nx + cl[0]]
    scale = np.abs(Rm).max()
    assert np.abs(Rm - Rm.T).max() > 1e-6 * scale          # the responses are not symmetric
    assert np.abs(Rm[6:8, 8:10]).max() > 1e-3 * scale        # the seam pair is coupled
    assert np.allclose(O.hqht(P, K, cells), 0.5 * (Rm + Rm.T), rtol=0, atol=1e-13 * scale)


def test_kalman_identity_with_close_and_seam_observations():
    """H(psi^a) - H(psi^f) = H Q H^T S d = d - R S d (eq. opd_update) once
    the pull reaches neighbouring observations and wraps around the seam."""
    P = O.Problem(nx=18, ny=17, dx=2000.0, dy=2500.0, c_omega=1)
    K = O.pull_stencil(P)
    rng = np.random.default_rng(11)
    A = O.s_matrix(P, K, SEAM_CELLS)
    d = rng.normal(0, 5, 2 * len(SEAM_CELLS))
    Sd = O.cholesky_solve(A, d)
    U = rng.normal(0, 1, (3, P.ny, P.nx))
    Ua = O.add_pull(P, K, SEAM_CELLS, Sd.reshape(-1, 2), U)
    dH = np.array([Ua[1 + q, c[1], c[0]] - U[1 + q, c[1], c[0]] for c in SEAM_CELLS for q in range(2)])
    assert np.allclose(dH, d - P.obs_sigma ** 2 * Sd, rtol=1e-11, atol=1e-11)


# --------------------------------------------------------------------------
# Sec. 3.1: tangential momentum carried with the upwind tangential velocity
# --------------------------------------------------------------------------
def _transport_state(P, axis, profile, U0=0.5):
    """Uniform flow U0 along `axis` (0: x, 1: y) carrying a tangential
    velocity that varies along the same axis; f = 0, eta = 0."""
    n = P.nx if axis == 0 else P.ny
    x = (np.arange(n) + 0.5) / n
    w = profile(x)
    U = np.zeros((3, P.ny, P.nx))
    if axis == 0:
        U[1] = P.H * U0
        U[2] = (P.H * w)[None, :]
    else:
        U[2] = P.H * U0
        U[1] = (P.H * w)[:, None]
    return U, x


def _transport(axis, n, profile, T, U0=0.5):
    L = 64e3
    dxy = L / n
    P = O.Problem(nx=n if axis == 0 else 4, ny=4 if axis == 0 else n, dx=dxy, dy=dxy, f=0.0)
    U, x = _transport_state(P, axis, profile, U0)
    dt = O.cfl_dt(P, U)
    steps = int(math.ceil(T / dt))
    out = U
    for _ in range(steps):
        out = O.swe_substep(P, out, T / steps)
    field = out[2] if axis == 0 else out[1]
    line = field[0, :] if axis == 0 else field[:, 0]
    other = out[1:3][axis]                       # the normal momentum
    exact = P.H * profile((x - U0 * T / L) % 1.0)
    return P, U, out, line, exact, other


@pytest.mark.parametrize("axis", [0, 1])
def test_tangential_momentum_is_transported_by_the_mass_flux(axis):
    """A smooth tangential velocity in a uniform flow is translated with the
    flow (exact solution of eq. swe_full with f = 0); the error converges
    at better than first order over two refinements, and eta and the normal
    momentum stay uniform."""
    prof = lambda x: 0.2 * np.sin(2 * np.pi * x)
    T = 32e3                                     # the flow moves a quarter of the domain
    errs = []
    for n in (32, 64, 128):
        P, U, out, line, exact, other = _transport(axis, n, prof, T)
        errs.append(np.sqrt(np.mean((line - exact) ** 2)) / (P.H * 0.2))
        assert np.all(out[0] == 0.0)
        assert np.all(other == other.flat[0])
        # nothing depends on the transverse coordinate
        f = out[2] if axis == 0 else out[1]
        assert np.all(f == (f[:1, :] if axis == 0 else f[:, :1]))
    assert errs[0] > errs[1] > errs[2]
    assert errs[0] / errs[2] > 6.0, errs              # order > 1.3
    assert errs[2] < 2e-3


@pytest.mark.parametrize("axis", [0, 1])
def test_transported_step_keeps_its_bounds_and_moves_with_the_flow(axis):
    """Upwinding keeps the transported velocity within its initial bounds
    (no new extrema at a step), and its centre of mass moves U0 T."""
    prof = lambda x: ((x > 0.25) & (x < 0.5)).astype(float)
    T = 12.8e3                                   # 0.1 of the domain
    P, U, out, line, exact, other = _transport(axis, 64, prof, T)
    lo, hi = 0.0, P.H * 1.0
    assert line.min() >= lo - 1e-9 * hi and line.max() <= hi + 1e-9 * hi
    x = (np.arange(64) + 0.5) / 64
    c0 = np.sum(P.H * prof(x) * x) / np.sum(P.H * prof(x))
    c1 = np.sum(line * x) / np.sum(line)
    assert c1 - c0 == pytest.approx(0.5 * T / 64e3, rel=1e-6)
    assert np.sum(line) == pytest.approx(np.sum(P.H * prof(x)), rel=1e-12)


# --------------------------------------------------------------------------
# eq. swe_full: gradient-wind vortex
# --------------------------------------------------------------------------
def _vortex(n, L=200e3, R=20e3, A=0.3, f=1e-4):
    """eta = -A exp(-r^2 / 2R^2) with the azimuthal velocity of gradient-wind
    balance, v^2 / r + f v = g deta/dr (the root that tends to geostrophy):
    an exact steady solution of the rotating shallow-water equations."""
    P = O.Problem(nx=n, ny=n, dx=L / n, dy=L / n, f=f)
    c = (np.arange(n) + 0.5) * (L / n) - 0.5 * L
    X, Y = np.meshgrid(c, c)
    r = np.hypot(X, Y)
    eta = -A * np.exp(-r ** 2 / (2 * R ** 2))
    detadr = A * r / R ** 2 * np.exp(-r ** 2 / (2 * R ** 2))
    vt = 0.5 * (-f * r + np.sqrt((f * r) ** 2 + 4 * P.g * r * detadr))
    with np.errstate(invalid="ignore", divide="ignore"):
        u = np.where(r > 0, -vt * Y / r, 0.0)
        v = np.where(r > 0, vt * X / r, 0.0)
    h = P.H + eta
    U = np.stack([eta, h * u, h * v])
    return P, U, vt.max()


def _vortex_error(n, T=1800.0):
    P, U, vmax = _vortex(n)
    dt = O.cfl_dt(P, U)
    steps = int(math.ceil(T / dt))
    out = U
    for _ in range(steps):
        out = O.swe_substep(P, out, T / steps)
    hU = P.H * vmax
    e_mom = np.sqrt(np.mean((out[1:] - U[1:]) ** 2)) / hU
    e_eta = np.sqrt(np.mean((out[0] - U[0]) ** 2)) / 0.3
    return e_mom, e_eta, vmax, P.f


def test_gradient_wind_vortex_is_steady_to_second_order():
    """Rossby number about 0.34 (v^2 / r about a third of f v at the radius
    of the strongest flow), so the centrifugal part of the balance, which
    comes from the nonlinear momentum fluxes (normal and tangential),
    matters at the 25% level: a scheme without the tangential flux leaves
    the balance by a fixed amount per unit time, whatever the resolution."""
    e = [_vortex_error(n) for n in (32, 64, 128)]
    vmax, f = e[0][2], e[0][3]
    assert vmax / (f * 20e3) > 0.3                  # Rossby number
    for q in range(2):
        assert e[0][q] > e[1][q] > e[2][q]
        assert e[0][q] / e[2][q] > 6.0, [x[q] for x in e]   # order > 1.3
    assert e[2][0] < 5e-3


# --------------------------------------------------------------------------
# Sec. 4, eq. optUpdateEquationTwoStage: one analysis, linear-Gaussian case
# --------------------------------------------------------------------------
def test_one_analysis_in_the_linear_gaussian_case():
    """Every particle starts from the same state psi_f, so every innovation
    d, every c_i and hence c_bar are equal: beta = 1 and c*_i = 0.  The
    two-stage posterior psi_f + Q H^T S d + P^{1/2}(beta^{1/2} nu +
    alpha^{1/2} xi) then has mean psi_f + Q H^T S d (the Kalman pull) and
    covariance P^{1/2}(beta E[nu nu^T] + E[alpha xi xi^T]) P^{1/2,T} =
    (1 + E[alpha gamma / N_psi]) P: nu is isotropic with E[nu nu^T] = I,
    alpha depends on xi only through its length, gamma / N_psi = |xi|^2 /
    N_R.  P = Q - Q H^T S H Q is formed from dense matrices of Q^{1/2} on a
    grid where the 7 x 7 block of Sec. 4.6 is exact (c_Omega = 1)."""
    P = O.Problem(nx=12, ny=12, dx=2000.0, dy=2000.0, c_omega=1, obs_sigma=2.3)
    rng = np.random.default_rng(2)
    ne = 4000
    psi_f = np.zeros((3, 12, 12))
    psi_f[0] = 0.05 * rng.standard_normal((12, 12))
    psi_f[1:] = 5.0 * rng.standard_normal((2, 12, 12))
    cells = [(6, 5)]
    y = np.array([[psi_f[1, 5, 6] + 4.0, psi_f[2, 5, 6] - 3.0]])
    ens = np.broadcast_to(psi_f, (ne, 3, 12, 12)).copy()
    out, dg = O.assimilate(P, ens, cells, y, t=3)
    assert dg["beta"] == 1.0 and np.all(dg["cstar"] == 0.0)
    # dense brute force of the pull and of P
    Qh = _dense_qhalf(P)
    Q = Qh @ Qh.T
    Hm = _obs_rows(P, cells)
    Sm = np.linalg.inv(Hm @ Q @ Hm.T + P.obs_sigma ** 2 * np.eye(2))
    d = dg["d"][0]
    pull = Q @ Hm.T @ Sm @ d
    Pm = Q - Q @ Hm.T @ Sm @ Hm @ Q
    X = out.reshape(ne, -1) - psi_f.ravel()
    mean = X.mean(axis=0)
    m = float(np.mean(dg["alpha"] * dg["gamma"] / P.N_psi))
    assert 0.8 < m < 1.0
    sd = np.sqrt((1.0 + m) * np.clip(np.diag(Pm), 0.0, None) / ne)
    big = sd > 1e-9 * sd.max()
    assert np.all(np.abs(mean - pull)[big] <= 6.0 * sd[big])
    if not big.all():
        assert np.abs(mean - pull)[~big].max() <= 1e-9 * np.abs(pull).max()
    # covariance: along the observed components, where P is far below Q,
    # and along the leading directions of P
    C = np.cov(X, rowvar=False)
    tol = 6.0 * math.sqrt(2.0 / ne)
    obs = Hm @ C @ Hm.T
    pred = (1.0 + m) * (Hm @ Pm @ Hm.T)
    assert np.all(np.abs(np.diag(obs) / np.diag(pred) - 1.0) < tol)
    assert np.all(np.diag(Hm @ Pm @ Hm.T) < 0.5 * np.diag(Hm @ Q @ Hm.T))
    lam, V = np.linalg.eigh(Pm)
    for k in range(1, 6):
        v = V[:, -k]
        assert abs(v @ C @ v / ((1.0 + m) * lam[-k]) - 1.0) < tol
