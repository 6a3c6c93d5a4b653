"""Pins of the oracle's IEWPF analysis (Sec. 4, App. A) against the paper's
printed non-zero counts, dense brute force on tiny grids, the Kalman
identity, the covariance identity of P, orthogonality of the random vectors,
Lambert-W identities and the equal-weights property."""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def p64(**kw):
    return O.Problem(nx=64, ny=64, dx=2000.0, dy=2000.0, **kw)


# --------------------------------------------------------------------------
# Fig. localsvd: non-zero counts on a 10 x 10 grid with Omega^M = Omega^R
# --------------------------------------------------------------------------
def test_localsvd_nonzero_patterns():
    g = json.load(open(os.path.join(GOLDEN, "localsvd_nonzeros.json")))
    P = p64()
    m = O.localsvd_matrices(P, n=g["grid"][0])
    N = 100
    Qs, GB, Hm, S = m["Qs"], m["GB"], m["H"], m["S"]

    def pat(X):  # index pattern of an operator (structural non-zeros)
        return (np.abs(X) > 0).astype(np.int64)

    def mul(X, Y):  # pattern of a product: union of supports
        return ((X @ Y) > 0).astype(np.int64)

    pQ, pG, pH = pat(Qs), pat(GB), pat(Hm)
    pS = np.ones((2, 2), np.int64)
    assert np.all(pQ.sum(axis=1) == g["nonzeros_per_row_Q_SOAR"])
    pGQ = mul(pG, pQ)
    assert np.all(pGQ[N:2 * N].sum(axis=1) == g["nonzeros_per_row_Q_GB_hu_rows"])
    assert np.all(pGQ[2 * N:].sum(axis=1) == g["nonzeros_per_row_Q_GB_hv_rows"])
    pHGQ = mul(pH, pGQ)
    assert np.all(pHGQ.sum(axis=1) == g["nonzeros_per_row_H_Q_GB_Q_SOAR"])
    pT = mul(pG.T, mul(pH.T, mul(pS, pHGQ)))
    assert (pT.sum(axis=1) > 0).sum() == g["nonzero_rows_after_adjoint_GB"]
    pA = mul(pQ, pT)
    rows = np.nonzero(pA.sum(axis=1))[0]
    assert len(rows) == g["nonzero_rows_A"]
    assert np.all(pA[rows].sum(axis=1) == g["nonzeros_per_nonzero_row_A"])
    # the numeric matrix lives inside that pattern (symmetry cancels the
    # row of the observed cell itself)
    A = np.eye(N) - m["I_minus_A"]
    num_rows = np.nonzero((np.abs(A) > 1e-12 * np.abs(A).max()).sum(axis=1))[0]
    assert set(num_rows) <= set(rows) and len(num_rows) >= 40
    # the 45 rows are the 7x7 block around the observation minus its corners
    j0, k0 = m["j0"], m["k0"]
    cells = {(r % 10 - j0, r // 10 - k0) for r in rows}
    block = {(p, q) for p in range(-3, 4) for q in range(-3, 4)} - \
        {(-3, -3), (-3, 3), (3, -3), (3, 3)}
    assert cells == block
    assert O.local_block(P).shape == tuple(g["local_block"])


def test_local_block_root():
    P = p64()
    Bk = O.local_block(P)
    lam = np.linalg.eigvalsh(0.5 * (Bk + Bk.T))
    assert np.all(lam > 0) and np.all(lam <= 1 + 1e-12)
    assert np.sum(np.abs(lam - 1) < 1e-12) == 47          # I minus a rank-2 term
    Msq = O.local_block_sqrt(P)
    assert np.allclose(Msq, Msq.T, atol=1e-14)
    assert np.allclose(Msq @ Msq, Bk, atol=1e-12)


def test_covariance_of_P_with_identity_interpolation():
    """With Omega^M = Omega^R the local root reproduces
    P = Q - Q H^T S H Q exactly (eq. PcovExpression)."""
    P = p64()
    m = O.localsvd_matrices(P)
    n, j0, k0 = m["n"], m["j0"], m["k0"]
    Qh = m["GB"] @ m["Qs"]                                 # Q^{1/2}: 3N x N
    Q = Qh @ Qh.T
    Hm, S = m["H"], m["S"]
    Pcov = Q - Q @ Hm.T @ S @ Hm @ Q
    idx = [((k0 + q) % n) * n + (j0 + p) % n for q in range(-3, 4) for p in range(-3, 4)]
    Mfull = np.eye(n * n)
    Mfull[np.ix_(idx, idx)] = O.local_block_sqrt(P)
    Ph = Qh @ Mfull
    assert np.allclose(Ph @ Ph.T, Pcov, rtol=0, atol=1e-12 * np.abs(Pcov).max())


# --------------------------------------------------------------------------
# Pull stencil and (HQH^T + R)
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


def _pull_field(P, K, cell, comp):
    Sd = np.zeros((1, 2))
    Sd[0, comp] = 1.0
    return O.add_pull(P, K, [cell], Sd, np.zeros((3, P.ny, P.nx))).ravel()


def test_pull_stencil_equals_dense_q_with_identity_interpolation():
    """c_Omega = 1: the adjoint chain is the exact transpose, so the pull of a
    unit observation must equal Q^{1/2} (Q^{1/2})^T H^T e built from dense
    matrices of the forward operator."""
    P = O.Problem(nx=18, ny=17, dx=2000.0, dy=2000.0, c_omega=1)
    K = O.pull_stencil(P)
    Qh = _dense_qhalf(P)
    N = P.nx * P.ny
    cell = (6, 9)
    for comp in range(2):
        e = np.zeros(3 * N)
        e[(1 + comp) * N + cell[1] * P.nx + cell[0]] = 1.0
        dense = Qh @ (Qh.T @ e)
        got = _pull_field(P, K, cell, comp)
        assert np.allclose(got, dense, rtol=0, atol=1e-12 * np.abs(dense).max())


def test_pull_stencil_equals_dense_chain_with_coarse_grid():
    """c_Omega = 3, observation on a coarse point of a uniform coarse grid:
    the pull equals Q^{1/2} Q_SOAR^{1/2} Q_GB^{1/2,T} I^T H^T e with the
    forward operator as a dense matrix and the adjoint geostrophic balance
    of eq. adjointGeoBalance on the coarse grid (coefficient g H / f)."""
    P = O.Problem(nx=48, ny=48, dx=2000.0, dy=2500.0, c_omega=3)
    K = O.pull_stencil(P)
    Qh = _dense_qhalf(P)
    a0, b0 = 7, 6
    cell = (1 + 3 * a0, 1 + 3 * b0)
    s = P.g * P.H / P.f
    for comp in range(2):
        dip = np.zeros((P.nRy, P.nRx))
        if comp == 0:
            dip[b0 + 1, a0] = -s / (2 * 3 * P.dy)
            dip[b0 - 1, a0] = s / (2 * 3 * P.dy)
        else:
            dip[b0, a0 + 1] = s / (2 * 3 * P.dx)
            dip[b0, a0 - 1] = -s / (2 * 3 * P.dx)
        dense = Qh @ O.soar(P, dip).ravel()
        got = _pull_field(P, K, cell, comp)
        assert np.allclose(got, dense, rtol=0, atol=1e-12 * np.abs(dense).max())


def test_single_observation_hqht_is_diagonal_and_isotropic():
    P = p64()
    K = O.pull_stencil(P)
    M = O.hqht(P, K, [(20, 30)])
    assert abs(M[0, 1]) < 1e-12 * M[0, 0] and abs(M[1, 0]) < 1e-12 * M[0, 0]
    assert math.isclose(M[0, 0], M[1, 1], rel_tol=1e-12)
    assert M[0, 0] > 0


def test_kalman_identity_of_the_pull():
    """The pull is linear, so at the observed cells
    H(psi^a) - H(psi^f) = (HQH^T) S d = d - R S d (eq. opd_update)."""
    P = p64()
    K = O.pull_stencil(P)
    rng = np.random.default_rng(5)
    cells = [(10, 12), (40, 20), (25, 50)]              # farther apart than the support
    for dense in (True, False):
        A = O.s_matrix(P, K, cells, dense)
        d = rng.normal(0, 5, 6)
        Sd = O.cholesky_solve(A, d)
        U = rng.normal(0, 1, (3, 64, 64))
        Ua = O.add_pull(P, K, cells, Sd.reshape(-1, 2), U)
        dH = np.array([Ua[1 + q, c[1], c[0]] - U[1 + q, c[1], c[0]] for c in cells for q in range(2)])
        assert np.allclose(dH, d - P.obs_sigma ** 2 * Sd, rtol=1e-11, atol=1e-11)


def test_dense_hqht_couples_close_observations():
    P = p64()
    K = O.pull_stencil(P)
    near = O.hqht(P, K, [(10, 10), (13, 11)])
    far = O.hqht(P, K, [(10, 10), (50, 40)])
    assert np.abs(near[:2, 2:]).max() > 1e-3 * near[0, 0]
    assert np.abs(far[:2, 2:]).max() == 0.0
    assert np.all(O.hqht(P, K, [(10, 10), (13, 11)], dense=False)[:2, 2:] == 0)
    assert np.all(np.linalg.eigvalsh(O.s_matrix(P, K, [(10, 10), (13, 11)])) > 0)


def test_cholesky_solve_matches_library_solve():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((30, 30))
    A = X @ X.T + 30 * np.eye(30)
    B = rng.standard_normal((30, 4))
    assert np.allclose(O.cholesky_solve(A, B), np.linalg.solve(A, B), rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------------
# Random vectors, target weight, beta, alpha
# --------------------------------------------------------------------------
def test_perpendicular_random_vectors():
    P = p64()
    rv = O.rand_vectors(P, 6, t=3)
    for i in range(6):
        nu, xi, nut = rv["nu"][i], rv["xi"][i], rv["nut"][i]
        assert abs(nu @ xi) <= 1e-12 * math.sqrt((nu @ nu) * (xi @ xi))
        assert math.isclose(nu @ nu, nut @ nut, rel_tol=1e-12)
    assert np.allclose(rv["gamma"], rv["xx"] * P.N_psi / P.N_R)


def test_gamma_zeta_statistics():
    """gamma_i = xi^T xi N_psi/N_R has mean N_psi and variance 2 N_psi^2/N_R."""
    P = p64()
    rv = O.rand_vectors(P, 400, t=1)
    sd = math.sqrt(2.0 / P.N_R) * P.N_psi
    for key in ("gamma", "zeta"):
        assert abs(rv[key].mean() - P.N_psi) < 5 * sd / math.sqrt(400)
        assert 0.7 < rv[key].std() / sd < 1.3


def _scalars_case(seed=0, ne=50, N=786432, Ny=128):
    rng = np.random.default_rng(seed)
    phi = rng.chisquare(Ny, ne)
    c = phi + math.log(ne)
    gamma = N + math.sqrt(2 * N) * rng.standard_normal(ne)
    zeta = N + math.sqrt(2 * N) * rng.standard_normal(ne)
    return c, gamma, zeta, N


def test_lambert_w0_against_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    for q in (0.0, 1e-300, 1e-14, 1e-9, 3e-6, 1e-3, 0.3, 2.0, 40.0):
        w = O.lambert_w0_branch(q)
        z = -mpmath.exp(-1 - mpmath.mpf(q))
        ref = mpmath.lambertw(z, 0)
        # relative error a few ulp (the last case is limited by log near 41)
        assert abs(float(ref.real) - w) <= 1e-14 * abs(w), q
        # w e^w = z, checked in high precision
        wm = mpmath.mpf(w)
        assert abs(wm * mpmath.exp(wm) - z) <= 1e-14 * abs(z), q


def test_lambert_w0_against_scipy_away_from_branch_point():
    from scipy.special import lambertw
    for q in (0.05, 0.5, 3.0, 10.0):
        z = -math.exp(-1 - q)
        assert math.isclose(O.lambert_w0_branch(q), lambertw(z, 0).real, rel_tol=1e-12)


def test_iewpf_scalars_properties():
    c, gamma, zeta, N = _scalars_case()
    sc = O.iewpf_scalars(c, gamma, zeta, N)
    cs = sc["cstar"]
    i0 = int(np.argmin((sc["cbar"] - c) / zeta + 1.0))
    assert np.all(cs >= -1e-9 * np.abs(c).max())
    assert abs(cs[i0]) <= 1e-9 * abs(c).max()                      # eq. betaRequirement tight
    assert 0.0 < sc["beta"] < 1.0
    assert np.all(sc["alpha"] <= 1.0) and np.all(sc["alpha"] > 0.0)
    res = (sc["alpha"] - 1) * gamma - N * np.log(sc["alpha"]) - np.maximum(cs, 0)
    assert np.all(np.abs(res) <= 1e-12 * N)
    # every particle reaches the target weight w_target = mean c_i
    assert np.allclose(sc["neglogw"], sc["cbar"], rtol=1e-10, atol=0)


def test_alpha_is_one_when_already_on_target():
    N = 1000.0
    gamma = np.array([900.0, 999.0, 1000.0])
    # choose c so that c* = 0 for all with beta = 1: c_i = cbar, zeta arbitrary
    c = np.array([5.0, 5.0, 5.0])
    zeta = np.array([1000.0, 1000.0, 1000.0])
    sc = O.iewpf_scalars(c, gamma, zeta, N)
    assert sc["beta"] == 1.0
    assert np.allclose(sc["alpha"], 1.0, rtol=1e-12)
    # and gamma > N with c* = 0 gives alpha < 1 (the other root of eq. implicitEquation)
    sc2 = O.iewpf_scalars(c, np.array([1100.0, 1100.0, 1100.0]), zeta, N)
    assert np.all(sc2["alpha"] < 1.0)


# --------------------------------------------------------------------------
# Whole analysis, drifters, forecast errors
# --------------------------------------------------------------------------
def test_assimilate_equal_weights_and_pull_toward_observations():
    P = p64()
    rng = np.random.default_rng(9)
    ne = 8
    base = rng.normal(0, 1, (3, 64, 64)) * np.array([0.01, 20, 20])[:, None, None]
    ens = np.stack([base + rng.normal(0, 1, (3, 64, 64)) * np.array([0.005, 10, 10])[:, None, None]
                    for _ in range(ne)])
    cells = [(20, 20), (45, 40)]
    y = np.array([[base[1, 20, 20], base[2, 20, 20]], [base[1, 40, 45], base[2, 40, 45]]])
    out, dg = O.assimilate(P, ens, cells, y, t=2)
    assert np.allclose(dg["neglogw"], dg["cbar"], rtol=1e-10, atol=0)
    d_after = O.innovations(P, out, cells, y).reshape(ne, -1)
    assert np.mean(d_after ** 2) < np.mean(dg["d"] ** 2)


def test_drifter_uniform_flow_is_exactly_linear():
    P = p64()
    U = np.zeros((3, 64, 64))
    u0, v0 = 0.25, -0.125
    U[1] = u0 * P.H
    U[2] = v0 * P.H
    xy = np.array([[100.0, 200.0], [127000.0, 3.0]])
    out = xy.copy()
    for _ in range(16):
        out = O.drift(P, U, 7.5, out)
    assert np.array_equal(out, xy + np.array([u0, v0]) * 120.0)


def test_forecast_errors_equal_rmse_for_mean_truth():
    rng = np.random.default_rng(3)
    traj = rng.normal(0, 1000, (5, 10, 4, 2))
    truth = traj.mean(axis=1)
    E, R = O.forecast_errors(traj, truth)
    assert np.allclose(E, R, rtol=1e-14)
    E2, _ = O.forecast_errors(traj, truth + 100.0)
    assert np.all(E2 > E)


def _phis(c_omega, cells, n=400):
    """phi = d^T (HQH^T + R)^{-1} d for innovations drawn as H Q^{1/2} xi + eps
    (the forward model-error chain at the observed cells plus observation
    noise), with HQH^T assembled from the pull stencils."""
    P = p64(obs_sigma=2.0, c_omega=c_omega)
    K = O.pull_stencil(P)
    A = O.s_matrix(P, K, cells, dense=True)
    rng = np.random.default_rng(17)
    zero = np.zeros((3, 64, 64))
    phis = []
    for k in range(n):
        xi = O.normals(P.seed, k, 3, O.STREAM_MODEL_ERROR, P.N_R)
        dpsi = O.add_qhalf(P, xi, zero)
        y = np.array([[dpsi[1, b, a], dpsi[2, b, a]] for a, b in cells])
        y = y + P.obs_sigma * rng.standard_normal(y.shape)
        d = O.innovations(P, zero[None], cells, y).reshape(-1)
        phis.append(float(d @ O.cholesky_solve(A, d)))
    return np.array(phis)


CHI2_CELLS = [(10, 12), (40, 15), (20, 45), (50, 50)]


def test_phi_is_chi_square_with_n_y_degrees_of_freedom():
    # with c_Omega = 1 the stencil HQH^T is the covariance of the forward
    # chain's output exactly, so phi follows chi^2(N_y) (Sec. 4, App. A:
    # c_bar - c_i about N_y +- sqrt(2 N_y)); the assembly from the stencils is
    # independent of the forward chain
    n_y = 2 * len(CHI2_CELLS)
    phis = _phis(1, CHI2_CELLS)
    se = math.sqrt(2 * n_y / len(phis))
    assert abs(phis.mean() - n_y) < 4 * se, (phis.mean(), n_y)
    assert 0.7 * 2 * n_y < phis.var() < 1.4 * 2 * n_y
    # a 20% error in the scale of HQH^T + R would be seen
    assert abs(0.8 * phis.mean() - n_y) > 4 * se


def test_observation_centred_lattice_bias_with_coarse_model_error():
    # with c_Omega = 3 the pull puts the coarse lattice on the observation
    # (Sec. 4.2, Fig. optimalproposalpull) while the model error lives on the
    # fixed lattice: for observations between coarse nodes HQH^T is the
    # at-node covariance and phi averages about 10% above N_y
    n_y = 2 * len(CHI2_CELLS)
    phis = _phis(3, CHI2_CELLS)
    assert 1.03 * n_y < phis.mean() < 1.2 * n_y, phis.mean()


def test_innovation_of_a_particle_equal_to_the_truth_is_zero():
    # eq. buoyObservation observes hu H/(H + eta) of the truth and eq.
    # etaCompensatedInnovation scales the observation back by (H + eta_i)/H
    # (the paper states the two are consistent): a particle equal to the
    # truth has zero innovation even where eta is far from 0, and a particle
    # with the truth's momentum but another eta does not
    P = p64()
    rng = np.random.default_rng(31)
    truth = np.stack([rng.normal(0, 1, (64, 64)) * 3.0,        # eta of metres
                      rng.normal(0, 1, (64, 64)) * 20.0,
                      rng.normal(0, 1, (64, 64)) * 20.0])
    cells = [(3, 5), (40, 22), (63, 63)]
    s = np.array([P.H / (P.H + truth[0, b, a]) for a, b in cells])
    y = np.array([[truth[1, b, a], truth[2, b, a]] for a, b in cells]) * s[:, None]
    d = O.innovations(P, truth[None], cells, y)
    assert np.max(np.abs(d)) <= 1e-12 * np.max(np.abs(y))
    other = truth.copy()
    other[0] += 1.0
    assert np.min(np.abs(O.innovations(P, other[None], cells, y))) > 1e-3


def test_observed_cell_contains_the_position():
    # the cell (j, k) covers [j dx, (j+1) dx) x [k dy, (k+1) dy) (cell centres
    # at ((j + 1/2) dx, (k + 1/2) dy)); positions outside the domain wrap
    P = O.Problem(nx=64, ny=48, dx=2000.0, dy=2500.0)
    for j, k in ((0, 0), (63, 47), (17, 30)):
        for fx, fy in ((0.5, 0.5), (0.0, 0.0), (0.999, 0.001)):
            assert O.obs_cell(P, (j + fx) * 2000.0, (k + fy) * 2500.0) == (j, k)
    assert O.obs_cell(P, -1.0, 48 * 2500.0 + 1.0) == (63, 0)


def test_nearest_coarse_point_and_its_7x7_block():
    # coarse points at o + c a (o = c // 2); the nearest one to a fine index,
    # across the seam of the short last gap; the block is 7 x 7 coarse points
    # around it, ordered (dy + 3) * 7 + (dx + 3), wrapping periodically
    n, c = 64, 3                          # points 1, 4, ..., 61; the gap 61 -> 65 = 1
    nR = O.Problem(nx=n, ny=n, dx=1.0, dy=1.0).nRx
    pos = [c // 2 + c * a for a in range(nR)]
    for j in range(n):
        dist = [min(abs(j - p), n - abs(j - p)) for p in pos]
        best = min(dist)
        a = O.nearest_coarse(n, nR, c, j)
        assert dist[a] == best, j
    P = p64()
    idx = O.block_indices(P, (4, 61))     # x at coarse 1, y at coarse 20 (the last)
    ax, by = O.nearest_coarse(64, P.nRx, 3, 4), O.nearest_coarse(64, P.nRy, 3, 61)
    assert (ax, by) == (1, 20)
    expect = [((by + dy) % P.nRy) * P.nRx + (ax + dx) % P.nRx for dy in range(-3, 4) for dx in range(-3, 4)]
    assert list(idx) == expect and len(set(expect)) == 49
