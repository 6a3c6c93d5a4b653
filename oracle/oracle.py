"""FP64 CPU oracle for the IEWPF hot path (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
import this module.  It shares no code with the CUDA path: the grid operators
live in iewpf_oracle.c (plain C loops, double precision), the small dense
algebra of the analysis lives here (numpy; library routines such as a
Cholesky factorisation or a symmetric eigensolver serve as single steps).

Citations are to arXiv 1910.01031 (section / equation label).
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        _declare(_lib)
    return _lib


class SWE(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("g", ctypes.c_double), ("f", ctypes.c_double), ("H", ctypes.c_double),
                ("theta", ctypes.c_double)]


class ERR(ctypes.Structure):
    _fields_ = [("c", ctypes.c_int), ("nRx", ctypes.c_int), ("nRy", ctypes.c_int),
                ("q0", ctypes.c_double), ("L0", ctypes.c_double)]


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_up = ctypes.POINTER(ctypes.c_uint32)


def _declare(L):
    sp, ep = ctypes.POINTER(SWE), ctypes.POINTER(ERR)
    L.orc_philox.argtypes = [_up, _up, _up]
    L.orc_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                              ctypes.c_uint32, ctypes.c_long, _dp]
    L.orc_swe_rhs.argtypes = [sp, _dp, _dp]
    L.orc_swe_substep.argtypes = [sp, ctypes.c_double, _dp]
    L.orc_cfl_dt.argtypes = [sp, _dp, ctypes.c_double]
    L.orc_cfl_dt.restype = ctypes.c_double
    L.orc_n_sub.argtypes = [sp, _dp, ctypes.c_double, ctypes.c_double]
    L.orc_coarse_n.argtypes = [ctypes.c_int, ctypes.c_int]
    L.orc_soar.argtypes = [sp, ep, _dp, _dp]
    L.orc_bicubic.argtypes = [sp, ep, _dp, _dp]
    L.orc_gb.argtypes = [sp, _dp, _dp, _dp]
    L.orc_add_qhalf.argtypes = [sp, ep, _dp, _dp]
    L.orc_model_error.argtypes = [sp, ep, ctypes.c_uint64, ctypes.c_uint32,
                                  ctypes.c_uint32, _dp]
    L.orc_drift.argtypes = [sp, _dp, ctypes.c_double, ctypes.c_int, _dp]
    L.orc_forecast.argtypes = [sp, ep, ctypes.c_uint64, ctypes.c_int, _dp, ctypes.c_int,
                               _ip, ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                               ctypes.c_int, _dp, _ip, ctypes.c_int]
    L.orc_innovations.argtypes = [sp, ctypes.c_int, _dp, ctypes.c_int, _ip, _dp, _dp]
    L.orc_add_pull.argtypes = [sp, ctypes.c_int, _dp, ctypes.c_int, _ip, _dp, _dp]


def _d(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _i(a):
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_ip)


# ---------------------------------------------------------------------------
# Parameters
# ---------------------------------------------------------------------------
@dataclass
class Problem:
    """Grid, physics and model-error parameters (Secs. 3.1-3.2)."""
    nx: int
    ny: int
    dx: float
    dy: float
    g: float = 9.81
    f: float = 1.2e-4
    H: float = 230.0
    theta: float = 1.3
    courant: float = 0.45
    dt_model: float = 60.0
    c_omega: int = 3
    q0: float = 5e-4
    L0: float | None = None      # metres; default 0.75 coarse cells
    seed: int = 0x1910_01031
    obs_sigma: float = 2.3       # observation std in hu/hv units (m^2/s)

    def __post_init__(self):
        if self.L0 is None:
            self.L0 = 0.75 * self.c_omega * self.dx

    @property
    def nRx(self):
        return lib().orc_coarse_n(self.nx, self.c_omega)

    @property
    def nRy(self):
        return lib().orc_coarse_n(self.ny, self.c_omega)

    @property
    def N_psi(self):
        return 3 * self.nx * self.ny

    @property
    def N_R(self):
        return self.nRx * self.nRy

    def swe(self):
        return SWE(self.nx, self.ny, self.dx, self.dy, self.g, self.f, self.H, self.theta)

    def err(self):
        return ERR(self.c_omega, self.nRx, self.nRy, self.q0, self.L0)


# ---------------------------------------------------------------------------
# Random numbers
# ---------------------------------------------------------------------------
STREAM_MODEL_ERROR, STREAM_XI, STREAM_NU, STREAM_RANK = 0, 1, 2, 3


def philox(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox(c, k, o)
    return [int(x) for x in o]


def normals(seed, p, t, stream, n):
    z = np.empty(n, np.float64)
    lib().orc_normals(ctypes.c_uint64(seed), p, t, stream, n, _d(z))
    return z


# ---------------------------------------------------------------------------
# Model and model error
# ---------------------------------------------------------------------------
def swe_rhs(P: Problem, U):
    U = np.ascontiguousarray(U, np.float64)
    L = np.empty_like(U)
    s = P.swe()
    lib().orc_swe_rhs(ctypes.byref(s), _d(U), _d(L))
    return L


def swe_substep(P: Problem, U, dt):
    U = np.array(U, np.float64, order="C")
    s = P.swe()
    lib().orc_swe_substep(ctypes.byref(s), dt, _d(U))
    return U


def cfl_dt(P: Problem, U):
    U = np.ascontiguousarray(U, np.float64)
    s = P.swe()
    return lib().orc_cfl_dt(ctypes.byref(s), _d(U), P.courant)


def n_sub(P: Problem, U):
    U = np.ascontiguousarray(U, np.float64)
    s = P.swe()
    return lib().orc_n_sub(ctypes.byref(s), _d(U), P.courant, P.dt_model)


def soar(P: Problem, xi):
    xi = np.ascontiguousarray(xi, np.float64).reshape(P.nRy, P.nRx)
    out = np.empty_like(xi)
    s, e = P.swe(), P.err()
    lib().orc_soar(ctypes.byref(s), ctypes.byref(e), _d(xi), _d(out))
    return out


def bicubic(P: Problem, coarse):
    coarse = np.ascontiguousarray(coarse, np.float64).reshape(P.nRy, P.nRx)
    out = np.empty((P.ny, P.nx), np.float64)
    s, e = P.swe(), P.err()
    lib().orc_bicubic(ctypes.byref(s), ctypes.byref(e), _d(coarse), _d(out))
    return out


def gb(P: Problem, deta):
    deta = np.ascontiguousarray(deta, np.float64).reshape(P.ny, P.nx)
    hu = np.empty_like(deta)
    hv = np.empty_like(deta)
    s = P.swe()
    lib().orc_gb(ctypes.byref(s), _d(deta), _d(hu), _d(hv))
    return hu, hv


def add_qhalf(P: Problem, x, U):
    """U + Q^{1/2} x for a coarse field x (eq. covarianceOperatorsDef)."""
    x = np.ascontiguousarray(x, np.float64).reshape(P.nRy, P.nRx)
    U = np.array(U, np.float64, order="C")
    s, e = P.swe(), P.err()
    lib().orc_add_qhalf(ctypes.byref(s), ctypes.byref(e), _d(x), _d(U))
    return U


def model_error(P: Problem, U, p, t):
    U = np.array(U, np.float64, order="C")
    s, e = P.swe(), P.err()
    lib().orc_model_error(ctypes.byref(s), ctypes.byref(e), ctypes.c_uint64(P.seed), p, t, _d(U))
    return U


def drift(P: Problem, U, dt, xy):
    U = np.ascontiguousarray(U, np.float64)
    xy = np.array(xy, np.float64, order="C")
    s = P.swe()
    lib().orc_drift(ctypes.byref(s), _d(U), dt, xy.shape[0], _d(xy))
    return xy


def forecast(P: Problem, ens, n_steps, add_err, t0, xy=None, fixed_n_sub=0):
    """Ensemble forecast of n_steps model steps (eq. model_equation).

    add_err: bool or per-step list; the model error of step s uses draw
    counter t0 + s.  Returns (ens, n_sub[ne][n_steps], xy)."""
    ens = np.array(ens, np.float64, order="C")
    ne = ens.shape[0]
    if isinstance(add_err, (bool, int)):
        add_err = [int(add_err)] * n_steps
    ae = np.ascontiguousarray(add_err, np.int32)
    nsub = np.zeros((ne, n_steps), np.int32)
    nd = 0
    xyp = None
    if xy is not None:
        xy = np.array(xy, np.float64, order="C")
        nd = xy.shape[1]
        xyp = _d(xy)
    s, e = P.swe(), P.err()
    lib().orc_forecast(ctypes.byref(s), ctypes.byref(e), ctypes.c_uint64(P.seed), ne, _d(ens),
                       n_steps, _i(ae), t0, P.courant, P.dt_model, nd, xyp, _i(nsub),
                       int(fixed_n_sub))
    return ens, nsub, xy


# ---------------------------------------------------------------------------
# IEWPF: pull stencil, (HQH^T + R), local block of P, scalars
# ---------------------------------------------------------------------------
def soar_weight(d, q0, L0):
    """SOAR function (eq. soar_function)."""
    return q0 * (1.0 + d / L0) * np.exp(-d / L0)


def cubic_weights(t):
    """Catmull-Rom cubic convolution weights for taps a-1..a+2."""
    t2, t3 = t * t, t * t * t
    return np.array([0.5 * (-t3 + 2 * t2 - t), 0.5 * (3 * t3 - 5 * t2 + 2),
                     0.5 * (-3 * t3 + 4 * t2 + t), 0.5 * (t3 - t2)])


def stencil_radius(P: Problem):
    return 7 * P.c_omega


def pull_stencil(P: Problem):
    """Response of Q H^T to a unit hu and a unit hv observation at offset 0.

    Follows the chain of eq. detailedOPDUpdate right to left on a coarse
    lattice centred on the observed cell (Sec. 4.2, Fig. optimalproposalpull):
    I_Omega^T H^T (point injection), Q_GB^{1/2,T} on the coarse lattice
    (eq. adjointGeoBalance, coefficient g H_eq / f), Q_SOAR^{1/2} twice,
    I_Omega to the fine grid, Q_GB^{1/2} on the fine grid.
    Returns K[2][3][2R+1][2R+1] (obs component, field, dy, dx)."""
    c = P.c_omega
    R = stencil_radius(P)
    A = 10                         # coarse lattice half-width (support is +-5)
    n = 2 * A + 1
    dxc, dyc = c * P.dx, c * P.dy
    s = P.g * P.H / P.f
    K = np.zeros((2, 3, 2 * R + 1, 2 * R + 1))
    for comp in range(2):
        e = np.zeros((n, n))            # coarse eta [b][a], index offset A
        if comp == 0:   # unit hu: dipole in y
            e[A + 1, A] += -s / (2 * dyc)
            e[A - 1, A] += s / (2 * dyc)
        else:           # unit hv: dipole in x
            e[A, A + 1] += s / (2 * dxc)
            e[A, A - 1] += -s / (2 * dxc)
        for _ in range(2):              # Q_SOAR^{1/2}, applied twice
            out = np.zeros_like(e)
            for b in range(2, n - 2):
                for a in range(2, n - 2):
                    acc = 0.0
                    for db in range(-2, 3):
                        for da in range(-2, 3):
                            d = math.hypot(da * dxc, db * dyc)
                            acc += soar_weight(d, P.q0, P.L0) * e[b + db, a + da]
                    out[b, a] = acc
            e = out
        # I_Omega: fine offsets -(R+1)..R+1 (one extra cell for the differences)
        Rf = R + 1
        eta = np.zeros((2 * Rf + 1, 2 * Rf + 1))
        for fy in range(-Rf, Rf + 1):
            by = fy // c
            wy = cubic_weights((fy - by * c) / c)
            for fx in range(-Rf, Rf + 1):
                bx = fx // c
                wx = cubic_weights((fx - bx * c) / c)
                acc = 0.0
                for q in range(4):
                    for p in range(4):
                        acc += wy[q] * wx[p] * e[A + by - 1 + q, A + bx - 1 + p]
                eta[fy + Rf, fx + Rf] = acc
        # Q_GB^{1/2} on the fine grid
        inner = slice(1, 2 * Rf)
        K[comp, 0] = eta[inner, inner]
        K[comp, 1] = -s * (eta[2:, 1:-1] - eta[:-2, 1:-1]) / (2 * P.dy)
        K[comp, 2] = s * (eta[1:-1, 2:] - eta[1:-1, :-2]) / (2 * P.dx)
    return K


def min_image(d, n):
    d = d % n
    return d - n if d > n // 2 else d


def hqht(P: Problem, K, cells, dense=True):
    """H Q H^T assembled from the pull stencils: entry ((l,alpha),(k,beta))
    is component alpha of the response to a unit beta observation at obs k,
    read at obs l's cell (eq. S_extended).  Periodic images are summed.
    dense=False keeps only the 2x2 blocks of each observation (the paper's
    block-diagonal form, Sec. 4.2).  The result is symmetrised."""
    R = stencil_radius(P)
    cells = np.asarray(cells, dtype=np.int64).reshape(-1, 2)
    nobs = len(cells)
    M = np.zeros((2 * nobs, 2 * nobs))
    ddx = (cells[:, None, 0] - cells[None, :, 0]) % P.nx        # [l][k]
    ddy = (cells[:, None, 1] - cells[None, :, 1]) % P.ny
    if not dense:
        keep = np.eye(nobs, dtype=bool)
    else:
        keep = np.ones((nobs, nobs), dtype=bool)
    for ix in range(-(R // P.nx) - 1, (R // P.nx) + 2):
        ox = ddx + ix * P.nx
        for iy in range(-(R // P.ny) - 1, (R // P.ny) + 2):
            oy = ddy + iy * P.ny
            hit = keep & (np.abs(ox) <= R) & (np.abs(oy) <= R)
            l, k = np.nonzero(hit)
            if len(l) == 0:
                continue
            for a in range(2):
                for b in range(2):
                    np.add.at(M, (2 * l + a, 2 * k + b), K[b, 1 + a, oy[l, k] + R, ox[l, k] + R])
    return 0.5 * (M + M.T)


def s_matrix(P: Problem, K, cells, dense=True):
    """(H Q H^T + R), R = obs_sigma^2 I."""
    M = hqht(P, K, cells, dense)
    return M + P.obs_sigma ** 2 * np.eye(M.shape[0])


def cholesky_solve(A, B):
    """Solve A X = B for symmetric positive definite A by a Cholesky
    factorisation and two triangular solves."""
    import scipy.linalg as sla
    Lc = np.linalg.cholesky(A)
    Y = sla.solve_triangular(Lc, B, lower=True)
    return sla.solve_triangular(Lc.T, Y, lower=False)


def localsvd_matrices(P: Problem, n=10, j0=5, k0=5):
    """The construction of Fig. localsvd on an n x n periodic grid with
    Omega^M = Omega^R (c_Omega = 1, spacing of the coarse grid).

    Returns a dict with the dense Q_SOAR^{1/2} (N x N), Q_GB^{1/2} (3N x N),
    H (2 x 3N), S (2 x 2) and the parenthesis I - A of eq. svdOfParenthesis
    (N x N).  Cell (j,k) has index k*n + j."""
    N = n * n
    dxc, dyc = P.c_omega * P.dx, P.c_omega * P.dy
    s = P.g * P.H / P.f
    Qs = np.zeros((N, N))
    for k in range(n):
        for j in range(n):
            for b in range(-2, 3):
                for a in range(-2, 3):
                    d = math.hypot(a * dxc, b * dyc)
                    Qs[k * n + j, ((k + b) % n) * n + (j + a) % n] += soar_weight(d, P.q0, P.L0)
    GB = np.zeros((3 * N, N))
    for k in range(n):
        for j in range(n):
            i = k * n + j
            GB[i, i] = 1.0
            GB[N + i, ((k + 1) % n) * n + j] += -s / (2 * dyc)
            GB[N + i, ((k - 1) % n) * n + j] += s / (2 * dyc)
            GB[2 * N + i, k * n + (j + 1) % n] += s / (2 * dxc)
            GB[2 * N + i, k * n + (j - 1) % n] += -s / (2 * dxc)
    Hm = np.zeros((2, 3 * N))
    Hm[0, N + k0 * n + j0] = 1.0
    Hm[1, 2 * N + k0 * n + j0] = 1.0
    B = Hm @ GB @ Qs                       # H Q_GB^{1/2} Q_SOAR^{1/2}
    S = np.linalg.inv(B @ B.T + P.obs_sigma ** 2 * np.eye(2))
    A = Qs @ GB.T @ Hm.T @ S @ B           # Q_SOAR Q_GB^T H^T S H Q_GB Q_SOAR
    return {"Qs": Qs, "GB": GB, "H": Hm, "S": S, "I_minus_A": np.eye(N) - A,
            "n": n, "j0": j0, "k0": k0}


def local_block(P: Problem):
    """The 49 x 49 block of I - A around the observation (Fig. localsvd g),
    entries ordered (dy+3)*7 + (dx+3)."""
    m = localsvd_matrices(P)
    n, j0, k0 = m["n"], m["j0"], m["k0"]
    idx = [((k0 + q) % n) * n + (j0 + p) % n for q in range(-3, 4) for p in range(-3, 4)]
    return m["I_minus_A"][np.ix_(idx, idx)]


def local_block_sqrt(P: Problem):
    """Square root of the local block used as U Sigma^{1/2} (eq. Psquareroot).

    The block is symmetric positive semidefinite, so its SVD is an
    eigendecomposition V Lambda V^T.  Because 47 of its 49 eigenvalues equal
    one, V is not unique; the symmetric root V Lambda^{1/2} V^T is, and it
    gives perturbations with the same covariance."""
    Bk = local_block(P)
    Bk = 0.5 * (Bk + Bk.T)
    lam, V = np.linalg.eigh(Bk)
    lam = np.clip(lam, 0.0, None)
    return (V * np.sqrt(lam)) @ V.T


def obs_cell(P: Problem, x, y):
    return (int(math.floor(x / P.dx)) % P.nx, int(math.floor(y / P.dy)) % P.ny)


def nearest_coarse(n, nR, c, j):
    """Index of the coarse point nearest to fine index j (ties to the lower)."""
    o = c // 2
    if j < o:
        a = -1
    else:
        a = min((j - o) // c, nR - 1)
    def pos(a):
        w = a // nR
        return o + c * (a - w * nR) + w * n
    x0, x1 = pos(a), pos(a + 1)
    near = a if (j - x0) <= (x1 - j) else a + 1
    return near % nR


def _phi_s(s):
    """-s - log(1 - s) for s in [0, 1): its power series sum_{n>=2} s^n / n
    below 0.1 (no cancellation), the closed form above."""
    if s < 0.1:
        acc, term, n = 0.0, s * s, 2
        while True:
            add = term / n
            if acc + add == acc:
                return acc
            acc += add
            term *= s
            n += 1
    return -s - math.log1p(-s)


def _bisect(fun, lo, hi, target, increasing):
    for _ in range(300):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if (fun(mid) < target) == increasing:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def lambert_w0_branch(q):
    """W_0(z) for z = -exp(-1 - q), q >= 0, by bisection on its definition.

    W_0(z) is the w >= -1 with w e^w = z.  Taking logarithms of -w e^w = -z
    gives, for u = -w in (0, 1], u - 1 - log u = q.  For q <= 1/2 it is
    solved for s = 1 - u from -s - log(1 - s) = q (increasing in s), inside
    the bracket s^2/(2(1-s)) >= q >= s^2/2; for larger q for u itself
    (decreasing in u) inside exp(-1-q) <= u <= exp(-q).  Working in s or u
    keeps full precision next to the branch point z = -1/e, where z itself
    cannot be represented well."""
    if q <= 0.0:
        return -1.0
    if q <= 0.5:
        lo = math.sqrt(q * q + 2.0 * q) - q
        hi = min(math.sqrt(2.0 * q), 1.0)
        s = _bisect(_phi_s, lo, hi, q, increasing=True)
        return -(1.0 - s)
    lo, hi = math.exp(-1.0 - q), min(1.0, math.exp(-q))
    u = _bisect(lambda u: u - 1.0 - math.log(u), lo, hi, q, increasing=False)
    return -u


def iewpf_scalars(c, gamma, zeta, N_psi, only=None):
    """Target weight, beta, c* and alpha of the two-stage IEWPF
    (App. A: eqs. cistarTwoStage, betaTwoStage, iewpfAlphaSol).
    only: indices whose alpha is solved (all when None; the others are NaN),
    for large ensembles checked on samples.

    Returns dict with cbar, beta, cstar[i], alpha[i], neglogw[i]."""
    c = np.asarray(c, np.float64)
    gamma = np.asarray(gamma, np.float64)
    zeta = np.asarray(zeta, np.float64)
    ne = len(c)
    cbar = float(np.sum(c) / ne)                     # w_target = mean c_i
    beta = float(np.min((cbar - c) / zeta + 1.0))    # eq. betaTwoStage
    cstar = cbar - c - (beta - 1.0) * zeta           # eq. cistarTwoStage
    alpha = np.full(ne, np.nan)
    for i in (range(ne) if only is None else only):
        x = gamma[i] / N_psi
        # W_0 argument -x e^{-x} e^{-c*/N} = -exp(-1 - q)
        q = ((x - 1.0) - math.log1p(x - 1.0)) + max(cstar[i], 0.0) / N_psi
        w = lambert_w0_branch(q)
        alpha[i] = -w / x                            # eq. iewpfAlphaSol
    neglogw = (alpha - 1.0) * gamma - N_psi * np.log(alpha) + (beta - 1.0) * zeta + c
    return {"cbar": cbar, "beta": beta, "cstar": cstar, "alpha": alpha, "neglogw": neglogw}


def iewpf_scalars_one_stage(c, gamma, N_psi):
    """Target weight, c* and alpha of the one-stage IEWPF (App. A: eqs.
    iewpf_targetWeight, iewpfCStar, iewpfAlphaSol).  There is no nu, so no
    beta; beta is returned as 0, which removes the nu term from the
    posterior of eq. optUpdateEquationTwoStage.

    Returns dict with w_target, cbar (mean c_i), beta, cstar[i], alpha[i],
    neglogw[i]."""
    c = np.asarray(c, np.float64)
    gamma = np.asarray(gamma, np.float64)
    ne = len(c)
    w_target = float(np.max(c))                      # eq. iewpf_targetWeight
    cstar = w_target - c                             # eq. iewpfCStar
    alpha = np.empty(ne)
    for i in range(ne):
        x = gamma[i] / N_psi
        q = ((x - 1.0) - math.log1p(x - 1.0)) + cstar[i] / N_psi
        alpha[i] = -lambert_w0_branch(q) / x         # eq. iewpfAlphaSol
    # eq. implicitEquation without the derivative term (the large-N_psi form
    # that eq. iewpfAlphaSol solves)
    neglogw = (alpha - 1.0) * gamma - N_psi * np.log(alpha) + c
    return {"w_target": w_target, "cbar": float(np.sum(c) / ne), "beta": 0.0, "cstar": cstar,
            "alpha": alpha, "neglogw": neglogw}


def log_gamma_p(s, x):
    """log P(s, x), P the regularised lower incomplete gamma function, from
    its power series (Abramowitz & Stegun 6.5.4 with 6.5.29):
        P(s, x) = x^s e^{-x} / Gamma(s + 1) * sum_{n>=0} x^n / ((s+1)...(s+n)),
    the terms formed by a running product and summed in FP64 (numpy's
    pairwise sum) until they fall below 1e-17 of the sum.  Beyond
    x = s + 30 sqrt(s) + 30 the upper function is below 1e-190 and log P is
    0 to FP64 precision."""
    if x <= 0.0:
        return -math.inf
    if x > s + 30.0 * math.sqrt(s) + 30.0:
        return 0.0
    n = int(max(x - s, 0.0) + 40.0 * math.sqrt(max(s, 1.0)) + 100.0)
    while True:
        terms = np.cumprod(x / (s + np.arange(1, n + 1, dtype=np.float64)))
        total = 1.0 + float(np.sum(terms))
        if terms[-1] < 1e-17 * total:
            break
        n *= 2
    return s * math.log(x) - x - math.lgamma(s + 1.0) + math.log(total)


def alpha_incomplete_gamma(gamma, cstar, N_psi):
    """alpha of the one-stage IEWPF from eq. numericalEqForAlpha (App. A):
    the lower incomplete gamma function at (N_psi/2, alpha gamma/2) equals
    exp(-c*/2) times its value at (N_psi/2, gamma/2); the ratio is the same
    for the regularised form P.  Solved in logarithms (log_gamma_p), by
    bisection on alpha in (0, 1] where log P(s, alpha gamma/2) is increasing."""
    s = 0.5 * N_psi
    out = np.empty(len(gamma))
    for i, (g, cs) in enumerate(zip(np.asarray(gamma, np.float64), np.asarray(cstar, np.float64))):
        if cs == 0.0:
            out[i] = 1.0
            continue
        target = log_gamma_p(s, 0.5 * g) - 0.5 * cs
        f = lambda a: log_gamma_p(s, 0.5 * a * g) - target
        # bracket [lo, hi] from alpha = 1 downwards, f(lo) < 0 <= f(hi)
        step, hi, lo = 1e-9, 1.0, 1.0 - 1e-9
        while f(lo) >= 0.0:
            hi = lo
            step *= 2.0
            lo = max(1.0 - step, 0.5 * lo) if step < 1.0 else 0.5 * lo
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if mid <= lo or mid >= hi:
                break
            if f(mid) < 0.0:
                lo = mid
            else:
                hi = mid
        out[i] = 0.5 * (lo + hi)
    return out


def rand_vectors(P: Problem, ne, t, p0=0):
    """xi, nu~ ~ N(0, I) on Omega^R (streams 1 and 2, draw t), the
    perpendicular nu (eq. nuPerpendicular) and gamma, zeta (eq.
    scalingGammaZeta).  Returns dict of arrays."""
    NR = P.N_R
    xi = np.stack([normals(P.seed, p0 + i, t, STREAM_XI, NR) for i in range(ne)])
    nut = np.stack([normals(P.seed, p0 + i, t, STREAM_NU, NR) for i in range(ne)])
    xx = np.einsum("ij,ij->i", xi, xi)
    nn = np.einsum("ij,ij->i", nut, nut)
    nx_ = np.einsum("ij,ij->i", nut, xi)
    a = nx_ / xx
    scale = np.sqrt(nn / (nn - a * nx_))
    nu = scale[:, None] * (nut - a[:, None] * xi)
    gamma = xx * P.N_psi / NR
    zeta = nn * P.N_psi / NR
    return {"xi": xi, "nut": nut, "nu": nu, "xx": xx, "nn": nn, "nx": nx_,
            "a": a, "gamma": gamma, "zeta": zeta}


def innovations(P: Problem, ens, cells, y):
    ens = np.ascontiguousarray(ens, np.float64)
    ne = ens.shape[0]
    cells = np.ascontiguousarray(cells, np.int32).reshape(-1, 2)
    y = np.ascontiguousarray(y, np.float64).reshape(-1, 2)
    d = np.empty((ne, len(cells), 2))
    s = P.swe()
    lib().orc_innovations(ctypes.byref(s), ne, _d(ens), len(cells), _i(cells), _d(y), _d(d))
    return d


def add_pull(P: Problem, K, cells, Sd, U):
    K = np.ascontiguousarray(K, np.float64)
    cells = np.ascontiguousarray(cells, np.int32).reshape(-1, 2)
    Sd = np.ascontiguousarray(Sd, np.float64).reshape(-1, 2)
    U = np.array(U, np.float64, order="C")
    s = P.swe()
    lib().orc_add_pull(ctypes.byref(s), stencil_radius(P), _d(K), len(cells), _i(cells),
                       _d(Sd), _d(U))
    return U


def block_indices(P: Problem, cell):
    """Coarse-grid linear indices of the 7x7 block around the coarse point
    nearest to an observed cell (Sec. 4.6), ordered (dy+3)*7 + (dx+3)."""
    a0 = nearest_coarse(P.nx, P.nRx, P.c_omega, cell[0])
    b0 = nearest_coarse(P.ny, P.nRy, P.c_omega, cell[1])
    return np.array([((b0 + q) % P.nRy) * P.nRx + (a0 + p) % P.nRx
                     for q in range(-3, 4) for p in range(-3, 4)])


def assimilate(P: Problem, ens, cells, y, t, dense=True, K=None, Msq=None, p0=0, one_stage=False, scalars=None):
    """One two-stage IEWPF analysis of the forecast ensemble (Sec. 4, steps
    1-6), or with one_stage=True the one-stage IEWPF of App. A (eq.
    iewpfUpdateAgain: the same steps without nu).  scalars: the ensemble-wide
    step's results (dict with beta and alpha for these particles) taken as
    given instead of computed from this ensemble, so that particles of a
    large ensemble can be updated one by one (particle ids p0, p0 + 1, ...).
    Returns (new ensemble, diagnostics dict)."""
    ens = np.array(ens, np.float64, order="C")
    ne = ens.shape[0]
    cells = [tuple(int(v) for v in cl) for cl in cells]
    if K is None:
        K = pull_stencil(P)
    if Msq is None:
        Msq = local_block_sqrt(P)
    # 1-2: innovations, S d and phi (eqs. etaCompensatedInnovation, iewpfPhi)
    d = innovations(P, ens, cells, y).reshape(ne, -1)
    A = s_matrix(P, K, cells, dense)
    Sd = cholesky_solve(A, d.T).T
    phi = np.einsum("ij,ij->i", d, Sd)
    c = phi + math.log(ne)                 # eq. iewpf_ci with w^{n-1} = 1/N_e
    # 3: perpendicular random vectors
    rv = rand_vectors(P, ne, t, p0)
    # 4-5: target weight, beta, alpha
    if scalars is not None:
        sc = {"beta": float(scalars["beta"]), "alpha": np.asarray(scalars["alpha"], np.float64)}
        r = math.sqrt(sc["beta"]) * rv["nu"] + np.sqrt(sc["alpha"])[:, None] * rv["xi"]
    elif one_stage:
        sc = iewpf_scalars_one_stage(c, rv["gamma"], P.N_psi)
        # 6: posterior (eq. iewpfUpdateAgain): psi^a + P^{1/2} a^.5 xi
        r = np.sqrt(sc["alpha"])[:, None] * rv["xi"]
    else:
        sc = iewpf_scalars(c, rv["gamma"], rv["zeta"], P.N_psi)
        # 6: posterior (eq. optUpdateEquationTwoStage): psi^a + P^{1/2}(b^.5 nu + a^.5 xi)
        r = math.sqrt(sc["beta"]) * rv["nu"] + np.sqrt(sc["alpha"])[:, None] * rv["xi"]
    for cl in cells:                       # U Sigma^{1/2} on each 7x7 block, in order
        idx = block_indices(P, cl)
        r[:, idx] = r[:, idx] @ Msq.T
    for i in range(ne):
        ens[i] = add_pull(P, K, cells, Sd[i].reshape(-1, 2), ens[i])
        ens[i] = add_qhalf(P, r[i], ens[i])
    diag = {"d": d, "Sd": Sd, "phi": phi, "c": c, "r": r, **rv, **sc}
    return ens, diag


def drifter_observation(P: Problem, xy, xy_prev, dt):
    """eq. drifterObservation without its observation error: the drifter
    velocity estimated from two fixes dt seconds apart times H_eq, the
    displacement taken by the minimum image on the periodic domain."""
    xy = np.asarray(xy, np.float64).reshape(-1, 2)
    xy_prev = np.asarray(xy_prev, np.float64).reshape(-1, 2)
    out = np.empty_like(xy)
    for d in range(len(xy)):
        for k, L in enumerate((P.nx * P.dx, P.ny * P.dy)):
            disp = math.fmod(xy[d, k] - xy_prev[d, k], L)
            if disp > 0.5 * L:
                disp -= L
            if disp < -0.5 * L:
                disp += L
            out[d, k] = disp / dt * P.H
    return out


def sir_weights(d, sets, sigma2, r_scale=1.0):
    """Normalised weights of the standard particle filter (Sec. 2.1, eqs.
    standardParticleFilter, standardParticleFilterWeight) for each subset of
    observations, R = r_scale sigma2 I, and the number of particles whose
    weight exceeds 1/N_e (kept for sure by residual resampling, Sec. 5.3).

    d: innovations [N_e][n_obs][2]; sets: [n_sets][set_size] indices.
    Returns (w [n_sets][N_e], kept [n_sets]).  exp(-l_i) is divided by
    exp(-min_j l_j) before the normalisation, which changes nothing but keeps
    the largest term at 1 instead of underflowing."""
    d = np.asarray(d, np.float64)
    ne = d.shape[0]
    sets = np.asarray(sets)
    w = np.empty((len(sets), ne))
    kept = np.empty(len(sets), np.int64)
    for s, S in enumerate(sets):
        l = np.array([0.5 * sum(d[i, k, 0] ** 2 + d[i, k, 1] ** 2 for k in S) / (r_scale * sigma2)
                      for i in range(ne)])
        e = np.exp(-(l - l.min()))
        w[s] = e / e.sum()
        kept[s] = int(np.sum(w[s] > 1.0 / ne))
    return w, kept


def ranks(P: Problem, ens, cells, y, t, p0=0):
    """Rank of each observed value within the ensemble (Sec. 5.1): members'
    hu (comp 0) or hv (comp 1) at the cell plus the observation error
    obs_sigma eps, eps the normal number 2m + comp of the particle's stream
    STREAM_RANK (draw t); the rank is the number of perturbed members below
    the observed value, i.e. its insertion position in their sorted list.
    cells [n][2] integer (j, k); y [n][2].  Returns int array [n][2]."""
    ens = np.asarray(ens, np.float64)
    ne = ens.shape[0]
    cells = np.asarray(cells).reshape(-1, 2)
    y = np.asarray(y, np.float64).reshape(-1, 2)
    eps = np.stack([normals(P.seed, p0 + i, t, STREAM_RANK, 2 * len(cells)) for i in range(ne)])
    out = np.zeros((len(cells), 2), np.int64)
    for m, (j, k) in enumerate(cells):
        for comp in (0, 1):
            below = 0
            for i in range(ne):
                if ens[i, 1 + comp, k, j] + P.obs_sigma * eps[i, 2 * m + comp] < y[m, comp]:
                    below += 1
            out[m, comp] = below
    return out


def forecast_errors(traj, truth):
    """Drift-forecast error E(t) and RMSE(t) (eqs. errorPerEnsembleDrifter,
    errorNorm).  traj: [n_out][N_e][N_D][2] unwrapped positions; truth:
    [n_out][N_D][2].  RMSE uses the ensemble mean in place of the truth."""
    traj = np.asarray(traj, np.float64)
    truth = np.asarray(truth, np.float64)
    Ed = np.mean(np.sum((traj - truth[:, None]) ** 2, axis=-1), axis=1)   # [n_out][N_D]
    E = np.sqrt(np.mean(Ed, axis=1))
    mean = np.mean(traj, axis=1)
    Rd = np.mean(np.sum((traj - mean[:, None]) ** 2, axis=-1), axis=1)
    RMSE = np.sqrt(np.mean(Rd, axis=1))
    return E, RMSE
