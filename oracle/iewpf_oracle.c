/*
 * FP64 CPU oracle for the IEWPF hot path (test infrastructure only).
 *
 * This file is test infrastructure.  Only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline leg may load it.  It shares no code with the CUDA
 * path under paper_1910_01031_gb300/csrc: both are written independently from
 * the paper (arXiv 1910.01031).
 *
 * Everything here is plain loops in double precision, in the order the paper
 * states the operations.  OpenMP is used only to run independent particles on
 * separate cores; it changes no arithmetic.
 *
 * Array conventions: a field is [ny][nx] with x (index j) fastest; a state is
 * [3][ny][nx] holding (eta, hu, hv); an ensemble is [Ne][3][ny][nx].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    int nx, ny;
    double dx, dy;
    double g, f, H;      /* gravity, Coriolis parameter, equilibrium depth */
    double theta;        /* generalized-minmod parameter of the reconstruction */
} orc_swe_t;

typedef struct {
    int c;               /* coarsening factor c_Omega (odd) */
    int nRx, nRy;        /* points of the coarse grid Omega^R per axis */
    double q0, L0;       /* SOAR amplitude and length scale (metres) */
} orc_err_t;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Ten rounds of the     */
/* multiply-xor round function; the key is bumped by the Weyl constants      */
/* between rounds.                                                           */
/* ------------------------------------------------------------------------ */
void orc_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint64_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = M0 * (uint64_t)c0;
        uint64_t p1 = M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Standard normals for random-number stream `stream` of particle `p` at draw
 * step `t`.  Normal number m comes from Philox block m/4 with counter
 * (m/4, p, t, stream); the four 32-bit words form two Box-Muller pairs
 * (words 0,1 and words 2,3): z_even = r cos(theta), z_odd = r sin(theta),
 * r = sqrt(-2 ln u_a), theta = 2 pi u_b, u = (k + 1/2) 2^-32. */
void orc_normals(uint64_t seed, uint32_t p, uint32_t t, uint32_t stream,
                 long n, double* z)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (long blk = 0; 4 * blk < n; ++blk) {
        uint32_t ctr[4] = {(uint32_t)blk, p, t, stream};
        uint32_t w[4];
        orc_philox(ctr, key, w);
        double zz[4];
        for (int pair = 0; pair < 2; ++pair) {
            double ua = ((double)w[2 * pair] + 0.5) * 0x1p-32;
            double ub = ((double)w[2 * pair + 1] + 0.5) * 0x1p-32;
            double r = sqrt(-2.0 * log(ua));
            double th = 2.0 * M_PI * ub;
            zz[2 * pair] = r * cos(th);
            zz[2 * pair + 1] = r * sin(th);
        }
        for (int l = 0; l < 4 && 4 * blk + l < n; ++l) z[4 * blk + l] = zz[l];
    }
}

/* ------------------------------------------------------------------------ */
/* Rotating shallow-water stepper (Sec. 3.1, eqs. swe_full, swecfl).        */
/* Central-upwind fluxes (Kurganov-Petrova form) for mass and normal        */
/* momentum, tangential momentum carried by the mass flux with the upwind   */
/* tangential velocity, and a reconstruction of eta through the Coriolis-   */
/* adjusted potential K = g eta - f V (V_x = v), limited by the generalized */
/* minmod, so that a jet in discrete geostrophic balance (Sec. 3.1,         */
/* eq. geostrophic_balance_cont) has continuous face values.                */
/* ------------------------------------------------------------------------ */
static inline int wrap(int i, int n) { i %= n; return i < 0 ? i + n : i; }

static double minmod3(double a, double b, double c)
{
    if (a > 0.0 && b > 0.0 && c > 0.0) return fmin(a, fmin(b, c));
    if (a < 0.0 && b < 0.0 && c < 0.0) return fmax(a, fmax(b, c));
    return 0.0;
}

/* generalized minmod of the backward and forward differences */
static double gminmod(double back, double fwd, double theta)
{
    return minmod3(theta * back, 0.5 * (back + fwd), theta * fwd);
}

/* eta-part of the hydrostatic pressure g h^2/2 with the constant g H^2/2
 * removed (constant fluxes cancel in every flux difference) */
static double pressure(double eta, double g, double H)
{
    return g * eta * (H + 0.5 * eta);
}

/* Right-hand side L(U) of U_t = L(U), U = (eta, hu, hv) */
void orc_swe_rhs(const orc_swe_t* P, const double* U, double* L)
{
    const int nx = P->nx, ny = P->ny;
    const long N = (long)nx * ny;
    const double g = P->g, f = P->f, H = P->H, dx = P->dx, dy = P->dy, th = P->theta;
    const double* eta = U;
    const double* hu = U + N;
    const double* hv = U + 2 * N;
    double* u = malloc(sizeof(double) * N);
    double* v = malloc(sizeof(double) * N);
    /* face values: E, W, N, S of eta, hu, hv */
    double* eE = malloc(sizeof(double) * N); double* eW = malloc(sizeof(double) * N);
    double* eN = malloc(sizeof(double) * N); double* eS = malloc(sizeof(double) * N);
    double* uE = malloc(sizeof(double) * N); double* uW = malloc(sizeof(double) * N);
    double* uN = malloc(sizeof(double) * N); double* uS = malloc(sizeof(double) * N);
    double* vE = malloc(sizeof(double) * N); double* vW = malloc(sizeof(double) * N);
    double* vN = malloc(sizeof(double) * N); double* vS = malloc(sizeof(double) * N);
    double* Fx = malloc(sizeof(double) * 3 * N);   /* flux at x-face j+1/2 of cell (j,k) */
    double* Gy = malloc(sizeof(double) * 3 * N);   /* flux at y-face k+1/2 of cell (j,k) */

    /* 1. cell velocities */
    for (long i = 0; i < N; ++i) {
        double h = H + eta[i];
        u[i] = hu[i] / h;
        v[i] = hv[i] / h;
    }
    /* 2. reconstruction */
    for (int k = 0; k < ny; ++k) {
        for (int j = 0; j < nx; ++j) {
            long c = (long)k * nx + j;
            long cw = (long)k * nx + wrap(j - 1, nx), ce = (long)k * nx + wrap(j + 1, nx);
            long cs = (long)wrap(k - 1, ny) * nx + j, cn = (long)wrap(k + 1, ny) * nx + j;
            /* x: Coriolis-adjusted potential K differences at faces j-1/2, j+1/2 */
            double dKw = g * (eta[c] - eta[cw]) - 0.5 * f * dx * (v[cw] + v[c]);
            double dKe = g * (eta[ce] - eta[c]) - 0.5 * f * dx * (v[c] + v[ce]);
            double sK = gminmod(dKw, dKe, th);
            double ex = (sK + f * dx * v[c]) / (2.0 * g);
            eE[c] = eta[c] + ex;
            eW[c] = eta[c] - ex;
            double shu = gminmod(hu[c] - hu[cw], hu[ce] - hu[c], th);
            double shv = gminmod(hv[c] - hv[cw], hv[ce] - hv[c], th);
            uE[c] = hu[c] + 0.5 * shu; uW[c] = hu[c] - 0.5 * shu;
            vE[c] = hv[c] + 0.5 * shv; vW[c] = hv[c] - 0.5 * shv;
            /* y: potential L differences at faces k-1/2, k+1/2 */
            double dLs = g * (eta[c] - eta[cs]) + 0.5 * f * dy * (u[cs] + u[c]);
            double dLn = g * (eta[cn] - eta[c]) + 0.5 * f * dy * (u[c] + u[cn]);
            double sL = gminmod(dLs, dLn, th);
            double ey = (sL - f * dy * u[c]) / (2.0 * g);
            eN[c] = eta[c] + ey;
            eS[c] = eta[c] - ey;
            double suy = gminmod(hu[c] - hu[cs], hu[cn] - hu[c], th);
            double svy = gminmod(hv[c] - hv[cs], hv[cn] - hv[c], th);
            uN[c] = hu[c] + 0.5 * suy; uS[c] = hu[c] - 0.5 * suy;
            vN[c] = hv[c] + 0.5 * svy; vS[c] = hv[c] - 0.5 * svy;
        }
    }
    /* 3. central-upwind fluxes */
    for (int k = 0; k < ny; ++k) {
        for (int j = 0; j < nx; ++j) {
            long c = (long)k * nx + j;
            /* x-face between (j,k) [left] and (j+1,k) [right] */
            {
                long r = (long)k * nx + wrap(j + 1, nx);
                double etaL = eE[c], huL = uE[c], hvL = vE[c];
                double etaR = eW[r], huR = uW[r], hvR = vW[r];
                double hL = H + etaL, hR = H + etaR;
                double ul = huL / hL, ur = huR / hR;
                double cl = sqrt(g * hL), cr = sqrt(g * hR);
                double ap = fmax(fmax(ul + cl, ur + cr), 0.0);
                double am = fmin(fmin(ul - cl, ur - cr), 0.0);
                double Fe = (ap * huL - am * huR + ap * am * (etaR - etaL)) / (ap - am);
                double Fu = (ap * (huL * ul + pressure(etaL, g, H))
                             - am * (huR * ur + pressure(etaR, g, H))
                             + ap * am * (huR - huL)) / (ap - am);
                double vup = (Fe >= 0.0) ? hvL / hL : hvR / hR;
                Fx[c] = Fe;
                Fx[N + c] = Fu;
                Fx[2 * N + c] = Fe * vup;
            }
            /* y-face between (j,k) [bottom] and (j,k+1) [top] */
            {
                long r = (long)wrap(k + 1, ny) * nx + j;
                double etaB = eN[c], huB = uN[c], hvB = vN[c];
                double etaT = eS[r], huT = uS[r], hvT = vS[r];
                double hB = H + etaB, hT = H + etaT;
                double vb = hvB / hB, vt = hvT / hT;
                double cb = sqrt(g * hB), ct = sqrt(g * hT);
                double ap = fmax(fmax(vb + cb, vt + ct), 0.0);
                double am = fmin(fmin(vb - cb, vt - ct), 0.0);
                double Ge = (ap * hvB - am * hvT + ap * am * (etaT - etaB)) / (ap - am);
                double Gv = (ap * (hvB * vb + pressure(etaB, g, H))
                             - am * (hvT * vt + pressure(etaT, g, H))
                             + ap * am * (hvT - hvB)) / (ap - am);
                double uup = (Ge >= 0.0) ? huB / hB : huT / hT;
                Gy[c] = Ge;
                Gy[N + c] = Ge * uup;
                Gy[2 * N + c] = Gv;
            }
        }
    }
    /* 4. flux differences and Coriolis source (f hv, -f hu) */
    for (int k = 0; k < ny; ++k) {
        for (int j = 0; j < nx; ++j) {
            long c = (long)k * nx + j;
            long cw = (long)k * nx + wrap(j - 1, nx);
            long cs = (long)wrap(k - 1, ny) * nx + j;
            for (int q = 0; q < 3; ++q) {
                L[q * N + c] = -(Fx[q * N + c] - Fx[q * N + cw]) / dx
                               - (Gy[q * N + c] - Gy[q * N + cs]) / dy;
            }
            L[N + c] += f * hv[c];
            L[2 * N + c] -= f * hu[c];
        }
    }
    free(u); free(v);
    free(eE); free(eW); free(eN); free(eS);
    free(uE); free(uW); free(uN); free(uS);
    free(vE); free(vW); free(vN); free(vS);
    free(Fx); free(Gy);
}

/* One step of the second-order strong-stability-preserving Runge-Kutta
 * method (Heun form, Sec. 3.1): U1 = U + dt L(U); U <- (U + U1 + dt L(U1))/2 */
void orc_swe_substep(const orc_swe_t* P, double dt, double* U)
{
    const long n3 = 3L * P->nx * P->ny;
    double* L = malloc(sizeof(double) * n3);
    double* U1 = malloc(sizeof(double) * n3);
    orc_swe_rhs(P, U, L);
    for (long i = 0; i < n3; ++i) U1[i] = U[i] + dt * L[i];
    orc_swe_rhs(P, U1, L);
    for (long i = 0; i < n3; ++i) U[i] = 0.5 * (U[i] + (U1[i] + dt * L[i]));
    free(L); free(U1);
}

/* CFL-limited step (eq. swecfl) scaled by the Courant number */
double orc_cfl_dt(const orc_swe_t* P, const double* U, double courant)
{
    const long N = (long)P->nx * P->ny;
    double ax = 0.0, ay = 0.0;
    for (long i = 0; i < N; ++i) {
        double h = P->H + U[i];
        double c = sqrt(P->g * h);
        double u = U[N + i] / h, v = U[2 * N + i] / h;
        ax = fmax(ax, fabs(u) + c);
        ay = fmax(ay, fabs(v) + c);
    }
    return courant * 0.25 * fmin(P->dx / ax, P->dy / ay);
}

/* Number of scheme steps that subdivide one model step dt_model */
int orc_n_sub(const orc_swe_t* P, const double* U, double courant, double dt_model)
{
    double dtc = orc_cfl_dt(P, U, courant);
    int n = (int)ceil(dt_model / dtc);
    return n < 1 ? 1 : n;
}

/* ------------------------------------------------------------------------ */
/* Model error Q^{1/2} = Q_GB^{1/2} I_Omega Q_SOAR^{1/2} (Sec. 3.2)          */
/* ------------------------------------------------------------------------ */

/* Number of coarse points on an axis of n fine cells: points at fine index
 * o + c a, o = floor(c/2), while that index is inside the domain. */
int orc_coarse_n(int n, int c)
{
    int o = c / 2;
    return (n - 1 - o) / c + 1;
}

/* fine index of coarse point a (any integer) in the periodic extension */
static long coarse_pos(long a, int nR, int c, int n)
{
    long w = a >= 0 ? a / nR : -((-a + nR - 1) / nR);
    long am = a - w * nR;
    return (long)(c / 2) + (long)c * am + w * (long)n;
}

/* SOAR kernel value (eq. soar_function) */
static double soar_w(double d, double q0, double L0)
{
    return q0 * (1.0 + d / L0) * exp(-d / L0);
}

/* Q_SOAR^{1/2} on the coarse grid with cut-off c_SOAR = 2 (eq.
 * local_soar_on_eta): a full 5x5 block of neighbours, distances measured
 * between the actual positions of the coarse points in metres. */
void orc_soar(const orc_swe_t* P, const orc_err_t* E, const double* xi, double* out)
{
    const int nRx = E->nRx, nRy = E->nRy, c = E->c;
    for (int b = 0; b < nRy; ++b) {
        for (int a = 0; a < nRx; ++a) {
            double acc = 0.0;
            for (int db = -2; db <= 2; ++db) {
                for (int da = -2; da <= 2; ++da) {
                    double DX = (double)(coarse_pos(a + da, nRx, c, P->nx) - coarse_pos(a, nRx, c, P->nx)) * P->dx;
                    double DY = (double)(coarse_pos(b + db, nRy, c, P->ny) - coarse_pos(b, nRy, c, P->ny)) * P->dy;
                    double d = sqrt(DX * DX + DY * DY);
                    acc += soar_w(d, E->q0, E->L0) * xi[(long)wrap(b + db, nRy) * nRx + wrap(a + da, nRx)];
                }
            }
            out[(long)b * nRx + a] = acc;
        }
    }
}

/* Catmull-Rom (Keys a = -1/2) cubic convolution weights for taps
 * a-1, a, a+1, a+2 at local coordinate t in [0,1) */
static void cubic_w(double t, double w[4])
{
    double t2 = t * t, t3 = t2 * t;
    w[0] = 0.5 * (-t3 + 2.0 * t2 - t);
    w[1] = 0.5 * (3.0 * t3 - 5.0 * t2 + 2.0);
    w[2] = 0.5 * (-3.0 * t3 + 4.0 * t2 + t);
    w[3] = 0.5 * (t3 - t2);
}

/* coarse interval holding fine index j and the local coordinate there */
static void coarse_interval(int j, int n, int nR, int c, long* a, double* t)
{
    int o = c / 2;
    long aa;
    if (j < o) aa = -1;
    else {
        aa = (j - o) / c;
        if (aa > nR - 1) aa = nR - 1;
    }
    long x0 = coarse_pos(aa, nR, c, n), x1 = coarse_pos(aa + 1, nR, c, n);
    *a = aa;
    *t = (double)(j - x0) / (double)(x1 - x0);
}

/* Bicubic interpolation I_Omega: Omega^R -> Omega^M, pointwise at the fine
 * cell centres, tensor product of the 1D cubic convolution */
void orc_bicubic(const orc_swe_t* P, const orc_err_t* E, const double* coarse, double* fine)
{
    const int nx = P->nx, ny = P->ny, nRx = E->nRx, nRy = E->nRy, c = E->c;
    for (int k = 0; k < ny; ++k) {
        long b; double ty, wy[4];
        coarse_interval(k, ny, nRy, c, &b, &ty);
        cubic_w(ty, wy);
        for (int j = 0; j < nx; ++j) {
            long a; double tx, wx[4];
            coarse_interval(j, nx, nRx, c, &a, &tx);
            cubic_w(tx, wx);
            double acc = 0.0;
            for (int q = 0; q < 4; ++q) {
                for (int p = 0; p < 4; ++p) {
                    acc += wy[q] * wx[p] * coarse[(long)wrap((int)(b - 1 + q), nRy) * nRx + wrap((int)(a - 1 + p), nRx)];
                }
            }
            fine[(long)k * nx + j] = acc;
        }
    }
}

/* Q_GB^{1/2}: momentum in geostrophic balance with eta by central
 * differences on the fine grid (eq. geostrophic_balance_disc) */
void orc_gb(const orc_swe_t* P, const double* deta, double* dhu, double* dhv)
{
    const int nx = P->nx, ny = P->ny;
    const double s = P->g * P->H / P->f;
    for (int k = 0; k < ny; ++k) {
        for (int j = 0; j < nx; ++j) {
            long c = (long)k * nx + j;
            double en = deta[(long)wrap(k + 1, ny) * nx + j], es = deta[(long)wrap(k - 1, ny) * nx + j];
            double ee = deta[(long)k * nx + wrap(j + 1, nx)], ew = deta[(long)k * nx + wrap(j - 1, nx)];
            dhu[c] = -s * (en - es) / (2.0 * P->dy);
            dhv[c] = s * (ee - ew) / (2.0 * P->dx);
        }
    }
}

/* dU += Q^{1/2} x for a coarse field x (eqs. model_error,
 * covarianceOperatorsDef) */
void orc_add_qhalf(const orc_swe_t* P, const orc_err_t* E, const double* x, double* U)
{
    const long N = (long)P->nx * P->ny, NR = (long)E->nRx * E->nRy;
    double* s = malloc(sizeof(double) * NR);
    double* deta = malloc(sizeof(double) * N);
    double* dhu = malloc(sizeof(double) * N);
    double* dhv = malloc(sizeof(double) * N);
    orc_soar(P, E, x, s);
    orc_bicubic(P, E, s, deta);
    orc_gb(P, deta, dhu, dhv);
    for (long i = 0; i < N; ++i) {
        U[i] += deta[i];
        U[N + i] += dhu[i];
        U[2 * N + i] += dhv[i];
    }
    free(s); free(deta); free(dhu); free(dhv);
}

/* psi += Q^{1/2} xi with xi ~ N(0, I) from stream 0 of particle p, draw t */
void orc_model_error(const orc_swe_t* P, const orc_err_t* E, uint64_t seed,
                     uint32_t p, uint32_t t, double* U)
{
    const long NR = (long)E->nRx * E->nRy;
    double* xi = malloc(sizeof(double) * NR);
    orc_normals(seed, p, t, 0u, NR, xi);
    orc_add_qhalf(P, E, xi, U);
    free(xi);
}

/* ------------------------------------------------------------------------ */
/* Drifters: forward Euler with the velocity of the containing cell         */
/* (Sec. 3.3).  Positions are kept unwrapped; the cell is found modulo the  */
/* domain.                                                                   */
/* ------------------------------------------------------------------------ */
static void cell_of(const orc_swe_t* P, double x, double y, int* j, int* k)
{
    *j = wrap((int)floor(x / P->dx), P->nx);
    *k = wrap((int)floor(y / P->dy), P->ny);
}

void orc_drift(const orc_swe_t* P, const double* U, double dt, int nd, double* xy)
{
    const long N = (long)P->nx * P->ny;
    for (int d = 0; d < nd; ++d) {
        int j, k;
        cell_of(P, xy[2 * d], xy[2 * d + 1], &j, &k);
        long c = (long)k * P->nx + j;
        double h = P->H + U[c];
        double u = U[N + c] / h, v = U[2 * N + c] / h;
        xy[2 * d] += dt * u;
        xy[2 * d + 1] += dt * v;
    }
}

/* ------------------------------------------------------------------------ */
/* Ensemble forecast: for each model step, choose the scheme step from the  */
/* CFL condition, run the substeps (advecting drifters after each), then    */
/* add the model error if requested.                                        */
/* ------------------------------------------------------------------------ */
void orc_forecast(const orc_swe_t* P, const orc_err_t* E, uint64_t seed, int ne,
                  double* ens, int n_steps, const int* add_err, uint32_t t0,
                  double courant, double dt_model, int nd, double* xy,
                  int* n_sub_out, int fixed_n_sub)
{
    const long n3 = 3L * P->nx * P->ny;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < ne; ++i) {
        double* U = ens + (long)i * n3;
        for (int s = 0; s < n_steps; ++s) {
            int nsub = fixed_n_sub > 0 ? fixed_n_sub : orc_n_sub(P, U, courant, dt_model);
            if (n_sub_out) n_sub_out[(long)i * n_steps + s] = nsub;
            double dts = dt_model / nsub;
            for (int q = 0; q < nsub; ++q) {
                orc_swe_substep(P, dts, U);
                if (nd > 0 && xy) orc_drift(P, U, dts, nd, xy + (long)i * 2 * nd);
            }
            if (add_err[s]) orc_model_error(P, E, seed, (uint32_t)i, t0 + (uint32_t)s, U);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* IEWPF pieces that touch the fine grid                                     */
/* ------------------------------------------------------------------------ */

/* eta-compensated innovations (eq. etaCompensatedInnovation):
 * d = y (H + eta)/H - (hu, hv) at the cell of each observation */
void orc_innovations(const orc_swe_t* P, int ne, const double* ens, int nobs,
                     const int* cells /*[nobs][2] = (j,k)*/, const double* y /*[nobs][2]*/,
                     double* d /*[ne][nobs][2]*/)
{
    const long N = (long)P->nx * P->ny;
    for (int i = 0; i < ne; ++i) {
        const double* U = ens + (long)i * 3 * N;
        for (int l = 0; l < nobs; ++l) {
            long c = (long)cells[2 * l + 1] * P->nx + cells[2 * l];
            double s = (P->H + U[c]) / P->H;
            d[((long)i * nobs + l) * 2 + 0] = y[2 * l] * s - U[N + c];
            d[((long)i * nobs + l) * 2 + 1] = y[2 * l + 1] * s - U[2 * N + c];
        }
    }
}

/* U += sum_l (Sd)_{l,hu} K_hu(. - cell_l) + (Sd)_{l,hv} K_hv(. - cell_l),
 * the optimal-proposal pull of eq. detailedOPDUpdate written with the
 * precomputed response K of the chain to a unit hu or hv observation.
 * K is [2][3][2R+1][2R+1] (component obs hu/hv, field eta/hu/hv, dy, dx). */
void orc_add_pull(const orc_swe_t* P, int R, const double* K, int nobs,
                  const int* cells, const double* Sd /*[nobs][2]*/, double* U)
{
    const long N = (long)P->nx * P->ny;
    const int W = 2 * R + 1;
    for (int l = 0; l < nobs; ++l) {
        for (int dyi = -R; dyi <= R; ++dyi) {
            for (int dxi = -R; dxi <= R; ++dxi) {
                int j = wrap(cells[2 * l] + dxi, P->nx), k = wrap(cells[2 * l + 1] + dyi, P->ny);
                long c = (long)k * P->nx + j;
                for (int fld = 0; fld < 3; ++fld) {
                    double kh = K[((0 * 3 + fld) * W + (dyi + R)) * W + (dxi + R)];
                    double kv = K[((1 * 3 + fld) * W + (dyi + R)) * W + (dxi + R)];
                    U[fld * N + c] += Sd[2 * l] * kh + Sd[2 * l + 1] * kv;
                }
            }
        }
    }
}
