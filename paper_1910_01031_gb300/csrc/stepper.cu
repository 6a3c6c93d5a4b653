// Shallow-water ensemble stepper (Sec. 3.1 of arXiv 1910.01031): one scheme
// step of the second-order SSP Runge-Kutta method with central-upwind fluxes
// and the Coriolis-adjusted (well-balanced) reconstruction of eta, both
// Runge-Kutta stages fused in one kernel on a shared-memory tile with a
// 4-cell halo; plus the per-particle CFL reduction (eq. swecfl), drifter
// advection and the state scan for non-finite values.
#include "common.cuh"
#include "kernels.h"

namespace iewpf {

namespace {

constexpr int HALO = 4;
constexpr int IW = TW + 2 * HALO;   // loaded tile width  (40)
constexpr int IH = TH + 2 * HALO;   // loaded tile height (24)
constexpr int S1W = TW + 4, S1H = TH + 4;   // stage-1 output region (36 x 20)

// shared-memory scratch sized for the larger (first) stage
constexpr int VEL_N = IW * IH;                    // u, v on the stage input
constexpr int SLP_N = (IW - 2) * (IH - 2);        // slopes on the inner ring
constexpr int FX_N = (S1W + 1) * S1H;             // x-face fluxes
constexpr int GY_N = S1W * (S1H + 1);             // y-face fluxes

struct Smem {
    float U0[3][IH][IW];
    float U1[3][S1H][S1W];
    float vel[2][VEL_N];
    float slp[6][SLP_N];
    float fx[3][FX_N];
    float gy[3][GY_N];
};

__device__ __forceinline__ float gminmod(float a, float b, float th)
{
    const float x = th * a, y = 0.5f * (a + b), z = th * b;
    const float mn = fminf(x, fminf(y, z));
    const float mx = fmaxf(x, fmaxf(y, z));
    return mn > 0.0f ? mn : (mx < 0.0f ? mx : 0.0f);
}

// Central-upwind flux across a face with left state L and right state R;
// qn is the momentum normal to the face, qt the tangential one.  Returns
// (mass, normal momentum, tangential momentum) fluxes.  The tangential
// momentum is carried by the mass flux with the upwind tangential velocity.
__device__ __forceinline__ void cu_flux(float etaL, float qnL, float qtL, float etaR, float qnR,
                                        float qtR, const Grid& G, float& F0, float& F1, float& F2)
{
    const float hL = G.H + etaL, hR = G.H + etaR;
    const float unL = qnL / hL, unR = qnR / hR;
    const float cL = sqrtf(G.g * hL), cR = sqrtf(G.g * hR);
    const float ap = fmaxf(fmaxf(unL + cL, unR + cR), 0.0f);
    const float am = fminf(fminf(unL - cL, unR - cR), 0.0f);
    const float inv = 1.0f / (ap - am);
    const float apam = ap * am;
    F0 = (ap * qnL - am * qnR + apam * (etaR - etaL)) * inv;
    const float pL = G.g * etaL * (G.H + 0.5f * etaL);
    const float pR = G.g * etaR * (G.H + 0.5f * etaR);
    F1 = (ap * (qnL * unL + pL) - am * (qnR * unR + pR) + apam * (qnR - qnL)) * inv;
    const float ut = (F0 >= 0.0f) ? qtL / hL : qtR / hR;
    F2 = F0 * ut;
}

// One evaluation of L(U) on an output region of RW x RH cells from an input
// array in[3][RH+4][RW+4] (2-cell halo); writes out(c, r, L0, L1, L2) for
// input-coordinates (c, r) in [2, RW+2) x [2, RH+2).
template <int RW, int RH, typename Out>
__device__ __forceinline__ void stage(const float* __restrict__ in, Smem& sm, const Grid& G, Out out)
{
    constexpr int W = RW + 4, Hh = RH + 4;
    constexpr int N = W * Hh;
    const int tid = threadIdx.x;
    const float* eta = in;
    const float* hu = in + N;
    const float* hv = in + 2 * N;
    float* u = sm.vel[0];
    float* v = sm.vel[1];
    // pass 0: velocities
    for (int i = tid; i < N; i += NTHREADS) {
        const float h = G.H + eta[i];
        u[i] = hu[i] / h;
        v[i] = hv[i] / h;
    }
    __syncthreads();
    // pass 1: limited slopes of K, hu, hv in x and of L, hu, hv in y
    constexpr int SW = W - 2, SH = Hh - 2;
    for (int i = tid; i < SW * SH; i += NTHREADS) {
        const int c = 1 + i % SW, r = 1 + i / SW;
        const int k = r * W + c;
        const int kw = k - 1, ke = k + 1, ks = k - W, kn = k + W;
        const float dKw = G.g * (eta[k] - eta[kw]) - G.fdx_half * (v[kw] + v[k]);
        const float dKe = G.g * (eta[ke] - eta[k]) - G.fdx_half * (v[k] + v[ke]);
        const float dLs = G.g * (eta[k] - eta[ks]) + G.fdy_half * (u[ks] + u[k]);
        const float dLn = G.g * (eta[kn] - eta[k]) + G.fdy_half * (u[k] + u[kn]);
        sm.slp[0][i] = gminmod(dKw, dKe, G.theta);
        sm.slp[1][i] = gminmod(hu[k] - hu[kw], hu[ke] - hu[k], G.theta);
        sm.slp[2][i] = gminmod(hv[k] - hv[kw], hv[ke] - hv[k], G.theta);
        sm.slp[3][i] = gminmod(dLs, dLn, G.theta);
        sm.slp[4][i] = gminmod(hu[k] - hu[ks], hu[kn] - hu[k], G.theta);
        sm.slp[5][i] = gminmod(hv[k] - hv[ks], hv[kn] - hv[k], G.theta);
    }
    __syncthreads();
    // pass 2a: x-faces between input columns c and c+1, c in [1, RW+2), rows [2, RH+2)
    constexpr int FXW = RW + 1;
    for (int i = tid; i < FXW * RH; i += NTHREADS) {
        const int c = 1 + i % FXW, r = 2 + i / FXW;
        const int kL = r * W + c, kR = kL + 1;
        const int sL = (r - 1) * SW + (c - 1), sR = sL + 1;
        const float eL = eta[kL] + (sm.slp[0][sL] + G.fdx * v[kL]) * G.inv_2g;
        const float eR = eta[kR] - (sm.slp[0][sR] + G.fdx * v[kR]) * G.inv_2g;
        const float quL = hu[kL] + 0.5f * sm.slp[1][sL], quR = hu[kR] - 0.5f * sm.slp[1][sR];
        const float qvL = hv[kL] + 0.5f * sm.slp[2][sL], qvR = hv[kR] - 0.5f * sm.slp[2][sR];
        float F0, F1, F2;
        cu_flux(eL, quL, qvL, eR, quR, qvR, G, F0, F1, F2);
        sm.fx[0][i] = F0;
        sm.fx[1][i] = F1;
        sm.fx[2][i] = F2;
    }
    // pass 2b: y-faces between input rows r and r+1, r in [1, RH+2), columns [2, RW+2)
    for (int i = tid; i < RW * (RH + 1); i += NTHREADS) {
        const int c = 2 + i % RW, r = 1 + i / RW;
        const int kB = r * W + c, kT = kB + W;
        const int sB = (r - 1) * SW + (c - 1), sT = sB + SW;
        const float eB = eta[kB] + (sm.slp[3][sB] - G.fdy * u[kB]) * G.inv_2g;
        const float eT = eta[kT] - (sm.slp[3][sT] - G.fdy * u[kT]) * G.inv_2g;
        const float quB = hu[kB] + 0.5f * sm.slp[4][sB], quT = hu[kT] - 0.5f * sm.slp[4][sT];
        const float qvB = hv[kB] + 0.5f * sm.slp[5][sB], qvT = hv[kT] - 0.5f * sm.slp[5][sT];
        float G0, Gv, Gu;
        cu_flux(eB, qvB, quB, eT, qvT, quT, G, G0, Gv, Gu);
        sm.gy[0][i] = G0;
        sm.gy[1][i] = Gu;
        sm.gy[2][i] = Gv;
    }
    __syncthreads();
    // pass 3: flux differences plus the Coriolis source (f hv, -f hu)
    for (int i = tid; i < RW * RH; i += NTHREADS) {
        const int c = 2 + i % RW, r = 2 + i / RW;
        const int k = r * W + c;
        const int fr = (r - 2) * FXW + (c - 1);      // right x-face; left is fr - 1
        const int gt = (r - 1) * RW + (c - 2);       // top y-face; bottom is gt - RW
        float L[3];
#pragma unroll
        for (int q = 0; q < 3; ++q)
            L[q] = -(sm.fx[q][fr] - sm.fx[q][fr - 1]) * G.inv_dx - (sm.gy[q][gt] - sm.gy[q][gt - RW]) * G.inv_dy;
        L[1] += G.f * hv[k];
        L[2] -= G.f * hu[k];
        out(c, r, L[0], L[1], L[2]);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(NTHREADS)
rk2_kernel(float* __restrict__ buf0, float* __restrict__ buf1, const int* __restrict__ par,
           const int* __restrict__ nsub, const float* __restrict__ dtp, int s, Grid G)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
    const int p = blockIdx.z;
    if (s >= nsub[p]) return;
    const int src = par[p] ^ (s & 1);
    const float* __restrict__ in = (src ? buf1 : buf0) + (long long)p * 3 * G.plane;
    float* __restrict__ outp = (src ? buf0 : buf1) + (long long)p * 3 * G.plane;
    const float dt = dtp[p];
    const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
    // load the tile with a 4-cell periodic halo
    for (int i = threadIdx.x; i < IW * IH; i += NTHREADS) {
        const int c = i % IW, r = i / IW;
        const int gx = pmod(x0 - HALO + c, G.nx), gy = pmod(y0 - HALO + r, G.ny);
        const long long g = (long long)gy * G.nx + gx;
        sm.U0[0][r][c] = in[g];
        sm.U0[1][r][c] = in[G.plane + g];
        sm.U0[2][r][c] = in[2 * G.plane + g];
    }
    __syncthreads();
    // stage 1: U1 = U0 + dt L(U0) on the 36 x 20 region at offset 2
    stage<S1W, S1H>(&sm.U0[0][0][0], sm, G, [&](int c, int r, float L0, float L1, float L2) {
        sm.U1[0][r - 2][c - 2] = sm.U0[0][r][c] + dt * L0;
        sm.U1[1][r - 2][c - 2] = sm.U0[1][r][c] + dt * L1;
        sm.U1[2][r - 2][c - 2] = sm.U0[2][r][c] + dt * L2;
    });
    // stage 2: U = (U0 + U1 + dt L(U1)) / 2 on the 32 x 16 tile
    stage<TW, TH>(&sm.U1[0][0][0], sm, G, [&](int c, int r, float L0, float L1, float L2) {
        const int gx = x0 + c - 2, gy = y0 + r - 2;
        if (gx < G.nx && gy < G.ny) {
            const long long g = (long long)gy * G.nx + gx;
            outp[g] = 0.5f * (sm.U0[0][r + 2][c + 2] + (sm.U1[0][r][c] + dt * L0));
            outp[G.plane + g] = 0.5f * (sm.U0[1][r + 2][c + 2] + (sm.U1[1][r][c] + dt * L1));
            outp[2 * G.plane + g] = 0.5f * (sm.U0[2][r + 2][c + 2] + (sm.U1[2][r][c] + dt * L2));
        }
    });
}

// max over the particle's cells of max((|u| + c)/dx, (|v| + c)/dy)
__global__ void __launch_bounds__(NTHREADS)
cfl_kernel(const float* __restrict__ buf0, const float* __restrict__ buf1, const int* __restrict__ par,
           float* __restrict__ amax, Grid G)
{
    const int p = blockIdx.y;
    const float* __restrict__ U = (par[p] ? buf1 : buf0) + (long long)p * 3 * G.plane;
    float m = 0.0f;
    for (long long i = (long long)blockIdx.x * NTHREADS + threadIdx.x; i < G.plane;
         i += (long long)gridDim.x * NTHREADS) {
        m = fmaxf(m, cfl_cell(U, i, G));
    }
    m = warp_max(m);
    __shared__ float red[NTHREADS / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < NTHREADS / 32 ? red[threadIdx.x] : 0.0f;
        v = warp_max(v);
        if (threadIdx.x == 0) atomicMax(reinterpret_cast<int*>(amax) + p, __float_as_int(v));
    }
}

// n_sub = ceil(dt_model / dt_cfl), dt_cfl = courant / 4 / amax; dt = dt_model / n_sub
__global__ void nsub_kernel(const float* __restrict__ amax, int* __restrict__ nsub, float* __restrict__ dtp,
                            int* __restrict__ maxsub, int ne, double courant, double dt_model, int fixed)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= ne) return;
    const int n = nsub_of(amax[p], courant, dt_model, fixed);
    nsub[p] = n;
    dtp[p] = (float)(dt_model / (double)n);
    atomicMax(maxsub, n);
}

__global__ void par_update_kernel(int* __restrict__ par, const int* __restrict__ nsub, int ne,
                                  unsigned long long* __restrict__ work)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < ne) {
        par[p] ^= (nsub[p] & 1);
        atomicAdd(work, (unsigned long long)nsub[p]);
    }
}

// forward Euler step of every drifter of every particle still stepping
__global__ void drift_kernel(const float* __restrict__ buf0, const float* __restrict__ buf1,
                             const int* __restrict__ par, const int* __restrict__ nsub,
                             const float* __restrict__ dtp, double* __restrict__ xy, int nd, int s, Grid G,
                             double dx, double dy)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G.ne * nd) return;
    const int p = i / nd;
    if (s >= nsub[p]) return;
    const int cur = par[p] ^ ((s + 1) & 1);     // buffer written by scheme step s
    const float* __restrict__ U = (cur ? buf1 : buf0) + (long long)p * 3 * G.plane;
    double x = xy[2 * i], y = xy[2 * i + 1];
    const int j = pmod((int)floor(x / dx), G.nx), k = pmod((int)floor(y / dy), G.ny);
    const long long c = (long long)k * G.nx + j;
    const float h = G.H + U[c];
    const float u = U[G.plane + c] / h, v = U[2 * G.plane + c] / h;
    const double dt = (double)dtp[p];
    xy[2 * i] = x + dt * (double)u;
    xy[2 * i + 1] = y + dt * (double)v;
}

__global__ void nonfinite_kernel(const float* __restrict__ buf0, const float* __restrict__ buf1,
                                 const int* __restrict__ par, Grid G, int* __restrict__ flag)
{
    const int p = blockIdx.y;
    const float* __restrict__ U = (par[p] ? buf1 : buf0) + (long long)p * 3 * G.plane;
    bool bad = false;
    for (long long i = (long long)blockIdx.x * NTHREADS + threadIdx.x; i < 3 * G.plane;
         i += (long long)gridDim.x * NTHREADS)
        bad |= !isfinite(U[i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, (int)FLAG_NONFINITE);
}

// E(t) and RMSE(t) of the drifters against the truth (eqs.
// errorPerEnsembleDrifter, errorNorm): one CTA, one warp per drifter at a
// time, FP64, fixed summation order
__global__ void __launch_bounds__(256)
drift_errors_kernel(const double* __restrict__ xy, const double* __restrict__ truth, int ne, int nd,
                    double* __restrict__ E, double* __restrict__ RMSE)
{
    __shared__ double se[8], sr[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double accE = 0.0, accR = 0.0;
    for (int d = w; d < nd; d += 8) {
        double mx = 0.0, my = 0.0, e = 0.0;
        for (int i = lane; i < ne; i += 32) {
            const double x = xy[((long long)i * nd + d) * 2], y = xy[((long long)i * nd + d) * 2 + 1];
            mx += x;
            my += y;
            const double ex = x - truth[2 * d], ey = y - truth[2 * d + 1];
            e += ex * ex + ey * ey;
        }
        mx = warp_sum(mx) / ne;
        my = warp_sum(my) / ne;
        e = warp_sum(e);
        double r = 0.0;
        for (int i = lane; i < ne; i += 32) {
            const double ex = xy[((long long)i * nd + d) * 2] - mx, ey = xy[((long long)i * nd + d) * 2 + 1] - my;
            r += ex * ex + ey * ey;
        }
        r = warp_sum(r);
        accE += e / ne;
        accR += r / ne;
    }
    if (lane == 0) {
        se[w] = accE;
        sr[w] = accR;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < 8; ++i) {
            a += se[i];
            b += sr[i];
        }
        *E = sqrt(a / nd);
        *RMSE = sqrt(b / nd);
    }
}

}  // namespace

cudaError_t launch_drift_errors(const double* xy, const double* truth, int ne, int nd, double* E, double* RMSE,
                                cudaStream_t st)
{
    drift_errors_kernel<<<1, 256, 0, st>>>(xy, truth, ne, nd, E, RMSE);
    return cudaGetLastError();
}

size_t rk2_smem_bytes() { return sizeof(Smem); }

cudaError_t launch_rk2(float* b0, float* b1, const int* par, const int* nsub, const float* dtp, int s,
                       const Grid& G, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(rk2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(Smem));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((G.nx + TW - 1) / TW, (G.ny + TH - 1) / TH, G.ne);
    rk2_kernel<<<grid, NTHREADS, sizeof(Smem), st>>>(b0, b1, par, nsub, dtp, s, G);
    return cudaGetLastError();
}

cudaError_t launch_cfl(const float* b0, const float* b1, const int* par, float* amax, int* nsub, float* dtp,
                       int* maxsub, const Grid& G, double courant, double dt_model, int fixed,
                       cudaStream_t st, bool have_amax)
{
    if (!have_amax) cudaMemsetAsync(amax, 0, sizeof(float) * G.ne, st);
    cudaMemsetAsync(maxsub, 0, sizeof(int), st);
    if (fixed <= 0 && !have_amax) {
        const long long blocks = (G.plane + NTHREADS * 8 - 1) / (NTHREADS * 8);
        dim3 grid((unsigned)(blocks < 1 ? 1 : (blocks > 4096 ? 4096 : blocks)), G.ne);
        cfl_kernel<<<grid, NTHREADS, 0, st>>>(b0, b1, par, amax, G);
    }
    nsub_kernel<<<(G.ne + 127) / 128, 128, 0, st>>>(amax, nsub, dtp, maxsub, G.ne, courant, dt_model, fixed);
    return cudaGetLastError();
}

cudaError_t launch_par_update(int* par, const int* nsub, int ne, unsigned long long* work, cudaStream_t st)
{
    par_update_kernel<<<(ne + 127) / 128, 128, 0, st>>>(par, nsub, ne, work);
    return cudaGetLastError();
}

cudaError_t launch_drift(const float* b0, const float* b1, const int* par, const int* nsub, const float* dtp,
                         double* xy, int nd, int s, const Grid& G, double dx, double dy, cudaStream_t st)
{
    const int n = G.ne * nd;
    drift_kernel<<<(n + 127) / 128, 128, 0, st>>>(b0, b1, par, nsub, dtp, xy, nd, s, G, dx, dy);
    return cudaGetLastError();
}

cudaError_t launch_nonfinite(const float* b0, const float* b1, const int* par, const Grid& G, int* flag,
                             cudaStream_t st)
{
    const long long blocks = (3 * G.plane + NTHREADS * 16 - 1) / (NTHREADS * 16);
    dim3 grid((unsigned)(blocks < 1 ? 1 : (blocks > 1024 ? 1024 : blocks)), G.ne);
    nonfinite_kernel<<<grid, NTHREADS, 0, st>>>(b0, b1, par, G, flag);
    return cudaGetLastError();
}

}  // namespace iewpf
