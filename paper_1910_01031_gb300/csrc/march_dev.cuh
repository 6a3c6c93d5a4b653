// Device code of the register-marching scheme step (Sec. 3.1 of arXiv 1910.01031):
// one step of the second-order SSP Runge-Kutta method with central-upwind
// fluxes and the Coriolis-adjusted (well-balanced) reconstruction of eta,
// organised for issue efficiency on GB300, in a scalar form (march_warp) and
// a form with the two stages paired in f32x2 registers (march_warp_paired).
//
// Each warp owns a strip of 32*NC columns (NC per lane) and marches down a
// chunk of rows.  Rows above and below live in a three-row rolling window in
// registers; x-neighbours come from the adjacent lanes by warp shuffles.  Both
// Runge-Kutta stages run in the same march, the second two rows behind the
// first, so a cell is read once and written once per scheme step, with no
// shared memory and no block barriers.  The 4 outermost columns on each side
// of a strip are halo (recomputed by the neighbouring strip) and 8 extra rows
// fill the pipeline of each chunk.  Divisions and square roots use the
// hardware approximations (rcp, sqrt; a few ulp).  The file is compiled
// without automatic multiply-add contraction and every fused multiply-add is
// written out, so each cell's arithmetic is the same whatever the tile shape.
#pragma once
#include "common.cuh"
#include "kernels.h"

namespace iewpf {
namespace march {

constexpr unsigned FULL = 0xffffffffu;

// single hardware approximations (flush-to-zero: depths and wave speeds are
// far from the subnormal range)
__device__ __forceinline__ float frcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float fsqrt(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// three-input minimum and maximum (one instruction each on sm_100 and later)
__device__ __forceinline__ float fmin3(float a, float b, float c)
{
    float y;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(y) : "f"(a), "f"(b), "f"(c));
    return y;
}
__device__ __forceinline__ float fmax3(float a, float b, float c)
{
    float y;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(y) : "f"(a), "f"(b), "f"(c));
    return y;
}

// twice the generalized minmod(theta a, (a + b)/2, theta b), i.e. the
// minmod of (x, y, z) = (2 theta a, a + b, 2 theta b), from the scaled
// differences x, z and the sum y: the smallest of the three when all are
// positive, the largest when all are negative, else 0 -- the median of
// (min, 0, max), max(min, min(max, 0)).  Every use scales the slope by a power
// of two, so carrying 2 sigma is exact.
__device__ __forceinline__ float gmm2s(float x, float y, float z)
{
    return fmaxf(fmin3(x, y, z), fminf(fmax3(x, y, z), 0.0f));
}

__device__ __forceinline__ float gmm2(float a, float b, float th2)
{
    return gmm2s(th2 * a, a + b, th2 * b);   // no contraction here
}

// central-upwind flux, normal momentum qn, tangential qt carried by the mass
// flux with the upwind tangential velocity
__device__ __forceinline__ void flux(float eL, float qnL, float qtL, float eR, float qnR, float qtR, const Grid& G,
                                     float& F0, float& F1, float& F2)
{
    const float hL = G.H + eL, hR = G.H + eR;
    const float rL = frcp(hL), rR = frcp(hR);
    const float unL = qnL * rL, unR = qnR * rR;
    const float cL = fsqrt(G.g * hL), cR = fsqrt(G.g * hR);
    const float ap = fmax3(unL + cL, unR + cR, 0.0f);
    const float am = fmin3(unL - cL, unR - cR, 0.0f);
    const float inv = frcp(ap - am);
    const float apam = ap * am;
    F0 = fmaf(apam, eR - eL, fmaf(ap, qnL, -(am * qnR))) * inv;
    // p(eta) = g eta (H + eta/2) = eta (g/2 eta + g H)
    const float pL = eL * fmaf(G.g_half, eL, G.gH);
    const float pR = eR * fmaf(G.g_half, eR, G.gH);
    const float mL = fmaf(qnL, unL, pL), mR = fmaf(qnR, unR, pR);
    F1 = fmaf(apam, qnR - qnL, fmaf(ap, mL, -(am * mR))) * inv;
    F2 = F0 * ((F0 >= 0.0f) ? qtL * rL : qtR * rR);
}

template <int NC>
struct Marcher {
    // rolling window: 0 = oldest (row being emitted), 1, 2 = newest
    float e[3][NC], qu[3][NC], qv[3][NC], u[3][NC];
    float dLp[NC];                  // dL on the face between rows 0 and 1
    float tLp[NC], tup[NC], tvp[NC]; // 2 theta times the differences on that face (dL, hu, hv)
    float sL[NC], su[NC], sv[NC];   // y-slopes of row 0 (twice their value)
    float G0[NC], Gu[NC], Gv[NC];   // y-flux on the face below row 0

    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int k = 0; k < NC; ++k) {
#pragma unroll
            for (int r = 0; r < 3; ++r) e[r][k] = qu[r][k] = qv[r][k] = u[r][k] = 0.0f;
            dLp[k] = sL[k] = su[k] = sv[k] = G0[k] = Gu[k] = Gv[k] = 0.0f;
            tLp[k] = tup[k] = tvp[k] = 0.0f;
        }
    }

    // Push the next row; returns L(U) of the row that leaves the window (two
    // rows behind the pushed one) and that row's state.
    __device__ __forceinline__ void push(const float* ne, const float* nqu, const float* nqv, const Grid& G,
                                         float* L0, float* L1, float* L2, float* oe, float* oqu, float* oqv)
    {
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            e[0][k] = e[1][k]; qu[0][k] = qu[1][k]; qv[0][k] = qv[1][k]; u[0][k] = u[1][k];
            e[1][k] = e[2][k]; qu[1][k] = qu[2][k]; qv[1][k] = qv[2][k]; u[1][k] = u[2][k];
            e[2][k] = ne[k]; qu[2][k] = nqu[k]; qv[2][k] = nqv[k];
            u[2][k] = nqu[k] * frcp(G.H + ne[k]);
        }
        // y direction: slopes of row 1, flux on the face between rows 0 and 1
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const float dLn = fmaf(G.fdy_half, u[1][k] + u[2][k], G.g * (e[2][k] - e[1][k]));
            const float dun = qu[2][k] - qu[1][k], dvn = qv[2][k] - qv[1][k];
            const float tLn = G.theta2 * dLn, tun = G.theta2 * dun, tvn = G.theta2 * dvn;
            const float s1L = gmm2s(tLp[k], dLp[k] + dLn, tLn);
            const float s1u = gmm2s(tup[k], (qu[1][k] - qu[0][k]) + dun, tun);
            const float s1v = gmm2s(tvp[k], (qv[1][k] - qv[0][k]) + dvn, tvn);
            tLp[k] = tLn; tup[k] = tun; tvp[k] = tvn;
            const float eB = fmaf(fmaf(-G.fdy2, u[0][k], sL[k]), G.inv_4g, e[0][k]);
            const float eT = fmaf(fmaf(-G.fdy2, u[1][k], s1L), -G.inv_4g, e[1][k]);
            float g0, gv, gu;
            flux(eB, fmaf(0.25f, sv[k], qv[0][k]), fmaf(0.25f, su[k], qu[0][k]), eT, fmaf(-0.25f, s1v, qv[1][k]),
                 fmaf(-0.25f, s1u, qu[1][k]), G, g0, gv, gu);
            L0[k] = (G0[k] - g0) * G.inv_dy;
            L1[k] = (Gu[k] - gu) * G.inv_dy;
            L2[k] = (Gv[k] - gv) * G.inv_dy;
            dLp[k] = dLn;
            sL[k] = s1L; su[k] = s1u; sv[k] = s1v;
            G0[k] = g0; Gu[k] = gu; Gv[k] = gv;
        }
        // x direction on row 0: neighbours from the adjacent lanes
        float E[NC + 2], QU[NC + 2], QV[NC + 2], V[NC + 2];
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            E[k + 1] = e[0][k]; QU[k + 1] = qu[0][k]; QV[k + 1] = qv[0][k];
            V[k + 1] = qv[0][k] * frcp(G.H + e[0][k]);
        }
        E[0] = __shfl_up_sync(FULL, E[NC], 1);
        QU[0] = __shfl_up_sync(FULL, QU[NC], 1);
        QV[0] = __shfl_up_sync(FULL, QV[NC], 1);
        V[0] = __shfl_up_sync(FULL, V[NC], 1);
        E[NC + 1] = __shfl_down_sync(FULL, E[1], 1);
        QU[NC + 1] = __shfl_down_sync(FULL, QU[1], 1);
        QV[NC + 1] = __shfl_down_sync(FULL, QV[1], 1);
        V[NC + 1] = __shfl_down_sync(FULL, V[1], 1);
        // differences on the faces f = 0..NC (left of column f) and their
        // 2 theta multiples, each formed once and shared by both neighbours
        float dK[NC + 1], dU[NC + 1], dV[NC + 1], tK[NC + 1], tU[NC + 1], tV[NC + 1];
#pragma unroll
        for (int f = 0; f <= NC; ++f) {
            dK[f] = fmaf(-G.fdx_half, V[f] + V[f + 1], G.g * (E[f + 1] - E[f]));
            dU[f] = QU[f + 1] - QU[f];
            dV[f] = QV[f + 1] - QV[f];
            tK[f] = G.theta2 * dK[f];
            tU[f] = G.theta2 * dU[f];
            tV[f] = G.theta2 * dV[f];
        }
        float eE[NC], eW[NC], uE[NC], uW[NC], vE[NC], vW[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const float sK = gmm2s(tK[k], dK[k] + dK[k + 1], tK[k + 1]);
            const float sU = gmm2s(tU[k], dU[k] + dU[k + 1], tU[k + 1]);
            const float sV = gmm2s(tV[k], dV[k] + dV[k + 1], tV[k + 1]);
            const float ex = fmaf(G.fdx2, V[k + 1], sK) * G.inv_4g;
            eE[k] = E[k + 1] + ex; eW[k] = E[k + 1] - ex;
            uE[k] = fmaf(0.25f, sU, QU[k + 1]); uW[k] = fmaf(-0.25f, sU, QU[k + 1]);
            vE[k] = fmaf(0.25f, sV, QV[k + 1]); vW[k] = fmaf(-0.25f, sV, QV[k + 1]);
        }
        // face f lies on the left of own column f; face NC is the right edge
        float F0[NC + 1], F1[NC + 1], F2[NC + 1];
#pragma unroll
        for (int f = 1; f < NC; ++f) flux(eE[f - 1], uE[f - 1], vE[f - 1], eW[f], uW[f], vW[f], G, F0[f], F1[f], F2[f]);
        {
            const float eRW = __shfl_down_sync(FULL, eW[0], 1);
            const float uRW = __shfl_down_sync(FULL, uW[0], 1);
            const float vRW = __shfl_down_sync(FULL, vW[0], 1);
            flux(eE[NC - 1], uE[NC - 1], vE[NC - 1], eRW, uRW, vRW, G, F0[NC], F1[NC], F2[NC]);
        }
        F0[0] = __shfl_up_sync(FULL, F0[NC], 1);
        F1[0] = __shfl_up_sync(FULL, F1[NC], 1);
        F2[0] = __shfl_up_sync(FULL, F2[NC], 1);
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            L0[k] = fmaf(F0[k] - F0[k + 1], G.inv_dx, L0[k]);
            L1[k] = fmaf(F1[k] - F1[k + 1], G.inv_dx, L1[k]);
            L2[k] = fmaf(F2[k] - F2[k + 1], G.inv_dx, L2[k]);
            L1[k] = fmaf(G.f, qv[0][k], L1[k]);
            L2[k] = fmaf(-G.f, qu[0][k], L2[k]);
            oe[k] = e[0][k]; oqu[k] = qu[0][k]; oqv[k] = qv[0][k];
        }
    }
};

// One warp's strip of one chunk of particle p in scheme step s.
template <int NC>
__device__ __forceinline__ void march_warp(const StepArgs& a, int p, int chunk, int strip, int s)
{
    constexpr int WUSE = 32 * NC - 8;          // useful columns per strip
    const Grid& G = a.G;
    const int TH = a.TH;
    const int lane = threadIdx.x & 31;
    if (s >= a.nsub[p]) return;
    const int src = a.par[p] ^ (s & 1);
    float* __restrict__ buf0 = a.buf0;
    float* __restrict__ buf1 = a.buf1;
    const float* __restrict__ dtp = a.dtp;
    const float* __restrict__ in = (src ? buf1 : buf0) + (long long)p * 3 * G.plane;
    float* __restrict__ out = (src ? buf0 : buf1) + (long long)p * 3 * G.plane;
    const float dt = dtp[p];
    const int y0 = chunk * TH;
    const int rows = min(TH, G.ny - y0);
    // columns of this lane: strip-local c = lane*NC + k, global x = strip*WUSE - 4 + c
    int gx[NC];
    bool keep[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const int c = lane * NC + k;
        const int x = strip * WUSE - 4 + c;
        gx[k] = pmod(x, G.nx);
        keep[k] = (c >= 4) && (c < 32 * NC - 4) && (x < G.nx);
    }
    Marcher<NC> S1, S2;
    S1.zero();
    S2.zero();
    float f0e[NC], f0u[NC], f0v[NC], f1e[NC], f1u[NC], f1v[NC];   // U0 of the last two emitted rows
#pragma unroll
    for (int k = 0; k < NC; ++k) f0e[k] = f0u[k] = f0v[k] = f1e[k] = f1u[k] = f1v[k] = 0.0f;
    const int n_it = rows + 8;
    float ne[NC], nqu[NC], nqv[NC];
    {
        const long long r0 = (long long)pmod(y0 - 4, G.ny) * G.nx;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            ne[k] = __ldg(in + r0 + gx[k]);
            nqu[k] = __ldg(in + G.plane + r0 + gx[k]);
            nqv[k] = __ldg(in + 2 * G.plane + r0 + gx[k]);
        }
    }
    int yn = pmod(y0 - 3, G.ny);     // row of the next prefetch, wrapped as it advances
    for (int it = 0; it < n_it; ++it) {
        // prefetch the next input row
        float pe[NC], pqu[NC], pqv[NC];
        if (it + 1 < n_it) {
            const long long rn = (long long)yn * G.nx;
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                pe[k] = __ldg(in + rn + gx[k]);
                pqu[k] = __ldg(in + G.plane + rn + gx[k]);
                pqv[k] = __ldg(in + 2 * G.plane + rn + gx[k]);
            }
        }
        yn = yn + 1 == G.ny ? 0 : yn + 1;
        // stage 1 on U0, then stage 2 on U1 = U0 + dt L(U0)
        float L0[NC], L1[NC], L2[NC], ue[NC], uu[NC], uv[NC];
        S1.push(ne, nqu, nqv, G, L0, L1, L2, ue, uu, uv);
        float we[NC], wu[NC], wv[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            we[k] = fmaf(dt, L0[k], ue[k]);
            wu[k] = fmaf(dt, L1[k], uu[k]);
            wv[k] = fmaf(dt, L2[k], uv[k]);
        }
        float M0[NC], M1[NC], M2[NC], ve[NC], vu[NC], vv[NC];
        S2.push(we, wu, wv, G, M0, M1, M2, ve, vu, vv);
        if (it >= 8) {
            const long long ro = (long long)(y0 + it - 8) * G.nx;
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                if (keep[k]) {
                    out[ro + gx[k]] = 0.5f * (f1e[k] + fmaf(dt, M0[k], ve[k]));
                    out[G.plane + ro + gx[k]] = 0.5f * (f1u[k] + fmaf(dt, M1[k], vu[k]));
                    out[2 * G.plane + ro + gx[k]] = 0.5f * (f1v[k] + fmaf(dt, M2[k], vv[k]));
                }
            }
        }
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            f1e[k] = f0e[k]; f1u[k] = f0u[k]; f1v[k] = f0v[k];
            f0e[k] = ue[k]; f0u[k] = uu[k]; f0v[k] = uv[k];
            ne[k] = pe[k]; nqu[k] = pqu[k]; nqv[k] = pqv[k];
        }
    }
}


// ---------------------------------------------------------------------------
// Paired form of the same march.  The two Runge-Kutta stages advance as the
// two halves of packed f32x2 registers: the low half carries stage 1 on U0,
// the high half stage 2 on U1 = U0 + dt L(U0), one row later than in
// march_warp so that both halves of a push are independent (stage 2 takes the
// row that stage 1 finished in the previous iteration).  Every add, multiply
// and fused multiply-add then covers both stages in one packed instruction;
// the hardware approximations, minima and maxima, selects and shuffles stay
// per half.  Each half performs exactly the scalar march's operations in the
// same order, so results are identical bit for bit.  The 2 theta multiples of
// the previous face differences are formed again instead of carried, and the
// original state of the output row is read again from the input (a row read
// five iterations earlier, normally still in L1) instead of being held, which
// keeps the live registers close to the scalar form's.
// ---------------------------------------------------------------------------
namespace pr {

using f2 = float2;

__device__ __forceinline__ f2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 add(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 neg(f2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ f2 sub(f2 a, f2 b) { return __fadd2_rn(a, neg(b)); }
__device__ __forceinline__ f2 mul(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 rcp(f2 a) { return make_float2(frcp(a.x), frcp(a.y)); }
__device__ __forceinline__ f2 sqr(f2 a) { return make_float2(fsqrt(a.x), fsqrt(a.y)); }
__device__ __forceinline__ f2 max3z(f2 a, f2 b) { return make_float2(fmax3(a.x, b.x, 0.0f), fmax3(a.y, b.y, 0.0f)); }
__device__ __forceinline__ f2 min3z(f2 a, f2 b) { return make_float2(fmin3(a.x, b.x, 0.0f), fmin3(a.y, b.y, 0.0f)); }
__device__ __forceinline__ f2 gmm(f2 x, f2 y, f2 z) { return make_float2(gmm2s(x.x, y.x, z.x), gmm2s(x.y, y.y, z.y)); }
__device__ __forceinline__ f2 shup(f2 v) { return make_float2(__shfl_up_sync(FULL, v.x, 1), __shfl_up_sync(FULL, v.y, 1)); }
__device__ __forceinline__ f2 shdn(f2 v)
{
    return make_float2(__shfl_down_sync(FULL, v.x, 1), __shfl_down_sync(FULL, v.y, 1));
}

// grid constants broadcast to both halves
struct K2 {
    f2 H, g, g_half, gH, theta2, inv_4g, ninv_4g, quarter, nquarter;
    f2 fdy_half, nfdy2, inv_dy, nfdx_half, fdx2, inv_dx, f, nf;
};
__device__ __forceinline__ K2 make_k2(const Grid& G)
{
    return K2{bc(G.H), bc(G.g), bc(G.g_half), bc(G.gH), bc(G.theta2), bc(G.inv_4g), bc(-G.inv_4g), bc(0.25f),
              bc(-0.25f), bc(G.fdy_half), bc(-G.fdy2), bc(G.inv_dy), bc(-G.fdx_half), bc(G.fdx2), bc(G.inv_dx),
              bc(G.f), bc(-G.f)};
}

// central-upwind flux of march::flux on both halves
__device__ __forceinline__ void flux(f2 eL, f2 qnL, f2 qtL, f2 eR, f2 qnR, f2 qtR, const K2& K, f2& F0, f2& F1,
                                     f2& F2)
{
    const f2 hL = add(K.H, eL), hR = add(K.H, eR);
    const f2 rL = rcp(hL), rR = rcp(hR);
    const f2 unL = mul(qnL, rL), unR = mul(qnR, rR);
    const f2 xL = mul(K.g, hL), xR = mul(K.g, hR);
    const f2 cL = sqr(xL), cR = sqr(xR);
    const f2 ap = max3z(add(unL, cL), add(unR, cR));
    const f2 am = min3z(sub(unL, cL), sub(unR, cR));
    const f2 inv = rcp(sub(ap, am));
    const f2 apam = mul(ap, am);
    const f2 nam = neg(am);
    F0 = mul(fma(apam, sub(eR, eL), fma(ap, qnL, mul(nam, qnR))), inv);
    const f2 pL = mul(eL, fma(K.g_half, eL, K.gH));
    const f2 pR = mul(eR, fma(K.g_half, eR, K.gH));
    const f2 mL = fma(qnL, unL, pL), mR = fma(qnR, unR, pR);
    F1 = mul(fma(apam, sub(qnR, qnL), fma(ap, mL, mul(nam, mR))), inv);
    const f2 vL = mul(qtL, rL), vR = mul(qtR, rR);
    F2 = mul(F0, make_float2(F0.x >= 0.0f ? vL.x : vR.x, F0.y >= 0.0f ? vL.y : vR.y));
}

template <int NC>
struct Marcher {
    // rolling window: 0 = oldest (row being emitted), 1, 2 = newest
    f2 e[3][NC], qu[3][NC], qv[3][NC], u[3][NC];
    f2 dLp[NC];                 // dL on the face between rows 0 and 1
    f2 sL[NC], su[NC], sv[NC];  // y-slopes of row 0 (twice their value)
    f2 G0[NC], Gu[NC], Gv[NC];  // y-flux on the face below row 0

    __device__ __forceinline__ void zero()
    {
        const f2 z = bc(0.0f);
#pragma unroll
        for (int k = 0; k < NC; ++k) {
#pragma unroll
            for (int r = 0; r < 3; ++r) e[r][k] = qu[r][k] = qv[r][k] = u[r][k] = z;
            dLp[k] = sL[k] = su[k] = sv[k] = G0[k] = Gu[k] = Gv[k] = z;
        }
    }

    __device__ __forceinline__ void push(const f2* ne, const f2* nqu, const f2* nqv, const K2& K, f2* L0, f2* L1,
                                         f2* L2, f2* oe, f2* oqu, f2* oqv)
    {
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            e[0][k] = e[1][k]; qu[0][k] = qu[1][k]; qv[0][k] = qv[1][k]; u[0][k] = u[1][k];
            e[1][k] = e[2][k]; qu[1][k] = qu[2][k]; qv[1][k] = qv[2][k]; u[1][k] = u[2][k];
            e[2][k] = ne[k]; qu[2][k] = nqu[k]; qv[2][k] = nqv[k];
            u[2][k] = mul(nqu[k], rcp(add(K.H, ne[k])));
        }
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const f2 dLn = fma(K.fdy_half, add(u[1][k], u[2][k]), mul(K.g, sub(e[2][k], e[1][k])));
            const f2 dun = sub(qu[2][k], qu[1][k]), dvn = sub(qv[2][k], qv[1][k]);
            const f2 dup = sub(qu[1][k], qu[0][k]), dvp = sub(qv[1][k], qv[0][k]);
            const f2 s1L = gmm(mul(K.theta2, dLp[k]), add(dLp[k], dLn), mul(K.theta2, dLn));
            const f2 s1u = gmm(mul(K.theta2, dup), add(dup, dun), mul(K.theta2, dun));
            const f2 s1v = gmm(mul(K.theta2, dvp), add(dvp, dvn), mul(K.theta2, dvn));
            const f2 eB = fma(fma(K.nfdy2, u[0][k], sL[k]), K.inv_4g, e[0][k]);
            const f2 eT = fma(fma(K.nfdy2, u[1][k], s1L), K.ninv_4g, e[1][k]);
            f2 g0, gv, gu;
            flux(eB, fma(K.quarter, sv[k], qv[0][k]), fma(K.quarter, su[k], qu[0][k]), eT,
                 fma(K.nquarter, s1v, qv[1][k]), fma(K.nquarter, s1u, qu[1][k]), K, g0, gv, gu);
            L0[k] = mul(sub(G0[k], g0), K.inv_dy);
            L1[k] = mul(sub(Gu[k], gu), K.inv_dy);
            L2[k] = mul(sub(Gv[k], gv), K.inv_dy);
            dLp[k] = dLn;
            sL[k] = s1L; su[k] = s1u; sv[k] = s1v;
            G0[k] = g0; Gu[k] = gu; Gv[k] = gv;
        }
        f2 E[NC + 2], QU[NC + 2], QV[NC + 2], V[NC + 2];
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            E[k + 1] = e[0][k]; QU[k + 1] = qu[0][k]; QV[k + 1] = qv[0][k];
            V[k + 1] = mul(qv[0][k], rcp(add(K.H, e[0][k])));
        }
        E[0] = shup(E[NC]); QU[0] = shup(QU[NC]); QV[0] = shup(QV[NC]); V[0] = shup(V[NC]);
        E[NC + 1] = shdn(E[1]); QU[NC + 1] = shdn(QU[1]); QV[NC + 1] = shdn(QV[1]); V[NC + 1] = shdn(V[1]);
        f2 dK[NC + 1], dU[NC + 1], dV[NC + 1];
#pragma unroll
        for (int f = 0; f <= NC; ++f) {
            dK[f] = fma(K.nfdx_half, add(V[f], V[f + 1]), mul(K.g, sub(E[f + 1], E[f])));
            dU[f] = sub(QU[f + 1], QU[f]);
            dV[f] = sub(QV[f + 1], QV[f]);
        }
        f2 eE[NC], eW[NC], uE[NC], uW[NC], vE[NC], vW[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const f2 sK = gmm(mul(K.theta2, dK[k]), add(dK[k], dK[k + 1]), mul(K.theta2, dK[k + 1]));
            const f2 sU = gmm(mul(K.theta2, dU[k]), add(dU[k], dU[k + 1]), mul(K.theta2, dU[k + 1]));
            const f2 sV = gmm(mul(K.theta2, dV[k]), add(dV[k], dV[k + 1]), mul(K.theta2, dV[k + 1]));
            const f2 ex = mul(fma(K.fdx2, V[k + 1], sK), K.inv_4g);
            eE[k] = add(E[k + 1], ex); eW[k] = sub(E[k + 1], ex);
            uE[k] = fma(K.quarter, sU, QU[k + 1]); uW[k] = fma(K.nquarter, sU, QU[k + 1]);
            vE[k] = fma(K.quarter, sV, QV[k + 1]); vW[k] = fma(K.nquarter, sV, QV[k + 1]);
        }
        f2 F0[NC + 1], F1[NC + 1], F2[NC + 1];
#pragma unroll
        for (int f = 1; f < NC; ++f) flux(eE[f - 1], uE[f - 1], vE[f - 1], eW[f], uW[f], vW[f], K, F0[f], F1[f], F2[f]);
        flux(eE[NC - 1], uE[NC - 1], vE[NC - 1], shdn(eW[0]), shdn(uW[0]), shdn(vW[0]), K, F0[NC], F1[NC], F2[NC]);
        F0[0] = shup(F0[NC]); F1[0] = shup(F1[NC]); F2[0] = shup(F2[NC]);
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            L0[k] = fma(sub(F0[k], F0[k + 1]), K.inv_dx, L0[k]);
            L1[k] = fma(sub(F1[k], F1[k + 1]), K.inv_dx, L1[k]);
            L2[k] = fma(sub(F2[k], F2[k + 1]), K.inv_dx, L2[k]);
            L1[k] = fma(K.f, qv[0][k], L1[k]);
            L2[k] = fma(K.nf, qu[0][k], L2[k]);
            oe[k] = e[0][k]; oqu[k] = qu[0][k]; oqv[k] = qv[0][k];
        }
    }
};

}  // namespace pr

// One warp's strip of one chunk of particle p in scheme step s, both stages
// paired (see above); the same strips, chunks and output as march_warp.
template <int NC>
__device__ __forceinline__ void march_warp_paired(const StepArgs& a, int p, int chunk, int strip, int s)
{
    using pr::f2;
    constexpr int WUSE = 32 * NC - 8;
    const Grid& G = a.G;
    const int TH = a.TH;
    const int lane = threadIdx.x & 31;
    if (s >= a.nsub[p]) return;
    const int src = a.par[p] ^ (s & 1);
    float* __restrict__ buf0 = a.buf0;
    float* __restrict__ buf1 = a.buf1;
    const float* __restrict__ in = (src ? buf1 : buf0) + (long long)p * 3 * G.plane;
    float* __restrict__ out = (src ? buf0 : buf1) + (long long)p * 3 * G.plane;
    const f2 dt = pr::bc(a.dtp[p]);
    const int y0 = chunk * TH;
    const int rows = min(TH, G.ny - y0);
    int gx[NC];
    bool keep[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const int c = lane * NC + k;
        const int x = strip * WUSE - 4 + c;
        gx[k] = pmod(x, G.nx);
        keep[k] = (c >= 4) && (c < 32 * NC - 4) && (x < G.nx);
    }
    const pr::K2 K = pr::make_k2(G);
    pr::Marcher<NC> S;
    S.zero();
    // push input: low half the next row of U0, high half W of the row that
    // stage 1 finished in the previous iteration
    f2 ne[NC], nqu[NC], nqv[NC];
    {
        const long long r0 = (long long)pmod(y0 - 4, G.ny) * G.nx;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            ne[k] = make_float2(__ldg(in + r0 + gx[k]), 0.0f);
            nqu[k] = make_float2(__ldg(in + G.plane + r0 + gx[k]), 0.0f);
            nqv[k] = make_float2(__ldg(in + 2 * G.plane + r0 + gx[k]), 0.0f);
        }
    }
    const int n_it = rows + 9;
    int yn = pmod(y0 - 3, G.ny);     // row of the next prefetch, wrapped as it advances
    for (int it = 0; it < n_it; ++it) {
        float pe[NC], pqu[NC], pqv[NC];
        if (it + 1 < n_it) {
            const long long rn = (long long)yn * G.nx;
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                pe[k] = __ldg(in + rn + gx[k]);
                pqu[k] = __ldg(in + G.plane + rn + gx[k]);
                pqv[k] = __ldg(in + 2 * G.plane + rn + gx[k]);
            }
        }
        yn = yn + 1 == G.ny ? 0 : yn + 1;
        // the original state of this iteration's output row, read again
        // (issued here so that the loads complete during the push)
        const bool emit = it >= 9;
        const long long ro = (long long)(y0 + it - 9) * G.nx;
        float o0[NC], o1[NC], o2[NC];
        if (emit) {
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                o0[k] = __ldg(in + ro + gx[k]);
                o1[k] = __ldg(in + G.plane + ro + gx[k]);
                o2[k] = __ldg(in + 2 * G.plane + ro + gx[k]);
            }
        }
        f2 L0[NC], L1[NC], L2[NC], oe[NC], ou[NC], ov[NC];
        S.push(ne, nqu, nqv, K, L0, L1, L2, oe, ou, ov);
        // low: W = U0 + dt L(U0) of the row stage 1 emitted; high: U1 + dt
        // L(U1) of the row stage 2 emitted
        f2 z0[NC], z1[NC], z2[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            z0[k] = pr::fma(dt, L0[k], oe[k]);
            z1[k] = pr::fma(dt, L1[k], ou[k]);
            z2[k] = pr::fma(dt, L2[k], ov[k]);
        }
        if (emit) {
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                if (keep[k]) {
                    out[ro + gx[k]] = 0.5f * (o0[k] + z0[k].y);
                    out[G.plane + ro + gx[k]] = 0.5f * (o1[k] + z1[k].y);
                    out[2 * G.plane + ro + gx[k]] = 0.5f * (o2[k] + z2[k].y);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            ne[k] = make_float2(pe[k], z0[k].x);
            nqu[k] = make_float2(pqu[k], z1[k].x);
            nqv[k] = make_float2(pqv[k], z2[k].x);
        }
    }
}

}  // namespace march
}  // namespace iewpf
