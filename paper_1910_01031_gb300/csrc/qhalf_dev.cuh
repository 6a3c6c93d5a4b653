// Device code of the model-error operator Q^{1/2} = Q_GB^{1/2} I_Omega Q_SOAR^{1/2}
// (Sec. 3.2 of arXiv 1910.01031, eqs. local_soar_on_eta,
// geostrophic_balance_disc, covarianceOperatorsDef) in three stages:
//   Philox normals once per coarse point (normals_block)
//   -> 5x5 SOAR once per coarse point (soar_point)
//   -> per fine tile: bicubic to the tile + 1-cell ring, central-difference
//      geostrophic momentum, read-modify-write of the state (fine_tile).
// The analysis update reuses the fine stage with the posterior coarse field
// and adds the optimal-proposal pull (eq. detailedOPDUpdate) in the same
// read-modify-write.
#pragma once
#include "common.cuh"
#include "kernels.h"

namespace iewpf {
namespace qhalf {

constexpr int TAB_MAX = 45;                   // 3 c for c <= 15
// fine tiles of the model error and of the analysis update (the tiles the
// observation lists are binned by)
constexpr int FINE_TX = OBS_TX, FINE_TY = OBS_TY;

// Per observation of a tile's list, once per tile: the minimum-image offset
// of the tile origin (x0, y0) from the observed cell, in (-n/2, n/2], and the
// particle's S d as float; the cells of the tile then add their own offset
// (at most one period above).  Returns the list length.  Ends with a barrier.
__device__ __forceinline__ int tile_obs_prep(const QhalfArgs& A, const Grid& G, int x0, int y0, int p, int tile,
                                             int* ox0, int* oy0, float* su, float* sv)
{
    const int n = min(A.tile_cnt[tile], MAX_TILE_OBS);
    for (int q = threadIdx.x; q < n; q += NTHREADS) {
        const int l = A.tile_obs[tile * A.tile_cap + q];
        int ox = pmod(x0 - A.obs_cell[2 * l], G.nx);
        int oy = pmod(y0 - A.obs_cell[2 * l + 1], G.ny);
        if (ox > G.nx / 2) ox -= G.nx;
        if (oy > G.ny / 2) oy -= G.ny;
        ox0[q] = ox;
        oy0[q] = oy;
        su[q] = (float)A.Sd[(long long)p * 2 * A.nobs + 2 * l];
        sv[q] = (float)A.Sd[(long long)p * 2 * A.nobs + 2 * l + 1];
    }
    __syncthreads();
    return n;
}

// Coarse stages once per coarse point.  Normals of block q (counter q) of a
// Philox stream: words (0, 1) and (2, 3) give the Box-Muller pairs of normals
// 4q, 4q + 1 and 4q + 2, 4q + 3 (the same numbers normal32 returns one by one).
__device__ __forceinline__ void normals_block(uint2 key, uint32_t p, uint32_t t, uint32_t stream, uint32_t q,
                                              long long NR, float* __restrict__ out)
{
    const uint4 w = philox4x32_10(make_uint4(q, p, t, stream), key);
    float z[4];
    box_muller32(w.x, w.y, z[0], z[1]);
    box_muller32(w.z, w.w, z[2], z[3]);
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (4LL * q + j < NR) out[4LL * q + j] = z[j];
}

// Q_SOAR^{1/2} at coarse point (am, bm) of field src [N_R]: the 5 x 5 sum of
// eq. local_soar_on_eta over the coarse neighbours, rows outer
__device__ __forceinline__ float soar_point(const float* __restrict__ src, const float* __restrict__ wtab,
                                            const Coarse& C, const Grid& G, int am, int bm)
{
    if (am >= 2 && am + 2 < C.nRx && bm >= 2 && bm + 2 < C.nRy) {
        // away from the periodic seam the neighbours are c fine cells apart:
        // the same weights and sums as below without the periodic index
        // arithmetic
        float acc = 0.0f;
#pragma unroll
        for (int db = -2; db <= 2; ++db) {
            const float* __restrict__ row = src + (bm + db) * C.nRx + am;
            const float* __restrict__ wr = wtab + C.c * (db < 0 ? -db : db) * C.tab;
#pragma unroll
            for (int da = -2; da <= 2; ++da) acc = fmaf(wr[C.c * (da < 0 ? -da : da)], row[da], acc);
        }
        return acc;
    }
    const int x0 = coarse_pos(am, C.nRx, C.c, C.o, G.nx), y0 = coarse_pos(bm, C.nRy, C.c, C.o, G.ny);
    int dxf[5], col[5];
#pragma unroll
    for (int da = -2; da <= 2; ++da) {
        dxf[da + 2] = abs(coarse_pos(am + da, C.nRx, C.c, C.o, G.nx) - x0);
        col[da + 2] = pmod(am + da, C.nRx);
    }
    float acc = 0.0f;
#pragma unroll
    for (int db = -2; db <= 2; ++db) {
        const int dyf = abs(coarse_pos(bm + db, C.nRy, C.c, C.o, G.ny) - y0);
        const int row = pmod(bm + db, C.nRy) * C.nRx;
#pragma unroll
        for (int da = -2; da <= 2; ++da) acc = fmaf(wtab[dyf * C.tab + dxf[da + 2]], src[row + col[da + 2]], acc);
    }
    return acc;
}

// One fine tile (TX x TY cells) from the SOAR field so_g [N_R] of particle
// p: bicubic to the tile and its 1-cell ring, geostrophic momentum, optional
// pull (`tile` indexes the observation lists, binned by the same tiles), and
// the read-modify-write of the state.  The interpolation runs separably (rows
// first).  Called by whole CTAs of NTHREADS threads; a CTA may call it for
// several tiles in turn.
template <bool PULL, int TX, int TY>
__device__ __forceinline__ void fine_tile(const QhalfArgs& A, const Grid& G, const Coarse& C, int x0, int y0, int p,
                                          int tile, const float* __restrict__ so_g)
{
    constexpr int FW = TX + 2, FH = TY + 2, SXW = FW + 3, SXH = FH + 3;
    static_assert(!PULL || (TX == OBS_TX && TY == OBS_TY), "pull tiles follow the observation lists");
    // the coarse patch, its rows interpolated and the interpolated field share
    // one pool; with the pull, the tile's per-cell sums take its start once
    // the interpolated field has been read
    constexpr int SO_N = SXH * SXW, ROWS_N = SXH * FW, DETA_N = FH * FW;
    static_assert(SO_N + ROWS_N + DETA_N >= 3 * TX * TY, "pull sums fit the pool");
    __shared__ float pool[SO_N + ROWS_N + DETA_N];
    float(*so)[SXW] = reinterpret_cast<float(*)[SXW]>(pool);
    float(*rows)[FW] = reinterpret_cast<float(*)[FW]>(pool + SO_N);
    float(*deta)[FW] = reinterpret_cast<float(*)[FW]>(pool + SO_N + ROWS_N);
    __shared__ int colA[FW], rowB[FH];
    __shared__ float colW[FW][4], rowW[FH][4];

    const int tid = threadIdx.x;
    __syncthreads();   // the shared arrays may still be in use by the previous tile
    float tdum;
    const int a_lo = coarse_interval(x0 - 1, C.nRx, C.c, C.o, G.nx, tdum);
    const int a_hi = coarse_interval(x0 + TX, C.nRx, C.c, C.o, G.nx, tdum);
    const int b_lo = coarse_interval(y0 - 1, C.nRy, C.c, C.o, G.ny, tdum);
    const int b_hi = coarse_interval(y0 + TY, C.nRy, C.c, C.o, G.ny, tdum);
    const int nsx = a_hi - a_lo + 4, nsy = b_hi - b_lo + 4;     // SOAR, first at a_lo - 1
    for (int i = tid; i < FW; i += NTHREADS) {
        float t;
        const int a = coarse_interval(x0 - 1 + i, C.nRx, C.c, C.o, G.nx, t);
        colA[i] = a - a_lo;
        cubic_weights(t, colW[i]);
    }
    for (int i = tid; i < FH; i += NTHREADS) {
        float t;
        const int b = coarse_interval(y0 - 1 + i, C.nRy, C.c, C.o, G.ny, t);
        rowB[i] = b - b_lo;
        cubic_weights(t, rowW[i]);
    }
    // the coarse patch, a row per warp (the indices lie within a period or
    // two of the grid: wrapped by steps, not by an integer modulo)
    for (int sy = tid >> 5; sy < nsy; sy += NTHREADS / 32) {
        int r = b_lo - 1 + sy;
        while (r < 0) r += C.nRy;
        while (r >= C.nRy) r -= C.nRy;
        for (int sx = tid & 31; sx < nsx; sx += 32) {
            int c = a_lo - 1 + sx;
            while (c < 0) c += C.nRx;
            while (c >= C.nRx) c -= C.nRx;
            so[sy][sx] = so_g[r * C.nRx + c];
        }
    }
    __syncthreads();
    // rows: the x-interpolation of every SOAR row at every fine column; a
    // lane keeps its columns' taps and weights, the warps take the rows
    {
        const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
        for (int j = 0; j < (FW + 31) / 32; ++j) {
            const int fx = lane + 32 * j;
            if (fx < FW) {
                const int a = colA[fx];
                const float w0 = colW[fx][0], w1 = colW[fx][1], w2 = colW[fx][2], w3 = colW[fx][3];
                for (int sy = warp; sy < nsy; sy += NTHREADS / 32) {
                    float row = 0.0f;
                    row = fmaf(w0, so[sy][a], row);
                    row = fmaf(w1, so[sy][a + 1], row);
                    row = fmaf(w2, so[sy][a + 2], row);
                    row = fmaf(w3, so[sy][a + 3], row);
                    rows[sy][fx] = row;
                }
            }
        }
    }
    __syncthreads();
    // the y-interpolation: a row of the tile per warp, the lanes along it
    for (int fy = tid >> 5; fy < FH; fy += NTHREADS / 32) {
        const int b = rowB[fy];
        const float w0 = rowW[fy][0], w1 = rowW[fy][1], w2 = rowW[fy][2], w3 = rowW[fy][3];
        for (int fx = tid & 31; fx < FW; fx += 32) {
            float acc = 0.0f;
            acc = fmaf(w0, rows[b][fx], acc);
            acc = fmaf(w1, rows[b + 1][fx], acc);
            acc = fmaf(w2, rows[b + 2][fx], acc);
            acc = fmaf(w3, rows[b + 3][fx], acc);
            deta[fy][fx] = acc;
        }
    }
    __syncthreads();
    __shared__ int obs_ox[PULL ? MAX_TILE_OBS : 1], obs_oy[PULL ? MAX_TILE_OBS : 1];
    __shared__ float obs_su[PULL ? MAX_TILE_OBS : 1], obs_sv[PULL ? MAX_TILE_OBS : 1];
    const int n_obs_tile = PULL ? tile_obs_prep(A, G, x0, y0, p, tile, obs_ox, obs_oy, obs_su, obs_sv) : 0;
    float* __restrict__ U = (A.par[p] ? A.b1 : A.b0) + (long long)p * 3 * G.plane;
    const int W = 2 * A.R + 1;
    float m = 0.0f;    // CFL rate max of the updated cells (with A.amax)
    if (PULL && n_obs_tile > 0) {
        // Pull by observation: each observation of the list, in list order,
        // adds its stencil to the cells it reaches (up to two column and two
        // row intervals of the tile, split where the minimum image wraps),
        // with a barrier between observations.  Every cell thus receives the
        // same operations in the same order as in the per-cell loop below,
        // without testing the observations that do not reach it.  The
        // stencil's reach 2R + 1 lies within the grid on both axes (iewpf_create
        // refuses smaller grids), so each cell sees one image of each stencil.
        static_assert(TX * TY % NTHREADS == 0, "whole tiles per thread");
        constexpr int PER = TX * TY / NTHREADS, N = TX * TY;
        float v0[PER], v1[PER], v2[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = tid + k * NTHREADS;
            const int fx = i % TX + 1, fy = i / TX + 1;
            v0[k] = deta[fy][fx];
            v1[k] = -G.sgh * (deta[fy + 1][fx] - deta[fy - 1][fx]) * G.inv_2dy;
            v2[k] = G.sgh * (deta[fy][fx + 1] - deta[fy][fx - 1]) * G.inv_2dx;
        }
        __syncthreads();
        float* __restrict__ acc = pool;     // [3][TY][TX]
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = tid + k * NTHREADS;
            acc[i] = v0[k];
            acc[N + i] = v1[k];
            acc[2 * N + i] = v2[k];
        }
        __syncthreads();
        const int txv = min(TX, G.nx - x0), tyv = min(TY, G.ny - y0);
        const int fs = W * W;
        for (int q = 0; q < n_obs_tile; ++q) {
            const int ox0 = obs_ox[q], oy0 = obs_oy[q];
            const float su = obs_su[q], sv = obs_sv[q];
            // cells tx with the offset ox0 + tx in [-R, R], or ox0 + tx - n
            // in [-R, R] past the wrap (offset at the interval's start)
            const int xa[2] = {max(0, -A.R - ox0), max(0, G.nx - A.R - ox0)};
            const int xb[2] = {min(txv, A.R - ox0 + 1), min(txv, G.nx + A.R - ox0 + 1)};
            const int ya[2] = {max(0, -A.R - oy0), max(0, G.ny - A.R - oy0)};
            const int yb[2] = {min(tyv, A.R - oy0 + 1), min(tyv, G.ny + A.R - oy0 + 1)};
#pragma unroll
            for (int ix = 0; ix < 2; ++ix) {
                const int w = xb[ix] - xa[ix];
                if (w <= 0) continue;
                const int oxa = ox0 + xa[ix] - (ix ? G.nx : 0) + A.R;
#pragma unroll
                for (int iy = 0; iy < 2; ++iy) {
                    const int h = yb[iy] - ya[iy];
                    if (h <= 0) continue;
                    const int oya = oy0 + ya[iy] - (iy ? G.ny : 0) + A.R;
                    // the rectangle's w x h cells, linearised over the CTA;
                    // row = floor((i + 1/2) / w) in float is exact here
                    // (w, h <= 2R + 1, far below float's integer range)
                    const float rw = 1.0f / (float)w;
                    for (int i = tid; i < w * h; i += NTHREADS) {
                        const int ry = __float2int_rz(((float)i + 0.5f) * rw);
                        const int rx = i - ry * w;
                        const int o = (oya + ry) * W + oxa + rx;
                        const int c = (ya[iy] + ry) * TX + xa[ix] + rx;
                        acc[c] = fmaf(sv, A.K[3 * fs + o], fmaf(su, A.K[0 * fs + o], acc[c]));
                        acc[N + c] = fmaf(sv, A.K[4 * fs + o], fmaf(su, A.K[1 * fs + o], acc[N + c]));
                        acc[2 * N + c] = fmaf(sv, A.K[5 * fs + o], fmaf(su, A.K[2 * fs + o], acc[2 * N + c]));
                    }
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = tid + k * NTHREADS;
            const int gx = x0 + i % TX, gy = y0 + i / TX;
            if (gx >= G.nx || gy >= G.ny) continue;
            const long long g = (long long)gy * G.nx + gx;
            const float e1 = U[g] + acc[i], u1 = U[G.plane + g] + acc[N + i], v1 = U[2 * G.plane + g] + acc[2 * N + i];
            U[g] = e1;
            U[G.plane + g] = u1;
            U[2 * G.plane + g] = v1;
            if (A.amax) m = fmaxf(m, cfl_of(e1, u1, v1, G));
        }
    } else
    for (int i = tid; i < TX * TY; i += NTHREADS) {
        const int tx = i % TX, ty = i / TX;
        const int gx = x0 + tx, gy = y0 + ty;
        if (gx >= G.nx || gy >= G.ny) continue;
        const int fx = tx + 1, fy = ty + 1;
        float de = deta[fy][fx];
        float dhu = -G.sgh * (deta[fy + 1][fx] - deta[fy - 1][fx]) * G.inv_2dy;
        float dhv = G.sgh * (deta[fy][fx + 1] - deta[fy][fx - 1]) * G.inv_2dx;
        const long long g = (long long)gy * G.nx + gx;
        const float e1 = U[g] + de, u1 = U[G.plane + g] + dhu, v1 = U[2 * G.plane + g] + dhv;
        U[g] = e1;
        U[G.plane + g] = u1;
        U[2 * G.plane + g] = v1;
        if (A.amax) m = fmaxf(m, cfl_of(e1, u1, v1, G));
    }
    if (A.amax) {
        __shared__ float red[NTHREADS / 32];
        m = warp_max(m);
        if ((tid & 31) == 0) red[tid >> 5] = m;
        __syncthreads();
        if (tid < 32) {
            float v = tid < NTHREADS / 32 ? red[tid] : 0.0f;
            v = warp_max(v);
            // non-negative floats order like their bit patterns
            if (tid == 0) atomicMax(reinterpret_cast<int*>(A.amax) + p, __float_as_int(v));
        }
    }
}

}  // namespace qhalf
}  // namespace iewpf
