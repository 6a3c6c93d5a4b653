// Device code of the IEWPF analysis (Sec. 4 and App. A of arXiv 1910.01031):
// observation set-up, eta-compensated innovations, assembly and FP64
// Cholesky factorisation of HQH^T + R, the S d solves with phi_i, the
// perpendicular random vectors' dot products, the ensemble-wide target
// weight / beta / Lambert-W alpha step, the posterior coarse field and the
// local 49x49 block root applied around each observation.  Each function
// does the work of one thread, warp or CTA (as named) for one problem, so
// that single-problem and batched kernels share it.
#pragma once
#include "common.cuh"
#include "kernels.h"

namespace iewpf {
namespace ana {

__device__ __forceinline__ int min_image(int d, int n)
{
    d = pmod(d, n);
    return d > n / 2 ? d - n : d;
}

// cell and nearest coarse point (ties to the lower one) of observation l
__device__ __forceinline__ void obs_cell_one(const double* __restrict__ xy, int l, const Grid& G, const Coarse& C,
                                             double dx, double dy, int* __restrict__ cell, int* __restrict__ block0)
{
    const int j = pmod((int)floor(xy[2 * l] / dx), G.nx);
    const int k = pmod((int)floor(xy[2 * l + 1] / dy), G.ny);
    cell[2 * l] = j;
    cell[2 * l + 1] = k;
    float t;
    int a = coarse_interval(j, C.nRx, C.c, C.o, G.nx, t);
    int xa = coarse_pos(a, C.nRx, C.c, C.o, G.nx), xb = coarse_pos(a + 1, C.nRx, C.c, C.o, G.nx);
    block0[2 * l] = pmod((j - xa) <= (xb - j) ? a : a + 1, C.nRx);
    int b = coarse_interval(k, C.nRy, C.c, C.o, G.ny, t);
    int ya = coarse_pos(b, C.nRy, C.c, C.o, G.ny), yb = coarse_pos(b + 1, C.nRy, C.c, C.o, G.ny);
    block0[2 * l + 1] = pmod((k - ya) <= (yb - k) ? b : b + 1, C.nRy);
}

// CTA of NTHREADS: observations whose stencil box meets `tile`, listed in
// observation order (deterministic sums in the update kernel)
__device__ __forceinline__ void tile_bin_cta(const int* __restrict__ cell, int nobs, const Grid& G, int R, int tile,
                                             int* __restrict__ cnt, int* __restrict__ list, int cap,
                                             int* __restrict__ flag)
{
    __shared__ int base;
    __shared__ int warp_tot[NTHREADS / 32];
    const int tx = tile % ((G.nx + OBS_TX - 1) / OBS_TX), ty = tile / ((G.nx + OBS_TX - 1) / OBS_TX);
    const int cx = tx * OBS_TX + OBS_TX / 2, cy = ty * OBS_TY + OBS_TY / 2;
    __syncthreads();
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int l0 = 0; l0 < nobs; l0 += NTHREADS) {
        const int l = l0 + threadIdx.x;
        bool hit = false;
        if (l < nobs) {
            const int ox = min_image(cell[2 * l] - cx, G.nx), oy = min_image(cell[2 * l + 1] - cy, G.ny);
            hit = abs(ox) <= R + OBS_TX / 2 + 1 && abs(oy) <= R + OBS_TY / 2 + 1;
        }
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (lane == 0) warp_tot[w] = __popc(m);
        __syncthreads();
        int off = base;
        for (int i = 0; i < w; ++i) off += warp_tot[i];
        off += __popc(m & ((1u << lane) - 1u));
        if (hit) {
            if (off < cap) list[tile * cap + off] = l;
            else atomicOr(flag, FLAG_TILE_OVERFLOW);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int i = 0; i < NTHREADS / 32; ++i) tot += warp_tot[i];
            base += tot;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) cnt[tile] = base < cap ? base : cap;
}

// d = y (H + eta)/H - (hu, hv) at the observed cell (eq. etaCompensatedInnovation)
__device__ __forceinline__ void innovate_one(const float* __restrict__ b0, const float* __restrict__ b1,
                                             const int* __restrict__ par, const int* __restrict__ cell,
                                             const double* __restrict__ y, int nobs, const Grid& G, double H,
                                             double* __restrict__ d, int i)
{
    const int p = i / nobs, l = i % nobs;
    const float* __restrict__ U = (par[p] ? b1 : b0) + (long long)p * 3 * G.plane;
    const long long c = (long long)cell[2 * l + 1] * G.nx + cell[2 * l];
    const double s = (H + (double)U[c]) / H;
    d[(long long)i * 2] = fma(y[2 * l], s, -(double)U[G.plane + c]);
    d[(long long)i * 2 + 1] = fma(y[2 * l + 1], s, -(double)U[2 * G.plane + c]);
}

// (HQH^T)_{(l,a),(k,b)}: component a of the response to a unit b observation
// at obs k, read at obs l's cell
__device__ __forceinline__ double kval(const double* K, int R, const int* cell, int l, int a, int k, int b,
                                       const Grid& G)
{
    const int ox = min_image(cell[2 * l] - cell[2 * k], G.nx);
    const int oy = min_image(cell[2 * l + 1] - cell[2 * k + 1], G.ny);
    if (abs(ox) > R || abs(oy) > R) return 0.0;
    const int W = 2 * R + 1;
    return K[((b * 3 + 1 + a) * W + (oy + R)) * W + (ox + R)];
}

// entry i of the symmetrised HQH^T + sigma^2 I
__device__ __forceinline__ void hqht_one(const double* __restrict__ K, int R, const int* __restrict__ cell, int nobs,
                                         const Grid& G, int dense, double sigma2, double* __restrict__ M, long long i)
{
    const int n = 2 * nobs;
    const int r = (int)(i / n), c = (int)(i % n);
    const int l = r >> 1, a = r & 1, k = c >> 1, b = c & 1;
    double v = 0.0;
    if (dense || l == k) v = 0.5 * (kval(K, R, cell, l, a, k, b, G) + kval(K, R, cell, k, b, l, a, G));
    if (r == c) v += sigma2;
    M[i] = v;
}

// Right-looking Cholesky of a dense SPD matrix in place (lower triangle), one
// CTA; the update of column k touches only rows with a non-zero in it, so
// block-diagonal and banded matrices cost their fill, not n^3/3.  A may live
// in global or shared memory; nzlist holds n ints.  The strict upper triangle
// is zeroed; *bad (shared) is set for a non-positive pivot.
__device__ __forceinline__ void cholesky_factor_cta(double* __restrict__ A, int n, int* __restrict__ nzlist, int* bad)
{
    __shared__ int nnz;
    __shared__ double piv;
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            const double dkk = A[(long long)k * n + k];
            if (!(dkk > 0.0)) *bad = 1;
            piv = dkk > 0.0 ? sqrt(dkk) : 1.0;
            A[(long long)k * n + k] = piv;
            nnz = 0;
        }
        __syncthreads();
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) {
            const double v = A[(long long)i * n + k];
            if (v != 0.0) {
                A[(long long)i * n + k] = v / piv;
                nzlist[atomicAdd(&nnz, 1)] = i;
            }
        }
        __syncthreads();
        const int m = nnz;
        const long long pairs = (long long)m * m;
        for (long long q = threadIdx.x; q < pairs; q += blockDim.x) {
            const int i = nzlist[q / m], j = nzlist[q % m];
            if (j <= i) A[(long long)i * n + j] = fma(-A[(long long)i * n + k], A[(long long)j * n + k], A[(long long)i * n + j]);
        }
        __syncthreads();
    }
    for (long long q = threadIdx.x; q < (long long)n * n; q += blockDim.x) {
        const int i = (int)(q / n), j = (int)(q % n);
        if (j > i) A[q] = 0.0;
    }
    __syncthreads();
}

// The factor's columns as CSC of the strictly lower part, rows increasing:
// one warp per column counts (ballots), a prefix sum gives colptr, and the
// warps write the row lists in order.
__device__ __forceinline__ void csc_cta(const double* __restrict__ L, int n, int* __restrict__ colptr,
                                        int* __restrict__ rowidx)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = warp; k < n; k += nw) {
        int cnt = 0;
        for (int i0 = k + 1; i0 < n; i0 += 32) {
            const int i = i0 + lane;
            cnt += __popc(__ballot_sync(0xffffffffu, i < n && L[(long long)i * n + k] != 0.0));
        }
        if (lane == 0) colptr[k + 1] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        colptr[0] = 0;
        for (int k = 0; k < n; ++k) colptr[k + 1] += colptr[k];
    }
    __syncthreads();
    for (int k = warp; k < n; k += nw) {
        int pos = colptr[k];
        for (int i0 = k + 1; i0 < n; i0 += 32) {
            const int i = i0 + lane;
            const bool nz = i < n && L[(long long)i * n + k] != 0.0;
            const unsigned bal = __ballot_sync(0xffffffffu, nz);
            if (nz) rowidx[pos + __popc(bal & ((1u << lane) - 1u))] = i;
            pos += __popc(bal);
        }
    }
    __syncthreads();
}

// Factor in global memory and list the factor's columns; rowidx doubles as
// the work list during the factorisation.
// rowidx and nzlist may be the same array (the work list of the
// factorisation, then the row indices of the factor), so neither is restrict
__device__ __forceinline__ void cholesky_cta(double* __restrict__ A, int n, int* __restrict__ colptr, int* rowidx,
                                             int* __restrict__ flag, int* nzlist)
{
    __shared__ int bad;
    __syncthreads();
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    cholesky_factor_cta(A, n, nzlist, &bad);
    csc_cta(A, n, colptr, rowidx);
    if (threadIdx.x == 0 && bad) atomicOr(flag, FLAG_NOTPD);
}

// Level schedule of the triangular solves with the factor L (CSC below the
// diagonal in colptr/rowidx).  Rows of one level of the forward sweep
// L y = d depend only on rows of lower levels, and likewise columns of one
// level of the backward sweep L^T x = y; 2 x 2 blocks (observations that do
// not interact) give two levels each.  Int layout of `plan`, n = order:
// rowptr[n+1] | forder[n] | fptr[n+1] | border[n] | bptr[n+1] | nlev[2] |
// lev[n] | colidx[n(n-1)/2] (CSR below the diagonal, column order in a row).
// rf, rb: per position t of the forward (backward) level order, the row
// (column) and the bounds of its entries: {i, start, end}
struct SolvePlan {
    int *rowptr, *forder, *fptr, *border, *bptr, *nlev, *lev, *rf, *rb, *colidx;
};

__host__ __device__ inline SolvePlan solve_plan_view(int* base, int n)
{
    SolvePlan P;
    P.rowptr = base;
    P.forder = P.rowptr + n + 1;
    P.fptr = P.forder + n;
    P.border = P.fptr + n + 1;
    P.bptr = P.border + n;
    P.nlev = P.bptr + n + 1;
    P.lev = P.nlev + 2;
    P.rf = P.lev + n;
    P.rb = P.rf + 3 * n;
    P.colidx = P.rb + 3 * n;
    return P;
}

// rows in increasing index within each level (deterministic); ptr gets the
// level boundaries; one thread
__device__ __forceinline__ int level_sort(const int* __restrict__ lev, int n, int* __restrict__ order,
                                          int* __restrict__ ptr)
{
    int nl = 0;
    for (int i = 0; i < n; ++i) nl = max(nl, lev[i] + 1);
    for (int l = 0; l <= nl; ++l) ptr[l] = 0;
    for (int i = 0; i < n; ++i) ptr[lev[i] + 1]++;
    for (int l = 0; l < nl; ++l) ptr[l + 1] += ptr[l];
    for (int i = 0; i < n; ++i) order[ptr[lev[i]]++] = i;
    for (int l = nl; l > 0; --l) ptr[l] = ptr[l - 1];
    ptr[0] = 0;
    return nl;
}

// CTA: reciprocal diagonal, CSR of L below the diagonal and both level
// schedules; after csc_cta (colptr/rowidx complete)
__device__ __forceinline__ void solve_plan_cta(const double* __restrict__ L, int n, const int* __restrict__ colptr,
                                               const int* __restrict__ rowidx, double* __restrict__ rdiag,
                                               int* plan_base)
{
    const SolvePlan P = solve_plan_view(plan_base, n);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) rdiag[i] = 1.0 / L[(long long)i * n + i];
    for (int i = warp; i < n; i += nw) {
        int cnt = 0;
        for (int j0 = 0; j0 < i; j0 += 32) {
            const int j = j0 + lane;
            cnt += __popc(__ballot_sync(0xffffffffu, j < i && L[(long long)i * n + j] != 0.0));
        }
        if (lane == 0) P.rowptr[i + 1] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        P.rowptr[0] = 0;
        for (int i = 0; i < n; ++i) P.rowptr[i + 1] += P.rowptr[i];
    }
    __syncthreads();
    for (int i = warp; i < n; i += nw) {
        int pos = P.rowptr[i];
        for (int j0 = 0; j0 < i; j0 += 32) {
            const int j = j0 + lane;
            const bool nz = j < i && L[(long long)i * n + j] != 0.0;
            const unsigned bal = __ballot_sync(0xffffffffu, nz);
            if (nz) P.colidx[pos + __popc(bal & ((1u << lane) - 1u))] = j;
            pos += __popc(bal);
        }
    }
    __syncthreads();
    // forward levels: 1 + the largest level among the row's columns
    if (warp == 0) {
        for (int i = 0; i < n; ++i) {
            int m = -1;
            for (int q = P.rowptr[i] + lane; q < P.rowptr[i + 1]; q += 32) m = max(m, P.lev[P.colidx[q]]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == 0) P.lev[i] = m + 1;
            __syncwarp();
        }
        if (lane == 0) P.nlev[0] = level_sort(P.lev, n, P.forder, P.fptr);
        __syncwarp();
        // backward levels: 1 + the largest level among the column's rows
        for (int i = n - 1; i >= 0; --i) {
            int m = -1;
            for (int q = colptr[i] + lane; q < colptr[i + 1]; q += 32) m = max(m, P.lev[rowidx[q]]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == 0) P.lev[i] = m + 1;
            __syncwarp();
        }
        if (lane == 0) P.nlev[1] = level_sort(P.lev, n, P.border, P.bptr);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int i = P.forder[t], k = P.border[t];
        P.rf[3 * t] = i;
        P.rf[3 * t + 1] = P.rowptr[i];
        P.rf[3 * t + 2] = P.rowptr[i + 1];
        P.rb[3 * t] = k;
        P.rb[3 * t + 1] = colptr[k];
        P.rb[3 * t + 2] = colptr[k + 1];
    }
    __syncthreads();
}

// warp: S d = (L L^T)^{-1} d for particle w and phi_w = d^T S d along the
// level schedule: a level of 32 rows or more gives one row per lane (the
// row's sum in column order), a narrower one a group of lanes to each row
// (lane-strided partial sums, then the group's sum)
// perm (may be null): the factor is that of P A P^T with unknown i of the
// factored system = unknown perm[i] of the observations; the sweeps then run
// in that order in scratch (n doubles per particle), d is read through perm
// and the result written back through it
// Lr, Lc (may be null): the factor's values below the diagonal in the order
// of the plan's CSR (colidx) and of the CSC (rowidx), so that a row's or a
// column's products read consecutive doubles instead of scattered entries of
// the dense factor (launch_pack_factor)
// sx (may be null): n doubles of shared memory owned by this warp; the sweeps
// then run there instead of in scratch or x, so that the products of a level
// wait on shared memory, not on L2, for the values of the levels before
__device__ __forceinline__ void solve_levels_warp(const double* __restrict__ L, const int* __restrict__ colptr,
                                                  const int* __restrict__ rowidx, const double* __restrict__ rdiag,
                                                  const int* plan_base, int n, const double* __restrict__ d,
                                                  double* __restrict__ x, double* __restrict__ phi, int w,
                                                  const int* __restrict__ perm = nullptr,
                                                  double* __restrict__ scratch = nullptr,
                                                  const double* __restrict__ Lr = nullptr,
                                                  const double* __restrict__ Lc = nullptr, double* sx = nullptr)
{
    const SolvePlan P = solve_plan_view(const_cast<int*>(plan_base), n);
    const int lane = threadIdx.x & 31;
    double* xp = sx ? sx : (perm ? scratch : x) + (long long)w * n;
    const double* dp = d + (long long)w * n;
    auto dval = [&](int i) { return perm ? dp[perm[i]] : dp[i]; };
    // entry q of row i (column j) of the CSR; entry q of column i (row k) of the CSC
    auto lrow = [&](int q, int i, int j) { return Lr ? Lr[q] : L[(long long)i * n + j]; };
    auto lcol = [&](int q, int i, int k) { return Lc ? Lc[q] : L[(long long)k * n + i]; };
    // the right-hand side in the order of the factored system; the forward
    // sweep then overwrites it row by row
    for (int i = lane; i < n; i += 32) xp[i] = dval(i);
    __syncwarp();
    // One sweep over the levels lv[0..nl] of a level order whose position t
    // holds row (or column) ri[3t] with entries ri[3t+1]..ri[3t+2] (index
    // idx[q], value val(q, i, idx[q])).  A level of m < 32 rows gives each row
    // a group of g = 32 / 2^ceil(log2 m) lanes (lane-strided partial sums in
    // entry order, then the group's sum), a wider one a lane per row, in
    // rounds of 32 rows.  None of the loads but those of xp depends on an
    // earlier level, so they are issued ahead: while level l is summed, the
    // first batch of entries and the diagonal of level l+1, the row
    // descriptors of level l+2 and the bounds of level l+3 are in flight.
    constexpr int U = 8;
    auto sweep = [&](const int* __restrict__ lv, int nl, const int* __restrict__ ri, const int* __restrict__ idx,
                     auto val) {
        auto bound = [&](int k) { return lv[k < nl ? k : nl]; };
        auto log_group = [](int m) { return m >= 32 ? 0 : 5 - (m <= 1 ? 0 : 32 - __clz(m - 1)); };
        // this lane's first row of a level: {i (-1: none), first entry, end}
        auto fetch_row = [&](int lo, int hi, int& i, int& q0, int& q1) {
            const int lg = log_group(hi - lo);
            const int t = lo + (lane >> lg);
            i = -1;
            q0 = q1 = 0;
            if (t < hi) {
                i = ri[3 * t];
                q0 = ri[3 * t + 1] + (lane & ((1 << lg) - 1));
                q1 = ri[3 * t + 2];
            }
        };
        auto fetch_batch = [&](int i, int q0, int q1, int g, int* jj, double* vv) {
#pragma unroll
            for (int u = 0; u < U; ++u) jj[u] = q0 + u * g < q1 ? idx[q0 + u * g] : -1;
#pragma unroll
            for (int u = 0; u < U; ++u) vv[u] = jj[u] >= 0 ? val(q0 + u * g, i, jj[u]) : 0.0;
        };
        auto sum_batch = [&](const int* jj, const double* vv, double acc) {
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (jj[u] >= 0) acc = fma(vv[u], xp[jj[u]], acc);
            return acc;
        };
        // the row of one round: the prefetched first batch, then the rest
        auto finish_row = [&](int lg, int i, int q0, int q1, const int* jj, const double* vv, double rd) {
            const int g = 1 << lg;
            double acc = 0.0;
            if (i >= 0) {
                // the next batch is in flight while the current one is summed
                int cj[U];
                double cv[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    cj[u] = jj[u];
                    cv[u] = vv[u];
                }
                for (int q = q0 + U * g;; q += U * g) {
                    const bool more = q < q1;
                    int kj[U];
                    double kv[U];
                    if (more) fetch_batch(i, q, q1, g, kj, kv);
                    acc = sum_batch(cj, cv, acc);
                    if (!more) break;
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        cj[u] = kj[u];
                        cv[u] = kv[u];
                    }
                }
            }
            for (int o = g >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (i >= 0 && (lane & (g - 1)) == 0) xp[i] = (xp[i] - acc) * rd;
        };
        // pipeline: level l (bounds, row, batch, diagonal), level l+1 (bounds,
        // row), level l+2 (bounds)
        int lo0 = bound(0), hi0 = bound(1), lo1 = hi0, hi1 = bound(2), lo2 = hi1, hi2 = bound(3);
        int i0, a0, e0, i1, a1, e1;
        fetch_row(lo0, hi0, i0, a0, e0);
        fetch_row(lo1, hi1, i1, a1, e1);
        int j0[U];
        double v0[U];
        fetch_batch(i0, a0, e0, 1 << log_group(hi0 - lo0), j0, v0);
        double rd0 = i0 >= 0 ? rdiag[i0] : 0.0;
        for (int l = 0; l < nl; ++l) {
            // issue the loads of the levels ahead
            int j1[U];
            double v1[U];
            fetch_batch(i1, a1, e1, 1 << log_group(hi1 - lo1), j1, v1);
            const double rd1 = i1 >= 0 ? rdiag[i1] : 0.0;
            int i2, a2, e2;
            fetch_row(lo2, hi2, i2, a2, e2);
            const int hi3 = bound(l + 4);
            // level l: the first round from the prefetched values, further
            // rounds (more than 32 rows) loaded here
            const int lg = log_group(hi0 - lo0);
            finish_row(lg, i0, a0, e0, j0, v0, rd0);
            for (int t = lo0 + 32 + lane; t - lane < hi0; t += 32) {
                int i = -1, q0 = 0, q1 = 0;
                if (t < hi0) {
                    i = ri[3 * t];
                    q0 = ri[3 * t + 1];
                    q1 = ri[3 * t + 2];
                }
                int jj[U];
                double vv[U];
                fetch_batch(i, q0, q1, 1, jj, vv);
                finish_row(0, i, q0, q1, jj, vv, i >= 0 ? rdiag[i] : 0.0);
            }
            __syncwarp();
            // advance the pipeline
            lo0 = lo1; hi0 = hi1; i0 = i1; a0 = a1; e0 = e1; rd0 = rd1;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                j0[u] = j1[u];
                v0[u] = v1[u];
            }
            lo1 = lo2; hi1 = hi2; i1 = i2; a1 = a2; e1 = e2;
            lo2 = hi2; hi2 = hi3;
        }
    };
    // forward: y_i = (d_i - sum_j L_ij y_j) / L_ii
    sweep(P.fptr, P.nlev[0], P.rf, P.colidx, lrow);
    // backward: x_i = (y_i - sum_k L_ki x_k) / L_ii over k > i
    sweep(P.bptr, P.nlev[1], P.rb, rowidx, lcol);
    double acc = 0.0;
    for (int i = lane; i < n; i += 32) acc = fma(dval(i), xp[i], acc);
    acc = warp_sum(acc);
    if (lane == 0) phi[w] = acc;
    if (perm || sx) {
        double* out = x + (long long)w * n;
        for (int i = lane; i < n; i += 32) out[perm ? perm[i] : i] = xp[i];
    }
}

constexpr int DOT_THREADS = 256;
constexpr int DOT_BLOCKS_PER_CTA = 8;

// CTA of DOT_THREADS: partial sums of xi^T xi, nu~^T nu~, nu~^T xi (FP64
// normals) of particle p over the Philox blocks of slice bx
__device__ __forceinline__ void rand_dots_cta(uint64_t seed, uint32_t t, uint32_t s_xi, uint32_t s_nu, int NR,
                                              double* __restrict__ partial, int nblk, int p, int bx)
{
    const uint2 key = seed_key(seed);
    const int nq = (NR + 3) / 4;
    double xx = 0.0, nn = 0.0, nx = 0.0;
    for (int b = bx * DOT_THREADS + threadIdx.x; b < nq; b += nblk * DOT_THREADS) {
        const uint4 wx = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)p, t, s_xi), key);
        const uint4 wn = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)p, t, s_nu), key);
        if (4 * b + 3 < NR) {
            // whole Box-Muller pairs: with z = r (cos, sin)(pi 2u_b) the pair
            // contributes r^2 = -2 log u_a to the squared norm, and to the cross
            // product r_nu r_xi cos(pi (2u_b,nu - 2u_b,xi)); one logarithm per
            // pair, one square root and one cosine per pair of pairs
            const uint32_t xa[2] = {wx.x, wx.z}, xb[2] = {wx.y, wx.w}, na[2] = {wn.x, wn.z}, nb[2] = {wn.y, wn.w};
#pragma unroll
            for (int l = 0; l < 2; ++l) {
                const double rx2 = -2.0 * log(((double)xa[l] + 0.5) * 0x1p-32);
                const double rn2 = -2.0 * log(((double)na[l] + 0.5) * 0x1p-32);
                const double d = ((double)nb[l] - (double)xb[l]) * 0x1p-31;   // 2u_b,nu - 2u_b,xi, exact
                xx += rx2;
                nn += rn2;
                // nu~^T xi sets only the projection coefficient a of eq.
                // nuPerpendicular, not gamma or zeta: its terms are formed in
                // FP32 and summed in FP64
                nx += (double)(sqrtf((float)(rx2 * rn2)) * cospif((float)d));
            }
        } else {
            double x[4], v[4];
            box_muller64(wx.x, wx.y, x[0], x[1]);
            box_muller64(wx.z, wx.w, x[2], x[3]);
            box_muller64(wn.x, wn.y, v[0], v[1]);
            box_muller64(wn.z, wn.w, v[2], v[3]);
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                if (4 * b + l < NR) {
                    xx = fma(x[l], x[l], xx);
                    nn = fma(v[l], v[l], nn);
                    nx = fma(v[l], x[l], nx);
                }
            }
        }
    }
    __shared__ double red[3][DOT_THREADS / 32];
    xx = warp_sum(xx);
    nn = warp_sum(nn);
    nx = warp_sum(nx);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = xx;
        red[1][threadIdx.x >> 5] = nn;
        red[2][threadIdx.x >> 5] = nx;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int w = 0; w < DOT_THREADS / 32; ++w) s += red[threadIdx.x][w];
        partial[((long long)p * nblk + bx) * 3 + threadIdx.x] = s;
    }
}

// -s - log(1 - s) for s in [0, 1): power series below 0.1, closed form above
__device__ __forceinline__ double phi_s(double s)
{
    if (s < 0.1) {
        double acc = 0.0, term = s * s;
        for (int n = 2; n < 40; ++n) {
            acc += term / n;
            term *= s;
        }
        return acc;
    }
    return -s - log1p(-s);
}

// alpha of eq. iewpfAlphaSol with W_0 solved through its defining equation
// u - 1 - log u = q (u = -W_0), q = (x - 1 - log x) + c*/N_psi, x = gamma/N_psi:
// Newton in s = 1 - u started from the branch-point series
// s = p - p^2/3 + 11 p^3/72 - 43 p^4/540, p = sqrt(2 (1 + e z)) (Corless et
// al. 1996), or in u itself for q > 1/2.  Returns alpha, or NaN on failure.
__device__ __forceinline__ double alpha_lambert(double gamma, double cstar, double N)
{
    const double x = gamma / N;
    const double dl = x - 1.0;
    double q = (dl - log1p(dl)) + fmax(cstar, 0.0) / N;
    if (!(q >= 0.0) || !isfinite(q)) return nan("");
    double u;
    if (q == 0.0) {
        u = 1.0;
    } else if (q <= 0.5) {
        const double pp = sqrt(-2.0 * expm1(-q));
        double s = pp * (1.0 + pp * (-1.0 / 3.0 + pp * (11.0 / 72.0 - pp * (43.0 / 540.0))));
        s = fmin(fmax(s, 0.0), 0.999);
        for (int it = 0; it < 8; ++it) {
            const double f = phi_s(s) - q;
            const double fp = s / (1.0 - s);
            if (fp <= 0.0) break;
            double sn = s - f / fp;
            if (sn <= 0.0) sn = 0.5 * s;
            if (sn >= 1.0) sn = 0.5 * (s + 1.0);
            if (sn == s) break;
            s = sn;
        }
        u = 1.0 - s;
    } else {
        u = exp(-1.0 - q);
        for (int it = 0; it < 60; ++it) {
            const double f = u - 1.0 - log(u) - q;
            const double fp = 1.0 - 1.0 / u;
            double un = u - f / fp;
            if (un <= 0.0) un = 0.5 * u;
            if (un >= 1.0) un = 0.5 * (u + 1.0);
            if (un == u) break;
            u = un;
        }
    }
    return u / x;
}

__device__ __forceinline__ void block_sum_min(double v_sum, double v_min, double* s_out, double* m_out)
{
    __shared__ double ws[32], wm[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double s = warp_sum(v_sum);
    double m = v_min;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    __syncthreads();
    if (lane == 0) {
        ws[w] = s;
        wm[w] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ts = 0.0, tm = INFINITY;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            ts += ws[i];
            tm = fmin(tm, wm[i]);
        }
        *s_out = ts;
        *m_out = tm;
    }
    __syncthreads();
}

// Schemes of the ensemble-wide step: the two-stage IEWPF (App. A, eqs.
// betaTwoStage, cistarTwoStage) and the one-stage IEWPF (App. A, eqs.
// iewpf_targetWeight, iewpfCStar), which has no nu and so no beta.
constexpr int TWO_STAGE = 0;
constexpr int ONE_STAGE = 1;

// CTA: the ensemble-wide step.  Two-stage: w_target = mean c_i, beta, c*,
// alpha, -log w.  One-stage: w_target = max c_i, beta reported as 0 (the nu
// term of the posterior vanishes with it), c* = w_target - c_i, alpha, -log w.
// scal[0] = w_target, scal[1] = beta, scal[2] = mean c_i.
__device__ __forceinline__ void weights_cta(const double* c, const double* gamma, const double* zeta, int ne,
                                            double N, int scheme, double* alpha, double* cstar, double* neglogw,
                                            double* scal, int* flag)
{
    __shared__ double s_sum, s_min;
    const bool one = scheme == ONE_STAGE;
    double acc = 0.0, mc = INFINITY;
    bool bad = false;
    for (int i = threadIdx.x; i < ne; i += blockDim.x) {
        acc += c[i];
        mc = fmin(mc, -c[i]);
        bad |= !isfinite(c[i]) || !isfinite(gamma[i]) || (!one && !isfinite(zeta[i]));
    }
    bad = __syncthreads_or(bad);
    block_sum_min(acc, mc, &s_sum, &s_min);
    const double cmean = s_sum / ne;
    const double target = one ? -s_min : cmean;
    double beta = 0.0;
    if (!one) {
        double mn = INFINITY;
        for (int i = threadIdx.x; i < ne; i += blockDim.x) mn = fmin(mn, (target - c[i]) / zeta[i] + 1.0);
        block_sum_min(0.0, mn, &s_sum, &s_min);
        beta = s_min;
    }
    bool dom = false;
    for (int i = threadIdx.x; i < ne; i += blockDim.x) {
        const double cs = one ? target - c[i] : target - c[i] - (beta - 1.0) * zeta[i];
        const double a = alpha_lambert(gamma[i], cs, N);
        dom |= !(a > 0.0) || !isfinite(a);
        alpha[i] = a;
        cstar[i] = cs;
        if (neglogw) {
            const double t = (a - 1.0) * gamma[i] - N * log(a);
            neglogw[i] = one ? t + c[i] : t + (beta - 1.0) * zeta[i] + c[i];
        }
    }
    dom = __syncthreads_or(dom);
    if (threadIdx.x == 0) {
        scal[0] = target;
        scal[1] = beta;
        scal[2] = cmean;
        int f = 0;
        if (bad) f |= FLAG_NONFINITE;
        if (!(beta >= 0.0)) f |= FLAG_BETA;
        if (dom) f |= FLAG_DOMAIN;
        if (f) atomicOr(flag, f);
    }
}

// CTA: gamma, zeta, a, the length scale and c from the partial dot products,
// then the weights step
__device__ __forceinline__ void sync_alpha_cta(const double* __restrict__ phi, const double* __restrict__ partial,
                                               int nblk, int ne, double NR, double N, double logNe, int scheme, double* c,
                                               double* gamma, double* zeta, double* alpha, double* cstar,
                                               double* neglogw, double* coef, double* scal, int* flag)
{
    for (int i = threadIdx.x; i < ne; i += blockDim.x) {
        double xx = 0.0, nn = 0.0, nx = 0.0;
        for (int b = 0; b < nblk; ++b) {
            xx += partial[((long long)i * nblk + b) * 3 + 0];
            nn += partial[((long long)i * nblk + b) * 3 + 1];
            nx += partial[((long long)i * nblk + b) * 3 + 2];
        }
        const double a = nx / xx;                                    // eq. nuPerpendicular
        coef[2 * i] = a;
        coef[2 * i + 1] = sqrt(nn / (nn - a * nx));
        gamma[i] = xx * N / NR;                                      // eq. scalingGammaZeta
        zeta[i] = nn * N / NR;
        c[i] = phi[i] + logNe;                                       // eq. iewpf_ci
    }
    __syncthreads();
    weights_cta(c, gamma, zeta, ne, N, scheme, alpha, cstar, neglogw, scal, flag);
}

// r = beta^{1/2} nu + alpha^{1/2} xi at coarse point m of particle p,
// nu = s (nu~ - a xi)
__device__ __forceinline__ void form_r_one(uint64_t seed, uint32_t t, uint32_t s_xi, uint32_t s_nu, int NR,
                                           const double* __restrict__ coef, const double* __restrict__ scal,
                                           const double* __restrict__ alpha, float* __restrict__ r, int p, int m)
{
    const uint2 key = seed_key(seed);
    const float xi = normal32(key, (uint32_t)p, t, s_xi, (uint32_t)m);
    const float nut = normal32(key, (uint32_t)p, t, s_nu, (uint32_t)m);
    const float a = (float)coef[2 * p], sc = (float)coef[2 * p + 1];
    // square roots in FP32 (the factors enter an FP32 field; an FP64 square
    // root per coarse point would cost more than the rest of the kernel)
    const float sb = sqrtf((float)fmax(scal[1], 0.0)), sa = sqrtf((float)alpha[p]);
    r[(long long)p * NR + m] = fmaf(sb, sc * fmaf(-a, xi, nut), sa * xi);
}

// CTA of at least 64 threads: the 7x7 block roots of every observation of
// particle p applied in observation order (eq. Psquareroot, Sec. 4.6)
__device__ __forceinline__ void block_seq_cta(float* __restrict__ r, int NR, const float* __restrict__ M49,
                                              const int* __restrict__ block0, int nobs, int nRx, int nRy, int p)
{
    __shared__ float v[49];
    __shared__ int idx[49];
    float* rp = r + (long long)p * NR;
    const int t = threadIdx.x;
    for (int l = 0; l < nobs; ++l) {
        __syncthreads();
        if (t < 49) {
            const int dxo = t % 7 - 3, dyo = t / 7 - 3;
            const int a = pmod(block0[2 * l] + dxo, nRx), b = pmod(block0[2 * l + 1] + dyo, nRy);
            idx[t] = b * nRx + a;
            v[t] = rp[idx[t]];
        }
        __syncthreads();
        if (t < 49) {
            float acc = 0.0f;
#pragma unroll 7
            for (int j = 0; j < 49; ++j) acc = fmaf(M49[t * 49 + j], v[j], acc);
            rp[idx[t]] = acc;
        }
    }
    __syncthreads();
}

}  // namespace ana
}  // namespace iewpf
