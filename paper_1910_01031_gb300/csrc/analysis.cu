// IEWPF analysis kernels for one problem per launch (Sec. 4 and App. A of
// arXiv 1910.01031); the device code is in analysis_dev.cuh.
#include <algorithm>
#include <vector>

#include "analysis_dev.cuh"

namespace iewpf {

namespace {

__global__ void obs_cells_kernel(const double* __restrict__ xy, int nobs, Grid G, Coarse C, double dx, double dy,
                                 int* __restrict__ cell, int* __restrict__ block0)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l < nobs) ana::obs_cell_one(xy, l, G, C, dx, dy, cell, block0);
}

__global__ void __launch_bounds__(NTHREADS)
tile_bin_kernel(const int* __restrict__ cell, int nobs, Grid G, int R, int* __restrict__ cnt, int* __restrict__ list,
                int cap, int* __restrict__ flag)
{
    ana::tile_bin_cta(cell, nobs, G, R, blockIdx.x, cnt, list, cap, flag);
}

__global__ void innovate_kernel(const float* __restrict__ b0, const float* __restrict__ b1,
                                const int* __restrict__ par, const int* __restrict__ cell,
                                const double* __restrict__ y, int nobs, Grid G, double H, double* __restrict__ d)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < G.ne * nobs) ana::innovate_one(b0, b1, par, cell, y, nobs, G, H, d, i);
}

__global__ void hqht_kernel(const double* __restrict__ K, int R, const int* __restrict__ cell, int nobs, Grid G,
                            int dense, double sigma2, double* __restrict__ M)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 4LL * nobs * nobs) ana::hqht_one(K, R, cell, nobs, G, dense, sigma2, M, i);
}

__global__ void __launch_bounds__(1024)
cholesky_kernel(double* __restrict__ A, int n, int* __restrict__ colptr, int* rowidx, int* __restrict__ flag,
                int* nzlist, double* __restrict__ rdiag, int* plan)
{
    ana::cholesky_cta(A, n, colptr, rowidx, flag, nzlist);
    ana::solve_plan_cta(A, n, colptr, rowidx, rdiag, plan);
}

// the same factorisation on a copy in shared memory (n * n doubles + n ints)
__global__ void __launch_bounds__(1024)
cholesky_small_kernel(double* __restrict__ A, int n, int* __restrict__ colptr, int* __restrict__ rowidx,
                      int* __restrict__ flag, double* __restrict__ rdiag, int* plan)
{
    extern __shared__ double sA[];
    int* work = reinterpret_cast<int*>(sA + (long long)n * n);
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    for (int q = threadIdx.x; q < n * n; q += blockDim.x) sA[q] = A[q];
    __syncthreads();
    ana::cholesky_factor_cta(sA, n, work, &bad);
    for (int q = threadIdx.x; q < n * n; q += blockDim.x) A[q] = sA[q];
    ana::csc_cta(sA, n, colptr, rowidx);
    ana::solve_plan_cta(sA, n, colptr, rowidx, rdiag, plan);
    if (threadIdx.x == 0 && bad) atomicOr(flag, FLAG_NOTPD);
}

// the factor's values below the diagonal in the order of the plan's CSR (Lr)
// and of the CSC (Lc): a warp per row and per column of the dense factor
__global__ void pack_factor_kernel(const double* __restrict__ L, int n, const int* __restrict__ colptr,
                                   const int* __restrict__ rowidx, const int* plan, double* __restrict__ Lr,
                                   double* __restrict__ Lc)
{
    const ana::SolvePlan P = ana::solve_plan_view(const_cast<int*>(plan), n);
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        for (int q = P.rowptr[i] + lane; q < P.rowptr[i + 1]; q += 32) Lr[q] = L[(long long)i * n + P.colidx[q]];
        for (int q = colptr[i] + lane; q < colptr[i + 1]; q += 32) Lc[q] = L[(long long)rowidx[q] * n + i];
    }
}

__global__ void solve_kernel(const double* __restrict__ L, const int* __restrict__ colptr,
                             const int* __restrict__ rowidx, const double* __restrict__ rdiag,
                             const int* __restrict__ plan, int n, const double* __restrict__ d,
                             double* __restrict__ x, double* __restrict__ phi, int ne, const int* __restrict__ perm,
                             double* __restrict__ scratch, const double* __restrict__ Lr, const double* __restrict__ Lc)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp < ne)
        ana::solve_levels_warp(L, colptr, rowidx, rdiag, plan, n, d, x, phi, warp, perm, scratch, Lr, Lc);
}

// the same with a CTA of one warp per particle and its vector in shared
// memory (n doubles)
__global__ void __launch_bounds__(32)
solve_smem_kernel(const double* __restrict__ L, const int* __restrict__ colptr, const int* __restrict__ rowidx,
                  const double* __restrict__ rdiag, const int* __restrict__ plan, int n, const double* __restrict__ d,
                  double* __restrict__ x, double* __restrict__ phi, const int* __restrict__ perm,
                  const double* __restrict__ Lr, const double* __restrict__ Lc)
{
    extern __shared__ double sx[];
    ana::solve_levels_warp(L, colptr, rowidx, rdiag, plan, n, d, x, phi, blockIdx.x, perm, nullptr, Lr, Lc, sx);
}

__global__ void __launch_bounds__(ana::DOT_THREADS)
rand_dots_kernel(uint64_t seed, uint32_t t, uint32_t s_xi, uint32_t s_nu, int NR, double* __restrict__ partial,
                 int nblk)
{
    ana::rand_dots_cta(seed, t, s_xi, s_nu, NR, partial, nblk, blockIdx.y, blockIdx.x);
}

__global__ void __launch_bounds__(1024)
sync_alpha_kernel(const double* __restrict__ phi, const double* __restrict__ partial, int nblk, int ne,
                  double NR, double N, double logNe, int scheme, double* c, double* gamma, double* zeta,
                  double* alpha, double* cstar, double* neglogw, double* coef, double* scal, int* flag)
{
    ana::sync_alpha_cta(phi, partial, nblk, ne, NR, N, logNe, scheme, c, gamma, zeta, alpha, cstar, neglogw, coef,
                        scal, flag);
}

__global__ void __launch_bounds__(1024)
weights_kernel(const double* c, const double* gamma, const double* zeta, int ne, double N, int scheme,
               double* alpha, double* cstar, double* neglogw, double* scal, int* flag)
{
    ana::weights_cta(c, gamma, zeta, ne, N, scheme, alpha, cstar, neglogw, scal, flag);
}

__global__ void form_r_kernel(uint64_t seed, uint32_t t, uint32_t s_xi, uint32_t s_nu, int NR,
                              const double* __restrict__ coef, const double* __restrict__ scal,
                              const double* __restrict__ alpha, float* __restrict__ r)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < NR) ana::form_r_one(seed, t, s_xi, s_nu, NR, coef, scal, alpha, r, blockIdx.y, m);
}

__global__ void block_seq_kernel(float* __restrict__ r, int NR, const float* __restrict__ M49,
                                 const int* __restrict__ block0, int nobs, int nRx, int nRy)
{
    ana::block_seq_cta(r, NR, M49, block0, nobs, nRx, nRy, blockIdx.x);
}

// all levels of the local blocks of particle blockIdx.x: the CTA's warps
// share the blocks of a level, a barrier separates the levels; lane t
// computes outputs t and t + 32 (< 49) with the FMA order of block_seq_cta,
// its two rows of the 49 x 49 root held in registers
constexpr int BL_THREADS = 64;
__global__ void __launch_bounds__(BL_THREADS) block_levels_kernel(float* __restrict__ r, int NR,
                                                                  const float* __restrict__ M49,
                                                                  const int* __restrict__ block0,
                                                                  const int* __restrict__ order,
                                                                  const int* __restrict__ level_off, int nlev,
                                                                  int nRx, int nRy)
{
    __shared__ float v[BL_THREADS / 32][49];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const bool two = lane + 32 < 49;
    float m0[49], m1[49];
#pragma unroll
    for (int j = 0; j < 49; ++j) {
        m0[j] = __ldg(M49 + lane * 49 + j);
        m1[j] = two ? __ldg(M49 + (lane + 32) * 49 + j) : 0.0f;
    }
    float* rp = r + (long long)blockIdx.x * NR;
    for (int lev = 0; lev < nlev; ++lev) {
        const int lo = level_off[lev], hi = level_off[lev + 1];
        for (int ib = lo + wl; ib < hi; ib += BL_THREADS / 32) {
            const int l = order[ib];
            const int cx = block0[2 * l], cy = block0[2 * l + 1];
            const int i0 = pmod(cy + lane / 7 - 3, nRy) * nRx + pmod(cx + lane % 7 - 3, nRx);
            const int t1 = two ? lane + 32 : 48;
            const int i1 = pmod(cy + t1 / 7 - 3, nRy) * nRx + pmod(cx + t1 % 7 - 3, nRx);
            v[wl][lane] = rp[i0];
            if (two) v[wl][lane + 32] = rp[i1];
            __syncwarp();
            float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
            for (int j = 0; j < 49; ++j) {
                const float vj = v[wl][j];
                a0 = fmaf(m0[j], vj, a0);
                a1 = fmaf(m1[j], vj, a1);
            }
            __syncwarp();
            rp[i0] = a0;
            if (two) rp[i1] = a1;
        }
        __syncthreads();     // the next level reads what this one wrote
    }
}

__global__ void philox_blocks_kernel(uint64_t seed, uint32_t p, uint32_t t, uint32_t stream, long long n,
                                     uint4* __restrict__ out)
{
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    out[b] = philox4x32_10(make_uint4((uint32_t)b, p, t, stream), seed_key(seed));
}

__global__ void normals_kernel(uint64_t seed, uint32_t p, uint32_t t, uint32_t stream, long long n,
                               double* __restrict__ o64, float* __restrict__ o32)
{
    const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    const uint2 key = seed_key(seed);
    const uint4 w = philox4x32_10(make_uint4((uint32_t)(m >> 2), p, t, stream), key);
    const bool hi = (m & 2) != 0;
    const uint32_t a = hi ? w.z : w.x, b = hi ? w.w : w.y;
    if (o64) {
        double z0, z1;
        box_muller64(a, b, z0, z1);
        o64[m] = (m & 1) ? z1 : z0;
    }
    if (o32) o32[m] = normal32(key, p, t, stream, (uint32_t)m);
}

}  // namespace

cudaError_t launch_obs_setup(const double* xy, int nobs, const Grid& G, const Coarse& C, double dx, double dy,
                             int R, int* obs_cell, int* obs_block0, int* tile_cnt, int* tile_obs, int tile_cap,
                             int* flag, cudaStream_t st)
{
    if (nobs > 0) obs_cells_kernel<<<(nobs + 127) / 128, 128, 0, st>>>(xy, nobs, G, C, dx, dy, obs_cell, obs_block0);
    const int ntiles = ((G.nx + OBS_TX - 1) / OBS_TX) * ((G.ny + OBS_TY - 1) / OBS_TY);
    tile_bin_kernel<<<ntiles, NTHREADS, 0, st>>>(obs_cell, nobs, G, R, tile_cnt, tile_obs, tile_cap, flag);
    return cudaGetLastError();
}

cudaError_t launch_innovate(const float* b0, const float* b1, const int* par, const int* obs_cell,
                            const double* y, int nobs, const Grid& G, double H, double* d, cudaStream_t st)
{
    const int n = G.ne * nobs;
    if (n > 0) innovate_kernel<<<(n + 127) / 128, 128, 0, st>>>(b0, b1, par, obs_cell, y, nobs, G, H, d);
    return cudaGetLastError();
}

cudaError_t launch_hqht(const double* K64, int R, const int* obs_cell, int nobs, const Grid& G, int dense,
                        double sigma2, double* M, cudaStream_t st)
{
    const long long n = 2LL * nobs * 2 * nobs;
    if (n > 0) hqht_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(K64, R, obs_cell, nobs, G, dense, sigma2, M);
    return cudaGetLastError();
}

cudaError_t launch_cholesky(double* M, int n, int* colptr, int* rowidx, int* flag, double* rdiag, int* plan,
                            cudaStream_t st)
{
    // small systems (drifter layouts change every cycle) factor in shared memory
    const size_t smem = (size_t)n * n * sizeof(double) + (size_t)n * sizeof(int);
    if (n >= 1 && smem <= 200 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(cholesky_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        cholesky_small_kernel<<<1, 1024, smem, st>>>(M, n, colptr, rowidx, flag, rdiag, plan);
        return cudaGetLastError();
    }
    // rowidx doubles as the per-column work list during the factorisation
    cholesky_kernel<<<1, 1024, 0, st>>>(M, n, colptr, rowidx, flag, rowidx, rdiag, plan);
    return cudaGetLastError();
}

cudaError_t launch_solve(const double* L, const int* colptr, const int* rowidx, const double* rdiag, const int* plan,
                         int n, const double* d, double* Sd, double* phi, int ne, cudaStream_t st, const int* perm,
                         double* scratch, const double* Lr, const double* Lc)
{
    if ((perm && !scratch) || (!Lr != !Lc)) return cudaErrorInvalidValue;
    if (ne <= 0) return cudaSuccess;
    if (n > 0 && (size_t)n * sizeof(double) <= kSolveSmemBytes) {
        solve_smem_kernel<<<ne, 32, (size_t)n * sizeof(double), st>>>(L, colptr, rowidx, rdiag, plan, n, d, Sd, phi,
                                                                       perm, Lr, Lc);
        return cudaGetLastError();
    }
    const int threads = 128;
    const int blocks = (ne * 32 + threads - 1) / threads;
    solve_kernel<<<blocks, threads, 0, st>>>(L, colptr, rowidx, rdiag, plan, n, d, Sd, phi, ne, perm, scratch, Lr,
                                             Lc);
    return cudaGetLastError();
}

cudaError_t launch_pack_factor(const double* L, int n, const int* colptr, const int* rowidx, const int* plan,
                               double* Lr, double* Lc, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = std::min((n * 32 + threads - 1) / threads, 65535);
    pack_factor_kernel<<<blocks, threads, 0, st>>>(L, n, colptr, rowidx, plan, Lr, Lc);
    return cudaGetLastError();
}

int rand_dots_blocks(int NR)
{
    const int nq = (NR + 3) / 4;
    int nblk = (nq + ana::DOT_THREADS * ana::DOT_BLOCKS_PER_CTA - 1) / (ana::DOT_THREADS * ana::DOT_BLOCKS_PER_CTA);
    return nblk < 1 ? 1 : nblk;
}

cudaError_t launch_rand_dots(uint64_t seed, uint32_t t, uint32_t s_xi, uint32_t s_nu, int NR, int ne,
                             double* partial, int nblk, cudaStream_t st)
{
    dim3 grid(nblk, ne);
    rand_dots_kernel<<<grid, ana::DOT_THREADS, 0, st>>>(seed, t, s_xi, s_nu, NR, partial, nblk);
    return cudaGetLastError();
}

cudaError_t launch_sync_alpha(const double* phi, const double* partial, int nblk, int ne, double NR,
                              double N_psi, double logNe, int scheme, double* c, double* gamma, double* zeta,
                              double* alpha, double* cstar, double* neglogw, double* coef, double* scal,
                              int* flag, cudaStream_t st)
{
    sync_alpha_kernel<<<1, 1024, 0, st>>>(phi, partial, nblk, ne, NR, N_psi, logNe, scheme, c, gamma, zeta,
                                          alpha, cstar, neglogw, coef, scal, flag);
    return cudaGetLastError();
}

cudaError_t launch_weights_only(const double* c, const double* gamma, const double* zeta, int ne, double N_psi,
                                int scheme, double* alpha, double* cstar, double* neglogw, double* scal, int* flag,
                                cudaStream_t st)
{
    weights_kernel<<<1, 1024, 0, st>>>(c, gamma, zeta, ne, N_psi, scheme, alpha, cstar, neglogw, scal, flag);
    return cudaGetLastError();
}

cudaError_t launch_form_r(uint64_t seed, uint32_t t, uint32_t s_xi, uint32_t s_nu, int NR, int ne,
                          const double* coef, const double* scal, const double* alpha, float* r,
                          cudaStream_t st)
{
    dim3 grid((NR + 255) / 256, ne);
    form_r_kernel<<<grid, 256, 0, st>>>(seed, t, s_xi, s_nu, NR, coef, scal, alpha, r);
    return cudaGetLastError();
}

cudaError_t launch_block_seq(float* r, int NR, int ne, const float* M49, const int* obs_block0, int nobs, int nRx,
                             int nRy, cudaStream_t st)
{
    if (nobs <= 0) return cudaSuccess;
    block_seq_kernel<<<ne, 64, 0, st>>>(r, NR, M49, obs_block0, nobs, nRx, nRy);
    return cudaGetLastError();
}

cudaError_t launch_block_levels(float* r, int NR, int ne, const float* M49, const int* obs_block0, const int* order,
                                const int* level_off, int nlev, int nRx, int nRy, cudaStream_t st)
{
    if (nlev <= 0 || ne <= 0) return cudaSuccess;
    block_levels_kernel<<<ne, BL_THREADS, 0, st>>>(r, NR, M49, obs_block0, order, level_off, nlev, nRx, nRy);
    return cudaGetLastError();
}

void block_levels(const int* block0, int nobs, int nRx, int nRy, std::vector<int>& order, std::vector<int>& level_off)
{
    // two 7-point windows on a circle of n points meet when their centres are
    // at most 6 apart (circular distance)
    auto near = [](int a, int b, int n) {
        int d = a - b;
        if (d < 0) d = -d;
        d %= n;
        return std::min(d, n - d) <= 6;
    };
    std::vector<int> level(nobs, 0);
    int top = 0;
    for (int l = 0; l < nobs; ++l) {
        int lv = 0;
        for (int k = 0; k < l; ++k)
            if (level[k] + 1 > lv && near(block0[2 * k], block0[2 * l], nRx) &&
                near(block0[2 * k + 1], block0[2 * l + 1], nRy))
                lv = level[k] + 1;
        level[l] = lv;
        top = std::max(top, lv);
    }
    level_off.assign(top + 2, 0);
    for (int l = 0; l < nobs; ++l) ++level_off[level[l] + 1];
    for (int v = 0; v <= top; ++v) level_off[v + 1] += level_off[v];
    order.assign(nobs, 0);
    std::vector<int> fill(level_off.begin(), level_off.end() - 1);
    for (int l = 0; l < nobs; ++l) order[fill[level[l]]++] = l;
}

namespace {

// breadth-first levels from `root` over the nodes with mark[v] == stamp;
// returns the levels (lists of nodes) and sets dist[v] for the reached ones
std::vector<std::vector<int>> bfs_levels(const std::vector<std::vector<int>>& adj, const std::vector<int>& mark,
                                         int stamp, int root, std::vector<int>& dist)
{
    std::vector<std::vector<int>> lev;
    lev.push_back({root});
    dist[root] = 0;
    for (;;) {
        std::vector<int> next;
        for (int v : lev.back())
            for (int w : adj[v])
                if (mark[w] == stamp && dist[w] < 0) {
                    dist[w] = (int)lev.size();
                    next.push_back(w);
                }
        if (next.empty()) break;
        lev.push_back(std::move(next));
    }
    return lev;
}

void nd_rec(const std::vector<std::vector<int>>& adj, std::vector<int> nodes, std::vector<int>& mark, int& stamp,
            std::vector<int>& dist, std::vector<int>& out)
{
    if (nodes.size() <= 32) {
        out.insert(out.end(), nodes.begin(), nodes.end());
        return;
    }
    ++stamp;
    for (int v : nodes) {
        mark[v] = stamp;
        dist[v] = -1;
    }
    // a far node of the component of nodes[0]: the last level of a search from it
    std::vector<std::vector<int>> lev = bfs_levels(adj, mark, stamp, nodes[0], dist);
    const int far = lev.back().front();
    for (int v : nodes) dist[v] = -1;
    lev = bfs_levels(adj, mark, stamp, far, dist);
    std::vector<int> rest;                                  // other components
    for (int v : nodes)
        if (dist[v] < 0) rest.push_back(v);
    const int D = (int)lev.size();
    if (D < 3) {
        // too shallow to split: this component as it is, then the rest
        for (const auto& l : lev) out.insert(out.end(), l.begin(), l.end());
        if (!rest.empty()) nd_rec(adj, rest, mark, stamp, dist, out);
        return;
    }
    size_t reached = 0;
    for (const auto& l : lev) reached += l.size();
    int m = 1;
    size_t below = lev[0].size();
    while (m < D - 2 && below + lev[m].size() < reached / 2) below += lev[m++].size();
    std::vector<int> a, b;
    for (int k = 0; k < m; ++k) a.insert(a.end(), lev[k].begin(), lev[k].end());
    for (int k = m + 1; k < D; ++k) b.insert(b.end(), lev[k].begin(), lev[k].end());
    const std::vector<int> sep = lev[m];
    nd_rec(adj, a, mark, stamp, dist, out);
    nd_rec(adj, b, mark, stamp, dist, out);
    if (!rest.empty()) nd_rec(adj, rest, mark, stamp, dist, out);
    out.insert(out.end(), sep.begin(), sep.end());
}

}  // namespace

long long nd_order(const int* cells, int nobs, int nx, int ny, int reach, std::vector<int>& order)
{
    long long pairs = 0;
    auto near = [&](int d, int n) {
        d = d < 0 ? -d : d;
        d %= n;
        return std::min(d, n - d) <= reach;
    };
    std::vector<std::vector<int>> adj(nobs);
    for (int k = 0; k < nobs; ++k)
        for (int l = k + 1; l < nobs; ++l)
            if (near(cells[2 * k] - cells[2 * l], nx) && near(cells[2 * k + 1] - cells[2 * l + 1], ny)) {
                adj[k].push_back(l);
                adj[l].push_back(k);
                ++pairs;
            }
    std::vector<int> nodes(nobs), mark(nobs, 0), dist(nobs, -1);
    for (int k = 0; k < nobs; ++k) nodes[k] = k;
    int stamp = 0;
    order.clear();
    order.reserve(nobs);
    nd_rec(adj, nodes, mark, stamp, dist, order);
    return pairs;
}

cudaError_t launch_philox_blocks(uint64_t seed, uint32_t p, uint32_t t, uint32_t stream, long long n,
                                 uint32_t* out, cudaStream_t st)
{
    if (n > 0)
        philox_blocks_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(seed, p, t, stream, n,
                                                                          reinterpret_cast<uint4*>(out));
    return cudaGetLastError();
}

cudaError_t launch_normals(uint64_t seed, uint32_t p, uint32_t t, uint32_t stream, long long n, double* o64,
                           float* o32, cudaStream_t st)
{
    if (n > 0) normals_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(seed, p, t, stream, n, o64, o32);
    return cudaGetLastError();
}

}  // namespace iewpf
