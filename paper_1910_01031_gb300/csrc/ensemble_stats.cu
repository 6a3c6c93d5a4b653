// Ensemble statistics outside the IEWPF update: the weights of the standard
// particle filter (Sec. 2.1) against many subsets of one observation set, as
// in the collapse experiment of Sec. 5.3, and the ranks of observed values
// within the ensemble (Sec. 5.1, rank histograms).
#include <math.h>

#include "kernels.h"

namespace iewpf {
namespace {

constexpr int SIR_THREADS = 256;

__device__ __forceinline__ double sir_block_min(double v, double* sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = INFINITY;
    for (int w = 0; w < SIR_THREADS / 32; ++w) r = fmin(r, sh[w]);
    return r;
}

__device__ __forceinline__ double sir_block_sum(double v, double* sh)
{
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    for (int w = 0; w < SIR_THREADS / 32; ++w) r += sh[w];
    return r;
}

// One CTA per observation subset s (grid-stride over subsets).  For every
// particle i: l_i = |d_i restricted to the subset|^2 / (2 r_scale sigma^2),
// the exponent of eq. standardParticleFilterWeight with R = r_scale sigma^2 I;
// w_i = exp(-(l_i - min_j l_j)) normalised to sum 1 (eq.
// standardParticleFilter; the common factor exp(-min l) cancels), and the
// count of particles with w_i > 1/N_e.  d: [ne][nobs][2]; sets:
// [n_sets][set_size]; w: [n_sets][ne]; kept: [n_sets].
__global__ void __launch_bounds__(SIR_THREADS)
sir_weights_kernel(const double* __restrict__ d, int ne, int nobs, const int* __restrict__ sets, int n_sets,
                   int set_size, double inv2R, double* __restrict__ w, int* __restrict__ kept)
{
    __shared__ double sh[SIR_THREADS / 32];
    for (int s = blockIdx.x; s < n_sets; s += gridDim.x) {
        const int* S = sets + (long long)s * set_size;
        double* ws = w + (long long)s * ne;
        double lmin = INFINITY;
        for (int i = threadIdx.x; i < ne; i += SIR_THREADS) {
            const double* di = d + (long long)i * nobs * 2;
            double acc = 0.0;
            for (int k = 0; k < set_size; ++k) {
                const int o = S[k];
                acc = fma(di[2 * o], di[2 * o], acc);
                acc = fma(di[2 * o + 1], di[2 * o + 1], acc);
            }
            const double l = acc * inv2R;
            ws[i] = l;
            lmin = fmin(lmin, l);
        }
        lmin = sir_block_min(lmin, sh);
        double sum = 0.0;
        for (int i = threadIdx.x; i < ne; i += SIR_THREADS) {
            const double e = exp(-(ws[i] - lmin));
            ws[i] = e;
            sum += e;
        }
        sum = sir_block_sum(sum, sh);
        const double thr = 1.0 / ne;
        double cnt = 0.0;
        for (int i = threadIdx.x; i < ne; i += SIR_THREADS) {
            const double wi = ws[i] / sum;
            ws[i] = wi;
            cnt += wi > thr ? 1.0 : 0.0;
        }
        cnt = sir_block_sum(cnt, sh);
        if (threadIdx.x == 0) kept[s] = (int)cnt;
        __syncthreads();
    }
}

// One warp per observed value q = 2 m + comp (point m, comp 0 for hu, 1 for
// hv), lanes over particles.  Rank = #{i : U_i(1 + comp, cell_m) + sigma
// eps_{i,q} < y_q}, eps_{i,q} the FP64 normal number q of particle i's
// Philox stream (draw t): the members perturbed by the observation error
// and the observed value inserted into their sorted list (Sec. 5.1).
__global__ void rank_kernel(const float* __restrict__ b0, const float* __restrict__ b1, const int* __restrict__ par,
                            Grid G, const int* __restrict__ cells, const double* __restrict__ y, int nq,
                            uint64_t seed, uint32_t t, uint32_t stream, double sigma, int* __restrict__ ranks)
{
    const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (q >= nq) return;
    const int m = q >> 1, comp = q & 1;
    const long long cell = (long long)cells[2 * m + 1] * G.nx + cells[2 * m];
    const double yq = y[q];
    const uint2 key = seed_key(seed);
    int cnt = 0;
    for (int i = lane; i < G.ne; i += 32) {
        const float* U = (par[i] ? b1 : b0) + (long long)i * 3 * G.plane;
        const uint4 w = philox4x32_10(make_uint4((uint32_t)q >> 2, (uint32_t)i, t, stream), key);
        const bool hi = (q & 2) != 0;
        double z0, z1;
        box_muller64(hi ? w.z : w.x, hi ? w.w : w.y, z0, z1);
        const double v = fma(sigma, (q & 1) ? z1 : z0, (double)U[(long long)(1 + comp) * G.plane + cell]);
        cnt += v < yq ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) ranks[q] = cnt;
}

}  // namespace

cudaError_t launch_rank(const float* b0, const float* b1, const int* par, const Grid& G, const int* cells,
                        const double* y, int npts, uint64_t seed, uint32_t t, uint32_t stream, double sigma,
                        int* ranks, cudaStream_t st)
{
    const int nq = 2 * npts;
    if (nq <= 0) return cudaSuccess;
    rank_kernel<<<(nq + 7) / 8, 256, 0, st>>>(b0, b1, par, G, cells, y, nq, seed, t, stream, sigma, ranks);
    return cudaGetLastError();
}

cudaError_t launch_sir_weights(const double* d, int ne, int nobs, const int* sets, int n_sets, int set_size,
                               double inv2R, double* w, int* kept, cudaStream_t st)
{
    if (n_sets <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = n_sets < 8 * sms ? n_sets : 8 * sms;
    sir_weights_kernel<<<grid, SIR_THREADS, 0, st>>>(d, ne, nobs, sets, n_sets, set_size, inv2R, w, kept);
    return cudaGetLastError();
}

}  // namespace iewpf
