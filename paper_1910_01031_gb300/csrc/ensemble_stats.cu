// Ensemble statistics outside the IEWPF update: the weights of the standard
// particle filter (Sec. 2.1) against many subsets of one observation set, as
// in the collapse experiment of Sec. 5.3.
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

}  // namespace

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
