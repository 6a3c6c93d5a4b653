// Per-particle services of the shallow-water ensemble stepper (Sec. 3.1 of
// arXiv 1910.01031; the scheme step itself is in march.cu): the CFL
// reduction (eq. swecfl), drifter advection, the drift-forecast errors and
// the state scan for non-finite values.
#include "common.cuh"
#include "kernels.h"

namespace iewpf {

namespace {

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
                            int* __restrict__ maxsub, int ne, double courant, double dt_model, int fixed,
                            int* __restrict__ flag)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= ne) return;
    int n = nsub_of(amax[p], courant, dt_model, fixed);
    if (flag && n > kMaxSubSingle) {
        // a non-finite or runaway state: cap the count so that a device-side
        // loop over the scheme steps ends, and report it
        n = kMaxSubSingle;
        atomicOr(flag, (int)FLAG_NONFINITE);
    }
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
                             double dx, double dy, const int* __restrict__ s_dev)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G.ne * nd) return;
    if (s_dev) s = *s_dev;
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
    const long long n = 3 * G.plane;
    long long i0 = 0;
    if ((G.plane & 3) == 0) {
        // four values per load (the particle's state starts 16-byte aligned)
        const float4* __restrict__ U4 = reinterpret_cast<const float4*>(U);
        for (long long i = (long long)blockIdx.x * NTHREADS + threadIdx.x; i < n / 4;
             i += (long long)gridDim.x * NTHREADS) {
            const float4 v = __ldcs(U4 + i);
            bad |= !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w));
        }
        i0 = n;
    }
    for (long long i = i0 + (long long)blockIdx.x * NTHREADS + threadIdx.x; i < n; i += (long long)gridDim.x * NTHREADS)
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

cudaError_t launch_cfl(const float* b0, const float* b1, const int* par, float* amax, int* nsub, float* dtp,
                       int* maxsub, const Grid& G, double courant, double dt_model, int fixed,
                       cudaStream_t st, bool have_amax, int* flag)
{
    if (!have_amax) cudaMemsetAsync(amax, 0, sizeof(float) * G.ne, st);
    cudaMemsetAsync(maxsub, 0, sizeof(int), st);
    if (fixed <= 0 && !have_amax) {
        const long long blocks = (G.plane + NTHREADS * 8 - 1) / (NTHREADS * 8);
        dim3 grid((unsigned)(blocks < 1 ? 1 : (blocks > 4096 ? 4096 : blocks)), G.ne);
        cfl_kernel<<<grid, NTHREADS, 0, st>>>(b0, b1, par, amax, G);
    }
    nsub_kernel<<<(G.ne + 127) / 128, 128, 0, st>>>(amax, nsub, dtp, maxsub, G.ne, courant, dt_model, fixed, flag);
    return cudaGetLastError();
}

cudaError_t launch_par_update(int* par, const int* nsub, int ne, unsigned long long* work, cudaStream_t st)
{
    par_update_kernel<<<(ne + 127) / 128, 128, 0, st>>>(par, nsub, ne, work);
    return cudaGetLastError();
}

cudaError_t launch_drift(const float* b0, const float* b1, const int* par, const int* nsub, const float* dtp,
                         double* xy, int nd, int s, const Grid& G, double dx, double dy, cudaStream_t st,
                         const int* s_dev)
{
    const int n = G.ne * nd;
    drift_kernel<<<(n + 127) / 128, 128, 0, st>>>(b0, b1, par, nsub, dtp, xy, nd, s, G, dx, dy, s_dev);
    return cudaGetLastError();
}

namespace {
__global__ void step_reset_kernel(int* s_dev) { *s_dev = 0; }

// advances the scheme-step index and sets the loop's condition; the cap keeps
// the loop finite whatever the largest n_sub holds
__global__ void step_ctl_kernel(int* s_dev, const int* maxsub, cudaGraphConditionalHandle h, unsigned int* iters)
{
    const int s = *s_dev + 1;
    *s_dev = s;
    if (iters) *iters += 1u;
    cudaGraphSetConditional(h, (s < *maxsub && s < kMaxSubSingle) ? 1u : 0u);
}

__global__ void counter_inc_kernel(uint32_t* t) { *t += 1u; }
}  // namespace

cudaError_t launch_step_reset(int* s_dev, cudaStream_t st)
{
    step_reset_kernel<<<1, 1, 0, st>>>(s_dev);
    return cudaGetLastError();
}

cudaError_t launch_step_ctl(int* s_dev, const int* maxsub, cudaGraphConditionalHandle h, unsigned int* iters,
                            cudaStream_t st)
{
    step_ctl_kernel<<<1, 1, 0, st>>>(s_dev, maxsub, h, iters);
    return cudaGetLastError();
}

cudaError_t launch_counter_inc(uint32_t* t_dev, cudaStream_t st)
{
    counter_inc_kernel<<<1, 1, 0, st>>>(t_dev);
    return cudaGetLastError();
}

cudaError_t launch_nonfinite(const float* b0, const float* b1, const int* par, const Grid& G, int* flag,
                             cudaStream_t st)
{
    const long long blocks = (3 * G.plane + NTHREADS * 32 - 1) / (NTHREADS * 32);
    dim3 grid((unsigned)(blocks < 1 ? 1 : (blocks > 1024 ? 1024 : blocks)), G.ne);
    nonfinite_kernel<<<grid, NTHREADS, 0, st>>>(b0, b1, par, G, flag);
    return cudaGetLastError();
}

}  // namespace iewpf
