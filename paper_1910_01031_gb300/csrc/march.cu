// Register-marching scheme step (Sec. 3.1 of arXiv 1910.01031), one problem
// per launch; the device code is in march_dev.cuh.
#include "march_dev.cuh"

namespace iewpf {

namespace {

template <int NC>
__global__ void __launch_bounds__(256)
rk2_march_kernel(march::StepArgs a, int s)
{
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long per_p = (long long)a.n_strips * a.n_chunks;
    if (warp >= per_p * a.G.ne) return;
    const int p = (int)(warp / per_p);
    const int rem = (int)(warp % per_p);
    march::march_warp<NC>(a, p, rem / a.n_strips, rem % a.n_strips, a.s_dev ? *a.s_dev : s);
}

template <int NC>
__global__ void __launch_bounds__(256)
rk2_march2_kernel(march::StepArgs a, int s)
{
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long per_p = (long long)a.n_strips * a.n_chunks;
    if (warp >= per_p * a.G.ne) return;
    const int p = (int)(warp / per_p);
    const int rem = (int)(warp % per_p);
    march::march_warp_paired<NC>(a, p, rem / a.n_strips, rem % a.n_strips, a.s_dev ? *a.s_dev : s);
}

template <int NC>
cudaError_t launch_nc(float* b0, float* b1, const int* par, const int* nsub, const float* dtp, int s, const Grid& G,
                      int TH, int warps_per_cta, int paired, const int* s_dev, cudaStream_t st)
{
    constexpr int WUSE = 32 * NC - 8;
    march::StepArgs a{b0, b1, par, nsub, dtp, G, TH, (G.nx + WUSE - 1) / WUSE, (G.ny + TH - 1) / TH, s_dev};
    const long long warps = (long long)a.n_strips * a.n_chunks * G.ne;
    const long long blocks = (warps + warps_per_cta - 1) / warps_per_cta;
    if (paired)
        rk2_march2_kernel<NC><<<(unsigned)blocks, 32 * warps_per_cta, 0, st>>>(a, s);
    else
        rk2_march_kernel<NC><<<(unsigned)blocks, 32 * warps_per_cta, 0, st>>>(a, s);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rk2_march(float* b0, float* b1, const int* par, const int* nsub, const float* dtp, int s,
                             const Grid& G, const MarchShape& shape, cudaStream_t st,
                             const int* s_dev)
{
    if (shape.TH < 1 || shape.warps < 1 || shape.warps > 8) return cudaErrorInvalidValue;
    switch (shape.nc) {
    case 2: return launch_nc<2>(b0, b1, par, nsub, dtp, s, G, shape.TH, shape.warps, shape.paired, s_dev, st);
    case 3: return launch_nc<3>(b0, b1, par, nsub, dtp, s, G, shape.TH, shape.warps, shape.paired, s_dev, st);
    case 4: return launch_nc<4>(b0, b1, par, nsub, dtp, s, G, shape.TH, shape.warps, shape.paired, s_dev, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace iewpf
