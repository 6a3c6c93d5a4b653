// Model error and analysis update (Sec. 3.2 and 4.6 of arXiv 1910.01031),
// one problem per launch; the device code is in qhalf_dev.cuh.
#include "qhalf_dev.cuh"

namespace iewpf {

namespace {

// normals of every particle, one Philox block per thread
__global__ void coarse_normals_kernel(QhalfArgs A, long long NR)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (4 * q >= NR) return;
    const int p = blockIdx.y;
    const uint32_t t = A.t_dev ? *A.t_dev : A.t;
    qhalf::normals_block(seed_key(A.seed), (uint32_t)p, t, A.stream, (uint32_t)q, NR, A.xi_buf + (long long)p * NR);
}

// Q_SOAR^{1/2} of every coarse point of every particle
__global__ void coarse_soar_kernel(const float* __restrict__ src, const float* __restrict__ wtab, Grid G, Coarse C,
                                   float* __restrict__ out)
{
    const long long NR = (long long)C.nRx * C.nRy;
    const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= NR) return;
    const int p = blockIdx.y;
    out[(long long)p * NR + m] =
        qhalf::soar_point(src + (long long)p * NR, wtab, C, G, (int)(m % C.nRx), (int)(m / C.nRx));
}

// model error and analysis update on FINE_TX x FINE_TY tiles (the analysis
// update's observation lists are binned by the same tiles)
using qhalf::FINE_TX;
using qhalf::FINE_TY;

template <bool PULL>
__global__ void __launch_bounds__(NTHREADS)
qhalf_fine_kernel(QhalfArgs A, Grid G, Coarse C)
{
    const long long NR = (long long)C.nRx * C.nRy;
    constexpr int TX = FINE_TX, TY = FINE_TY;
    qhalf::fine_tile<PULL, TX, TY>(A, G, C, blockIdx.x * TX, blockIdx.y * TY, blockIdx.z,
                                   blockIdx.y * gridDim.x + blockIdx.x, A.soar_buf + (long long)blockIdx.z * NR);
}

}  // namespace

int qhalf_launches(const QhalfArgs& A)
{
    if (!A.xi_buf || !A.soar_buf) return 0;
    return A.from_philox ? 3 : 2;
}

cudaError_t launch_qhalf(const QhalfArgs& A, const Grid& G, const Coarse& C, cudaStream_t st)
{
    if (C.tab > qhalf::TAB_MAX || !A.xi_buf || !A.soar_buf) return cudaErrorInvalidValue;
    const long long NR = (long long)C.nRx * C.nRy;
    const float* src = A.x;
    if (A.from_philox) {
        const long long nq = (NR + 3) / 4;
        coarse_normals_kernel<<<dim3((unsigned)((nq + 255) / 256), G.ne), 256, 0, st>>>(A, NR);
        src = A.xi_buf;
    }
    coarse_soar_kernel<<<dim3((unsigned)((NR + 255) / 256), G.ne), 256, 0, st>>>(src, A.wtab, G, C, A.soar_buf);
    const dim3 grid((G.nx + FINE_TX - 1) / FINE_TX, (G.ny + FINE_TY - 1) / FINE_TY, G.ne);
    if (A.with_pull) qhalf_fine_kernel<true><<<grid, NTHREADS, 0, st>>>(A, G, C);
    else qhalf_fine_kernel<false><<<grid, NTHREADS, 0, st>>>(A, G, C);
    return cudaGetLastError();
}

}  // namespace iewpf
