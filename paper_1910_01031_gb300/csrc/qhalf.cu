// Model error and analysis update (Sec. 3.2 and 4.6 of arXiv 1910.01031),
// one problem per launch; the device code is in qhalf_dev.cuh.
#include "qhalf_dev.cuh"

namespace iewpf {

namespace {

template <bool PULL>
__global__ void __launch_bounds__(NTHREADS)
qhalf_kernel(QhalfArgs A, Grid G, Coarse C)
{
    qhalf::qhalf_tile<PULL>(A, G, C, blockIdx.x * TW, blockIdx.y * TH, blockIdx.z, blockIdx.y * gridDim.x + blockIdx.x,
                            A.t_dev ? *A.t_dev : A.t);
}

}  // namespace

cudaError_t launch_qhalf(const QhalfArgs& A, const Grid& G, const Coarse& C, cudaStream_t st)
{
    if (C.tab > qhalf::TAB_MAX) return cudaErrorInvalidValue;
    dim3 grid((G.nx + TW - 1) / TW, (G.ny + TH - 1) / TH, G.ne);
    if (A.with_pull) qhalf_kernel<true><<<grid, NTHREADS, 0, st>>>(A, G, C);
    else qhalf_kernel<false><<<grid, NTHREADS, 0, st>>>(A, G, C);
    return cudaGetLastError();
}

}  // namespace iewpf
