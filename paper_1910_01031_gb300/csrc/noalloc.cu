// iewpf_weights_noalloc: the ensemble-wide weights step of iewpf_weights run
// out of a fixed device scratch array instead of memory from cudaMalloc.
//
// The scratch is one file-scope __device__ array that every GPU loading the
// library holds until the process exits.  Host code must not use its name as
// a device address (in host code it is only a stand-in symbol), so every call
// looks the address up with cudaGetSymbolAddress while the caller's device is
// current.  Nothing is cached: a context torn down and created again (after
// cudaDeviceReset, say) loads the module at a new address, and the next call
// sees it.
#include "../../include/iewpf.h"
#include "common.cuh"
#include "kernels.h"

namespace {

// layout: c, gamma, zeta, alpha, c*, -log w (IEWPF_WEIGHTS_NOALLOC_MAX_NE
// doubles each), then c_bar and beta (4 doubles), then the error flag
constexpr int kMax = IEWPF_WEIGHTS_NOALLOC_MAX_NE;
constexpr int kScal = 6 * kMax;
constexpr int kFlag = 6 * kMax + 4;
constexpr int kDoubles = 6 * kMax + 8;

static __device__ __align__(256) double g_weights_scratch[kDoubles];

// Device address of the scratch in the current device's context.
int scratch_address(double** out)
{
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_weights_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return IEWPF_ECUDA;
    }
    *out = static_cast<double*>(p);
    return IEWPF_OK;
}

}  // namespace

extern "C" int iewpf_weights_noalloc(int ne, double N_psi, const double* c, const double* gamma,
                                     const double* zeta, double* out2, double* alpha, double* cstar,
                                     double* neglogw)
{
    if (ne < 1 || ne > kMax || !(N_psi > 0) || !c || !gamma || !zeta || !out2 || !alpha || !cstar)
        return IEWPF_EINVAL;
    double* s = nullptr;
    int rc = scratch_address(&s);
    if (rc != IEWPF_OK) return rc;
    const size_t n = (size_t)ne;
    double *dc = s, *dg = s + kMax, *dz = s + 2 * kMax, *da = s + 3 * kMax, *ds = s + 4 * kMax,
           *dw = s + 5 * kMax, *dsc = s + kScal;
    int* flag = reinterpret_cast<int*>(s + kFlag);
    int hf = 0;
    // the flag keeps the last call's value: clear it first
    if (cudaMemset(flag, 0, sizeof(int)) != cudaSuccess ||
        cudaMemcpy(dc, c, 8 * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dg, gamma, 8 * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dz, zeta, 8 * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        iewpf::launch_weights_only(dc, dg, dz, ne, N_psi, 0, da, ds, dw, dsc, flag, 0) != cudaSuccess ||
        cudaMemcpy(out2, dsc, 16, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(alpha, da, 8 * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(cstar, ds, 8 * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
        (neglogw && cudaMemcpy(neglogw, dw, 8 * n, cudaMemcpyDeviceToHost) != cudaSuccess) ||
        cudaMemcpy(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return IEWPF_ECUDA;
    }
    if (hf & iewpf::FLAG_NONFINITE) return IEWPF_ENONFINITE;
    if (hf & iewpf::FLAG_BETA) return IEWPF_EBETA;
    if (hf & iewpf::FLAG_DOMAIN) return IEWPF_EDOMAIN;
    return IEWPF_OK;
}
