// Shared device helpers of the IEWPF kernels: problem constants, the
// counter-based Philox4x32-10 generator with Box-Muller normals, and the
// geometry of the coarse random-number grid Omega^R.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace iewpf {

// Tile of the fine model-error and analysis-update kernels, and of the
// observation lists of the pull.
constexpr int OBS_TX = 64;
constexpr int OBS_TY = 32;
constexpr int NTHREADS = 256;
// Capacity of a tile's observation list (observations whose pull stencil
// reaches the tile); more give FLAG_TILE_OVERFLOW.
constexpr int MAX_TILE_OBS = 256;

// Fine-grid constants in float, precomputed on the host.
struct Grid {
    int nx, ny;
    float dx, dy, g, f, H, theta;
    float inv_dx, inv_dy;
    float fdx, fdy;            // f dx, f dy
    float fdx_half, fdy_half;  // f dx / 2, f dy / 2
    float inv_2g;
    float sgh;                 // g H / f (geostrophic balance)
    float inv_2dx, inv_2dy;
    // exact doublings / halvings of the above for the marching kernel, whose
    // slopes are carried as twice their value; g/2 and g H for the pressure
    float theta2, fdx2, fdy2, inv_4g;
    float g_half, gH;
    int ne;
    long long plane;           // nx * ny
};

// Coarse grid Omega^R: points at fine index o + c a, a = 0..nR-1, periodic.
struct Coarse {
    int c, o, nRx, nRy;
    int tab;                   // side of the SOAR weight table (fine offsets)
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
// (L, R) <- (hi(M R) ^ key ^ other, lo(M R)) on the two lanes, key bumped by
// the Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint2 seed_key(uint64_t seed)
{
    return make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
}

// Box-Muller in double: u = (k + 1/2) 2^-32, r = sqrt(-2 ln u_a),
// theta = 2 pi u_b; (r cos theta, r sin theta), the angle taken as pi (2 u_b)
// (2 u_b is exact, so no rounding of 2 pi u_b enters).
__device__ __forceinline__ void box_muller64(uint32_t a, uint32_t b, double& z0, double& z1)
{
    const double ua = ((double)a + 0.5) * 0x1p-32;
    const double ub2 = ((double)b + 0.5) * 0x1p-31;   // 2 u_b
    const double r = sqrt(-2.0 * log(ua));
    double s, c;
    sincospi(ub2, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

// The same pair in float.  For u_a > 1/2 the logarithm is taken as
// log1p(-(1 - u_a)) with 1 - u_a = (~a + 1/2) 2^-32 formed exactly, so the
// radius keeps full float precision next to u_a = 1.
__device__ __forceinline__ void box_muller32(uint32_t a, uint32_t b, float& z0, float& z1)
{
    float l;
    if (a < 0x80000000u) l = logf(((float)a + 0.5f) * 0x1p-32f);
    else l = log1pf(-(((float)(~a) + 0.5f) * 0x1p-32f));
    const float r = sqrtf(-2.0f * l);
    const float ub2 = ((float)b + 0.5f) * 0x1p-31f;   // 2 u_b
    float s, c;
    sincospif(ub2, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

// Normal number m of a stream: Philox block m/4, lane m%4 (pairs (0,1), (2,3)).
__device__ __forceinline__ float normal32(uint2 key, uint32_t p, uint32_t t, uint32_t stream, uint32_t m)
{
    const uint4 w = philox4x32_10(make_uint4(m >> 2, p, t, stream), key);
    float z0, z1;
    if ((m & 2u) == 0u) box_muller32(w.x, w.y, z0, z1);
    else box_muller32(w.z, w.w, z0, z1);
    return (m & 1u) ? z1 : z0;
}

__device__ __forceinline__ int floor_div(int a, int n)
{
    return a >= 0 ? a / n : -((-a + n - 1) / n);
}

__device__ __forceinline__ int pmod(int a, int n)
{
    int r = a % n;
    return r < 0 ? r + n : r;
}

// Fine index of coarse point a (any integer) in the periodic extension.
__device__ __forceinline__ int coarse_pos(int a, int nR, int c, int o, int n)
{
    const int w = floor_div(a, nR);
    return o + c * (a - w * nR) + w * n;
}

// Coarse interval [X(a), X(a+1)) holding fine index j (any integer, periodic
// extension); returns a (extended index) and the local coordinate t.
__device__ __forceinline__ int coarse_interval(int j, int nR, int c, int o, int n, float& t)
{
    const int w = floor_div(j, n);
    const int jm = j - w * n;
    int a = (jm < o) ? -1 : min((jm - o) / c, nR - 1);
    const int x0 = coarse_pos(a, nR, c, o, n);
    const int x1 = coarse_pos(a + 1, nR, c, o, n);
    t = (float)(jm - x0) / (float)(x1 - x0);
    return a + w * nR;
}

// Catmull-Rom (Keys, a = -1/2) weights of taps a-1, a, a+1, a+2.
__device__ __forceinline__ void cubic_weights(float t, float w[4])
{
    const float t2 = t * t, t3 = t2 * t;
    w[0] = 0.5f * (-t3 + 2.0f * t2 - t);
    w[1] = 0.5f * (3.0f * t3 - 5.0f * t2 + 2.0f);
    w[2] = 0.5f * (-3.0f * t3 + 4.0f * t2 + t);
    w[3] = 0.5f * (t3 - t2);
}

// max((|u| + c)/dx, (|v| + c)/dy) of one cell, c = sqrt(g h) (eq. swecfl),
// with the hardware reciprocal and square root (a few ulp: only the ceiling
// of dt_model over the CFL step is used, which such errors move only at
// exact ties)
__device__ __forceinline__ float cfl_of(float eta, float hu, float hv, const Grid& G)
{
    const float h = G.H + eta;
    float r, c;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(h));
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(c) : "f"(G.g * h));
    return fmaxf(fmaf(fabsf(hu), r, c) * G.inv_dx, fmaf(fabsf(hv), r, c) * G.inv_dy);
}

__device__ __forceinline__ float cfl_cell(const float* __restrict__ U, long long i, const Grid& G)
{
    return cfl_of(U[i], U[G.plane + i], U[2 * G.plane + i], G);
}

// scheme steps per model step: n_sub = ceil(dt_model / dt_cfl),
// dt_cfl = courant / 4 / amax
__device__ __forceinline__ int nsub_of(float amax, double courant, double dt_model, int fixed)
{
    if (fixed > 0) return fixed;
    const double dtc = courant * 0.25 / (double)amax;
    int n = (int)ceil(dt_model / dtc);
    return (n >= 1) ? n : 1;
}

__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace iewpf
