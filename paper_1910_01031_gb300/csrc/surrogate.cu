// Learned surrogate of the scheme: a periodic 3x3 convolutional network (width
// 64, BF16 weights and activations, FP32 accumulation on the tensor cores)
// that maps the normalised state (eta, hu, hv) to the change of the state over
// k model steps, trained on pairs the plain scheme generates.  Hand-written
// kernels for the forward convolution (implicit GEMM, bias + SiLU fused), the
// backward data pass (the same kernel with the flipped, transposed weights and
// the activation derivative fused), the weight gradients (implicit GEMM over
// pixels, deterministic two-level reduction), the loss, and Adam.
//
// Tensor layout: activations NHWC [batch][ny][nx][C] bf16 with C = 16
// (network input, 3 used) or 64; weights [tap = 3 ky + kx][cout][cin] bf16.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "../../include/iewpf.h"
#include "common.cuh"
#include "kernels.h"
#include "surrogate.h"
#include "tc_dev.cuh"

#include <cuda_bf16.h>

namespace iewpf {

namespace {

constexpr int TROWS = 8, TCOLS = 16;      // pixel tile of the convolution kernels (128 pixels)
// polls of the injected bounded wait (iewpf_surrogate_inject_timeout): a
// few milliseconds, against 2^24 for the pipeline's own waits
constexpr int kInjectedWaitPolls = 1 << 16;
constexpr int CONV_THREADS = 256;

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

// D = A (16x16 bf16, row) * B (16x8 bf16, col) + D, fp32
__device__ __forceinline__ void mma_bf16(float* d, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

enum ConvMode : int {
    MODE_HIDDEN = 0,    // z = conv + b: store z and silu(z) (bf16)
    MODE_OUT = 1,       // out = conv + b: store fp32 (first 3 channels)
    MODE_DGRAD = 2,     // dA = conv(dZ, flipped W^T): store dZ_prev = dA * silu'(z_prev) (bf16)
};

// Implicit-GEMM 3x3 periodic convolution over 8x16 pixel tiles, all COUT
// output channels per CTA, persistent over tiles.  CIN, COUT in {16, 64}.
template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(CONV_THREADS)
conv_kernel(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ W, const float* __restrict__ bias,
            int nb, int ny, int nx, __nv_bfloat16* __restrict__ zout, __nv_bfloat16* __restrict__ aout,
            float* __restrict__ fout, const __nv_bfloat16* __restrict__ zprev)
{
    constexpr int CP = CIN + 8;               // padded channel stride (conflict-free ldmatrix)
    constexpr int PR = TROWS + 2, PC = TCOLS + 2;
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16* Ws = reinterpret_cast<__nv_bfloat16*>(smem);                  // [9][COUT][CP]
    __nv_bfloat16* Ps = Ws + 9 * COUT * CP;                                      // [PR][PC][CP]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // weights once per CTA
    for (int i = tid; i < 9 * COUT * (CIN / 8); i += CONV_THREADS) {
        const int c8 = i % (CIN / 8), row = i / (CIN / 8);
        *reinterpret_cast<uint4*>(Ws + row * CP + c8 * 8) = *reinterpret_cast<const uint4*>(W + row * CIN + c8 * 8);
    }
    const int tiles_x = nx / TCOLS, tiles_y = ny / TROWS;
    const long long ntiles = (long long)nb * tiles_x * tiles_y;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int b = (int)(tile / (tiles_x * tiles_y));
        const int rem = (int)(tile % (tiles_x * tiles_y));
        const int y0 = (rem / tiles_x) * TROWS, x0 = (rem % tiles_x) * TCOLS;
        __syncthreads();
        for (int i = tid; i < PR * PC * (CIN / 8); i += CONV_THREADS) {
            const int c8 = i % (CIN / 8), pix = i / (CIN / 8);
            const int py = pix / PC, px = pix % PC;
            const int gy = pmod(y0 - 1 + py, ny), gx = pmod(x0 - 1 + px, nx);
            *reinterpret_cast<uint4*>(Ps + pix * CP + c8 * 8) =
                *reinterpret_cast<const uint4*>(in + (((long long)b * ny + gy) * nx + gx) * CIN + c8 * 8);
        }
        __syncthreads();
        float acc[COUT / 8][4];
#pragma unroll
        for (int j = 0; j < COUT / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
        // warp w: pixel row w of the tile, 16 pixels
#pragma unroll 1
        for (int tap = 0; tap < 9; ++tap) {
            const int ky = tap / 3, kx = tap % 3;
#pragma unroll
            for (int kc = 0; kc < CIN / 16; ++kc) {
                const int mi = lane >> 3, r = lane & 7;
                const int pc = (mi & 1) * 8 + r + kx;
                const uint32_t aaddr = smem_u32(Ps + ((warp + ky) * PC + pc) * CP + kc * 16 + (mi >> 1) * 8);
                uint32_t a0, a1, a2, a3;
                ldsm_x4(aaddr, a0, a1, a2, a3);
#pragma unroll
                for (int j = 0; j < COUT / 8; j += 2) {
                    const int n = (j + (mi >> 1)) * 8 + r;
                    const uint32_t baddr = smem_u32(Ws + (tap * COUT + n) * CP + kc * 16 + (mi & 1) * 8);
                    uint32_t b0, b1, b2, b3;
                    ldsm_x4(baddr, b0, b1, b2, b3);
                    mma_bf16(acc[j], a0, a1, a2, a3, b0, b1);
                    mma_bf16(acc[j + 1], a0, a1, a2, a3, b2, b3);
                }
            }
        }
        // epilogue: rows lane/4 and lane/4 + 8 of the warp's 16 pixels
        const int gy = y0 + warp;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int gx = x0 + (lane >> 2) + half * 8;
            const long long pix = ((long long)b * ny + gy) * nx + gx;
#pragma unroll
            for (int j = 0; j < COUT / 8; ++j) {
                const int co = j * 8 + (lane & 3) * 2;
                float v0 = acc[j][half * 2], v1 = acc[j][half * 2 + 1];
                if (MODE == MODE_HIDDEN) {
                    v0 += bias[co];
                    v1 += bias[co + 1];
                    *reinterpret_cast<__nv_bfloat162*>(zout + pix * COUT + co) = __floats2bfloat162_rn(v0, v1);
                    *reinterpret_cast<__nv_bfloat162*>(aout + pix * COUT + co) =
                        __floats2bfloat162_rn(silu_act(v0), silu_act(v1));
                } else if (MODE == MODE_OUT) {
                    if (co < 3) fout[pix * 3 + co] = v0 + bias[co];
                    if (co + 1 < 3) fout[pix * 3 + co + 1] = v1 + bias[co + 1];
                } else {
                    const __nv_bfloat162 z = *reinterpret_cast<const __nv_bfloat162*>(zprev + pix * COUT + co);
                    v0 *= silu_grad(__bfloat162float(z.x));
                    v1 *= silu_grad(__bfloat162float(z.y));
                    *reinterpret_cast<__nv_bfloat162*>(aout + pix * COUT + co) = __floats2bfloat162_rn(v0, v1);
                }
            }
        }
    }
}

// Weight gradients of one tap: dW[tap][co][ci] = sum_p dZ[p][co] X[p + off(tap)][ci]
// over the pixel tiles [t0, t1) of CTA (tap, group); partial sums per group.
// PAD: dZ and X in the halo-padded layout [b][ny + 2][nx + 2][C].
template <int CIN, int COUT, bool PAD>
__global__ void __launch_bounds__(CONV_THREADS)
wgrad_kernel(const __nv_bfloat16* __restrict__ dz, const __nv_bfloat16* __restrict__ X, int nb, int ny, int nx,
             int tiles_per_group, float* __restrict__ partial)
{
    constexpr int CPI = CIN + 8, CPO = COUT + 8;
    constexpr int MT = COUT / 16, NT = CIN / 8;          // m16 blocks (co), n8 blocks (ci)
    constexpr int TILES = MT * NT;                        // of the 64x64 (or smaller) output
    constexpr int PER_WARP = (TILES + 7) / 8;
    __shared__ __align__(16) __nv_bfloat16 Ds[TROWS * TCOLS * CPO];
    __shared__ __align__(16) __nv_bfloat16 Xs[TROWS * TCOLS * CPI];
    const int tap = blockIdx.y, group = blockIdx.x;
    const int ky = tap / 3, kx = tap % 3;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tiles_x = nx / TCOLS, tiles_y = ny / TROWS;
    const long long ntiles = (long long)nb * tiles_x * tiles_y;
    float acc[PER_WARP][4];
#pragma unroll
    for (int q = 0; q < PER_WARP; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.0f;
    const long long t0 = (long long)group * tiles_per_group, t1 = min(ntiles, t0 + tiles_per_group);
    for (long long tile = t0; tile < t1; ++tile) {
        const int b = (int)(tile / (tiles_x * tiles_y));
        const int rem = (int)(tile % (tiles_x * tiles_y));
        const int y0 = (rem / tiles_x) * TROWS, x0 = (rem % tiles_x) * TCOLS;
        __syncthreads();
        for (int i = tid; i < TROWS * TCOLS * (COUT / 8); i += CONV_THREADS) {
            const int c8 = i % (COUT / 8), pix = i / (COUT / 8);
            const int gy = y0 + pix / TCOLS, gx = x0 + pix % TCOLS;
            const long long src = PAD ? ((long long)b * (ny + 2) + gy + 1) * (nx + 2) + gx + 1
                                      : ((long long)b * ny + gy) * nx + gx;
            *reinterpret_cast<uint4*>(Ds + pix * CPO + c8 * 8) =
                *reinterpret_cast<const uint4*>(dz + src * COUT + c8 * 8);
        }
        for (int i = tid; i < TROWS * TCOLS * (CIN / 8); i += CONV_THREADS) {
            const int c8 = i % (CIN / 8), pix = i / (CIN / 8);
            long long src;
            if (PAD)
                src = ((long long)b * (ny + 2) + y0 + pix / TCOLS + ky) * (nx + 2) + x0 + pix % TCOLS + kx;
            else
                src = ((long long)b * ny + pmod(y0 + pix / TCOLS + ky - 1, ny)) * nx + pmod(x0 + pix % TCOLS + kx - 1, nx);
            *reinterpret_cast<uint4*>(Xs + pix * CPI + c8 * 8) =
                *reinterpret_cast<const uint4*>(X + src * CIN + c8 * 8);
        }
        __syncthreads();
        // K = 128 pixels in 8 steps of 16
#pragma unroll 1
        for (int k0 = 0; k0 < TROWS * TCOLS; k0 += 16) {
#pragma unroll
            for (int q = 0; q < PER_WARP; ++q) {
                const int t = warp * PER_WARP + q;
                if (t < TILES) {
                    const int mt = t / NT, nt = t % NT;
                    const int mi = lane >> 3, r = lane & 7;
                    // A = dZ^T (co x p): stored [p][co], transposed load
                    const uint32_t aaddr = smem_u32(Ds + (k0 + (mi >> 1) * 8 + r) * CPO + mt * 16 + (mi & 1) * 8);
                    uint32_t a0, a1, a2, a3;
                    ldsm_x4_t(aaddr, a0, a1, a2, a3);
                    // B = X (p x ci): stored [p][ci], transposed load of two 8x8 blocks
                    const int bi = lane & 15;
                    const uint32_t baddr = smem_u32(Xs + (k0 + (bi >> 3) * 8 + (bi & 7)) * CPI + nt * 8);
                    uint32_t b0, b1;
                    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
                                 : "=r"(b0), "=r"(b1)
                                 : "r"(baddr));
                    mma_bf16(acc[q], a0, a1, a2, a3, b0, b1);
                }
            }
        }
    }
    // partial[group][tap][co][ci]
#pragma unroll
    for (int q = 0; q < PER_WARP; ++q) {
        const int t = warp * PER_WARP + q;
        if (t < TILES) {
            const int mt = t / NT, nt = t % NT;
            const int co = mt * 16 + (lane >> 2), ci = nt * 8 + (lane & 3) * 2;
            float* P = partial + (((long long)group * 9 + tap) * COUT) * CIN;
            P[co * CIN + ci] = acc[q][0];
            P[co * CIN + ci + 1] = acc[q][1];
            P[(co + 8) * CIN + ci] = acc[q][2];
            P[(co + 8) * CIN + ci + 1] = acc[q][3];
        }
    }
}

// Weight gradients of all 9 taps of a 16 -> 64 layer per CTA: the CTA loads
// each pixel tile's dZ once and X once with its one-pixel halo, and every
// tap's B fragment is read at the tap's offset in that patch; warp w owns the
// same 16 x 8 output tile for every tap.  Partial sums per group, taps and
// tiles summed in the order of wgrad_kernel.
template <bool PAD>
__global__ void __launch_bounds__(CONV_THREADS)
wgrad9_kernel(const __nv_bfloat16* __restrict__ dz, const __nv_bfloat16* __restrict__ X, int nb, int ny, int nx,
              int tiles_per_group, float* __restrict__ partial)
{
    constexpr int CIN = 16, COUT = 64;
    constexpr int CPI = CIN + 8, CPO = COUT + 8;
    constexpr int NT = CIN / 8;                           // n8 blocks (ci); COUT / 16 = 4 m16 blocks (co)
    constexpr int PR = TROWS + 2, PC = TCOLS + 2;
    __shared__ __align__(16) __nv_bfloat16 Ds[TROWS * TCOLS * CPO];
    __shared__ __align__(16) __nv_bfloat16 Xs[PR * PC * CPI];
    const int group = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int mt = warp / NT, nt = warp % NT;
    const int tiles_x = nx / TCOLS, tiles_y = ny / TROWS;
    const long long ntiles = (long long)nb * tiles_x * tiles_y;
    float acc[9][4];
#pragma unroll
    for (int t = 0; t < 9; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.0f;
    const long long t0 = (long long)group * tiles_per_group, t1 = min(ntiles, t0 + tiles_per_group);
    for (long long tile = t0; tile < t1; ++tile) {
        const int b = (int)(tile / (tiles_x * tiles_y));
        const int rem = (int)(tile % (tiles_x * tiles_y));
        const int y0 = (rem / tiles_x) * TROWS, x0 = (rem % tiles_x) * TCOLS;
        __syncthreads();
        for (int i = tid; i < TROWS * TCOLS * (COUT / 8); i += CONV_THREADS) {
            const int c8 = i % (COUT / 8), pix = i / (COUT / 8);
            const int gy = y0 + pix / TCOLS, gx = x0 + pix % TCOLS;
            const long long src = PAD ? ((long long)b * (ny + 2) + gy + 1) * (nx + 2) + gx + 1
                                      : ((long long)b * ny + gy) * nx + gx;
            *reinterpret_cast<uint4*>(Ds + pix * CPO + c8 * 8) =
                *reinterpret_cast<const uint4*>(dz + src * COUT + c8 * 8);
        }
        for (int i = tid; i < PR * PC * (CIN / 8); i += CONV_THREADS) {
            const int c8 = i % (CIN / 8), q = i / (CIN / 8);
            const int py = q / PC, px = q % PC;
            const long long src = PAD ? ((long long)b * (ny + 2) + y0 + py) * (nx + 2) + x0 + px
                                      : ((long long)b * ny + pmod(y0 - 1 + py, ny)) * nx + pmod(x0 - 1 + px, nx);
            *reinterpret_cast<uint4*>(Xs + q * CPI + c8 * 8) = *reinterpret_cast<const uint4*>(X + src * CIN + c8 * 8);
        }
        __syncthreads();
        // K = the tile's 128 pixels in 8 steps of 16 (one tile row each)
#pragma unroll 1
        for (int k0 = 0; k0 < TROWS * TCOLS; k0 += 16) {
            const int mi = lane >> 3, r = lane & 7;
            // A = dZ^T (co x p): stored [p][co], transposed load
            const uint32_t aaddr = smem_u32(Ds + (k0 + (mi >> 1) * 8 + r) * CPO + mt * 16 + (mi & 1) * 8);
            uint32_t a0, a1, a2, a3;
            ldsm_x4_t(aaddr, a0, a1, a2, a3);
            const int bi = lane & 15, qy = k0 / TCOLS, qx = (bi >> 3) * 8 + (bi & 7);
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
                const int ky = tap / 3, kx = tap % 3;
                // B = X at the tap's shift (p x ci): rows of the halo patch, transposed load
                const uint32_t baddr = smem_u32(Xs + ((qy + ky) * PC + qx + kx) * CPI + nt * 8);
                uint32_t b0, b1;
                asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
                             : "=r"(b0), "=r"(b1)
                             : "r"(baddr));
                mma_bf16(acc[tap], a0, a1, a2, a3, b0, b1);
            }
        }
    }
    // partial[group][tap][co][ci]
    const int co = mt * 16 + (lane >> 2), ci = nt * 8 + (lane & 3) * 2;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
        float* P = partial + (((long long)group * 9 + tap) * COUT) * CIN;
        P[co * CIN + ci] = acc[tap][0];
        P[co * CIN + ci + 1] = acc[tap][1];
        P[(co + 8) * CIN + ci] = acc[tap][2];
        P[(co + 8) * CIN + ci + 1] = acc[tap][3];
    }
}

// grad[i] = sum over groups of partial (fixed order)
__global__ void reduce_groups_kernel(const float* __restrict__ partial, int groups, long long n, float* __restrict__ grad)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.0f;
    for (int g = 0; g < groups; ++g) s += partial[(long long)g * n + i];
    grad[i] = s;
}

// bias gradients db[co] = sum_p dZ[p][co] in two fixed-order levels: block k
// sums the pixel rows [k R, (k + 1) R) of the batch (thread: 8 channels of
// one pixel lane, 16-byte loads), then bias_reduce_kernel adds the blocks
constexpr int BIAS_BLOCKS = 256;
__global__ void __launch_bounds__(256) bias_partial_kernel(const __nv_bfloat16* __restrict__ dz, int nb, int ny, int nx,
                                                           int C, int pad, float* __restrict__ partial)
{
    const int groups = C / 8, lanes = 256 / groups;
    const int cg = threadIdx.x % groups, pl = threadIdx.x / groups;
    const long long rows = (long long)nb * ny;
    const long long per = (rows + gridDim.x - 1) / gridDim.x;
    const long long r0 = (long long)blockIdx.x * per, r1 = min(rows, r0 + per);
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long row = r0; row < r1; ++row) {
        const long long b = row / ny;
        const int y = (int)(row % ny);
        const long long base = pad ? (b * (ny + 2) + y + 1) * (nx + 2) + 1 : row * nx;
        for (int x = pl; x < nx; x += lanes) {
            const uint4 u = *reinterpret_cast<const uint4*>(dz + (base + x) * C + cg * 8);
            const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                s[2 * k] += __bfloat162float(h[k].x);
                s[2 * k + 1] += __bfloat162float(h[k].y);
            }
        }
    }
    __shared__ float red[256 * 8];
#pragma unroll
    for (int k = 0; k < 8; ++k) red[threadIdx.x * 8 + k] = s[k];
    __syncthreads();
    if (threadIdx.x < C) {
        const int c = threadIdx.x, g = c / 8, k = c % 8;
        float t = 0.0f;
        for (int l = 0; l < lanes; ++l) t += red[(l * groups + g) * 8 + k];
        partial[blockIdx.x * C + c] = t;
    }
}

__global__ void bias_reduce_kernel(const float* __restrict__ partial, int blocks, int C, float* __restrict__ db)
{
    const int c = threadIdx.x;
    if (c >= C) return;
    float s = 0.0f;
    for (int k = 0; k < blocks; ++k) s += partial[k * C + c];
    db[c] = s;
}

// 16 BF16 channels of one pixel into the padded [b][ny + 2][nx + 2][16]
// array at the pixel and at its periodic halo images
__device__ __forceinline__ void store_padded16(__nv_bfloat16* __restrict__ out, const uint4* src, long long b, int y,
                                               int x, int ny, int nx)
{
    const long long pw = nx + 2, plane = (long long)(ny + 2) * pw;
    const int ys[2] = {y + 1, y == 0 ? ny + 1 : (y == ny - 1 ? 0 : -1)};
    const int xs[2] = {x + 1, x == 0 ? nx + 1 : (x == nx - 1 ? 0 : -1)};
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 2; ++c)
            if (ys[a] >= 0 && xs[c] >= 0) {
                uint4* d = reinterpret_cast<uint4*>(out + (b * plane + (long long)ys[a] * pw + xs[c]) * 16);
                d[0] = src[0];
                d[1] = src[1];
            }
}

// fp32 last-layer output (3 ch) vs target (3 ch): loss partials (per block)
// and dZ_out = 2 (out - target) / count into the 16-channel bf16 buffer
__global__ void loss_kernel(const float* __restrict__ out, const float* __restrict__ target, long long npix,
                            int ny, int nx, int pad, double inv_count, __nv_bfloat16* __restrict__ dz,
                            double* __restrict__ partial)
{
    double s = 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += (long long)gridDim.x * blockDim.x) {
        __align__(16) __nv_bfloat16 g[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) g[c] = __float2bfloat16(0.0f);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float r = out[p * 3 + c] - target[p * 3 + c];
            s += (double)r * r;
            g[c] = __float2bfloat16((float)(2.0 * inv_count) * r);
        }
        if (pad) {
            const long long b = p / ((long long)ny * nx);
            const int r = (int)(p % ((long long)ny * nx));
            store_padded16(dz, reinterpret_cast<const uint4*>(g), b, r / nx, r % nx, ny, nx);
        } else {
            uint4* d = reinterpret_cast<uint4*>(dz + p * 16);
            d[0] = *reinterpret_cast<uint4*>(&g[0]);
            d[1] = *reinterpret_cast<uint4*>(&g[8]);
        }
    }
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// the loss of the batch; added to *acc as well when acc is given
// (one block of 256 threads; a fixed-order tree)
__global__ void sum_kernel(const double* __restrict__ partial, int n, double scale, double* __restrict__ out,
                           double* __restrict__ acc)
{
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *out = red[0] * scale;
        if (acc) *acc += red[0] * scale;
    }
}

// Adam on the FP32 master parameters and, in the same pass, the BF16 copies
// of each updated weight in the forward layout [tap][co][ci] and the
// backward-data layout [8 - tap][ci][co].  The bias corrections c1, c2 are
// arguments, or (bc != nullptr) bc[2 t], bc[2 t + 1] of optimizer step t =
// *step (a captured training step).
struct AdamArgs {
    float *w, *m, *v;
    const float* g;
    long long n;
    float lr, b1, b2, eps, c1, c2;
    const float* bc;
    const int* step;
};
struct CastPlan {
    int depth;
    long long w_off[16], b_off[16];
    int cin[16], cout[16];
    __nv_bfloat16* wf[16];
    __nv_bfloat16* wd[16];
};

__device__ __forceinline__ void cast_one(const CastPlan& P, long long i, float wi)
{
    for (int l = 0; l < P.depth; ++l)
        if (i >= P.w_off[l] && i < P.b_off[l]) {
            const int j = (int)(i - P.w_off[l]), cin = P.cin[l], cout = P.cout[l];
            const int ci = j % cin, co = (j / cin) % cout, tap = j / (cin * cout);
            const __nv_bfloat16 b = __float2bfloat16(wi);
            P.wf[l][j] = b;
            P.wd[l][((8 - tap) * cin + ci) * cout + co] = b;
            return;
        }
}

__global__ void adam_cast_kernel(AdamArgs A, CastPlan P)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    float c1 = A.c1, c2 = A.c2;
    if (A.bc) {
        const int t = *A.step;
        c1 = A.bc[2 * t];
        c2 = A.bc[2 * t + 1];
    }
    const float gi = A.g[i];
    const float mi = A.b1 * A.m[i] + (1.0f - A.b1) * gi;
    const float vi = A.b2 * A.v[i] + (1.0f - A.b2) * gi * gi;
    A.m[i] = mi;
    A.v[i] = vi;
    const float wi = A.w[i] - A.lr * (mi / c1) / (sqrtf(vi / c2) + A.eps);
    A.w[i] = wi;
    cast_one(P, i, wi);
}

// the BF16 copies of every weight (after new parameters)
__global__ void cast_all_kernel(const float* __restrict__ w, long long n, CastPlan P)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cast_one(P, i, w[i]);
}

__global__ void advance_kernel(int* __restrict__ cursor, int* __restrict__ step, int batch)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        *cursor += batch;
        *step += 1;
    }
}

// state [n][3][ny][nx] fp32 -> network input [n][ny][nx][16] bf16
// (normalised); field b of the input is field idx[b] of U (b without idx)
__global__ void pack_input_kernel(const float* __restrict__ U, const int* __restrict__ idx,
                                  const int* __restrict__ cursor, int n, int ny, int nx, float s0, float s1, float s2,
                                  __nv_bfloat16* __restrict__ x)
{
    const long long plane = (long long)ny * nx;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n * plane) return;
    const long long b0 = p / plane, c = p % plane, b = idx ? idx[(cursor ? *cursor : 0) + b0] : b0;
    __align__(16) __nv_bfloat16 g[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) g[k] = __float2bfloat16(0.0f);
    g[0] = __float2bfloat16(U[(b * 3 + 0) * plane + c] * s0);
    g[1] = __float2bfloat16(U[(b * 3 + 1) * plane + c] * s1);
    g[2] = __float2bfloat16(U[(b * 3 + 2) * plane + c] * s2);
    uint4* d = reinterpret_cast<uint4*>(x + p * 16);
    d[0] = *reinterpret_cast<uint4*>(&g[0]);
    d[1] = *reinterpret_cast<uint4*>(&g[8]);
}

// the same into the halo-padded layout [n][ny + 2][nx + 2][16]: padded
// position (yp, xp) holds interior cell ((yp - 1) mod ny, (xp - 1) mod nx)
__global__ void pack_input_padded_kernel(const float* __restrict__ U, const int* __restrict__ idx,
                                         const int* __restrict__ cursor, int n, int ny, int nx, float s0, float s1,
                                         float s2, __nv_bfloat16* __restrict__ x)
{
    const long long pw = nx + 2, pplane = (long long)(ny + 2) * pw, plane = (long long)ny * nx;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n * pplane) return;
    const long long b0 = p / pplane, r = p % pplane, b = idx ? idx[(cursor ? *cursor : 0) + b0] : b0;
    const int yp = (int)(r / pw), xq = (int)(r % pw);
    const long long c = (long long)pmod(yp - 1, ny) * nx + pmod(xq - 1, nx);
    __align__(16) __nv_bfloat16 g[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) g[k] = __float2bfloat16(0.0f);
    g[0] = __float2bfloat16(U[(b * 3 + 0) * plane + c] * s0);
    g[1] = __float2bfloat16(U[(b * 3 + 1) * plane + c] * s1);
    g[2] = __float2bfloat16(U[(b * 3 + 2) * plane + c] * s2);
    uint4* d = reinterpret_cast<uint4*>(x + p * 16);
    d[0] = *reinterpret_cast<uint4*>(&g[0]);
    d[1] = *reinterpret_cast<uint4*>(&g[8]);
}

// target of a pair: normalised change (Y - X) / scale, [n][ny][nx][3] fp32
__global__ void pack_target_kernel(const float* __restrict__ X, const float* __restrict__ Y,
                                   const int* __restrict__ idx, const int* __restrict__ cursor, int n, int ny, int nx,
                                   float d0, float d1, float d2, float* __restrict__ t)
{
    const long long plane = (long long)ny * nx;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n * plane) return;
    const long long b0 = p / plane, c = p % plane, b = idx ? idx[(cursor ? *cursor : 0) + b0] : b0;
    t[p * 3 + 0] = (Y[(b * 3 + 0) * plane + c] - X[(b * 3 + 0) * plane + c]) * d0;
    t[p * 3 + 1] = (Y[(b * 3 + 1) * plane + c] - X[(b * 3 + 1) * plane + c]) * d1;
    t[p * 3 + 2] = (Y[(b * 3 + 2) * plane + c] - X[(b * 3 + 2) * plane + c]) * d2;
}

// state += change from the network output (scaled back); out [n][ny][nx][3]
__global__ void apply_output_kernel(float* __restrict__ U, const float* __restrict__ out, int n, int ny, int nx,
                                    float e0, float e1, float e2)
{
    const long long plane = (long long)ny * nx;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n * plane) return;
    const long long b = p / plane, c = p % plane;
    U[(b * 3 + 0) * plane + c] += out[p * 3 + 0] * e0;
    U[(b * 3 + 1) * plane + c] += out[p * 3 + 1] * e1;
    U[(b * 3 + 2) * plane + c] += out[p * 3 + 2] * e2;
}

__global__ void sur_drift_kernel(const float* __restrict__ S0, const float* __restrict__ S1, int ne, int nd,
                                 double* __restrict__ xy, Grid G, double dx, double dy, double T)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne * nd) return;
    const int p = i / nd;
    const double x = xy[2 * i], y = xy[2 * i + 1];
    const int j = pmod((int)floor(x / dx), G.nx), k = pmod((int)floor(y / dy), G.ny);
    const long long c = (long long)k * G.nx + j, b = (long long)p * 3 * G.plane;
    const double h0 = G.H + S0[b + c], h1 = G.H + S1[b + c];
    const double u = 0.5 * (S0[b + G.plane + c] / h0 + S1[b + G.plane + c] / h1);
    const double v = 0.5 * (S0[b + 2 * G.plane + c] / h0 + S1[b + 2 * G.plane + c] / h1);
    xy[2 * i] = x + T * u;
    xy[2 * i + 1] = y + T * v;
}

// per particle: max |eta| and the largest |hu/h|, |hv/h| of a state
// [ne][3][ny][nx] (non-negative floats: integer atomicMax on the bits)
__global__ void sur_stats_kernel(const float* __restrict__ S, Grid G, float* __restrict__ out)
{
    const int p = blockIdx.y;
    const float* U = S + (long long)p * 3 * G.plane;
    float e = 0.0f, v = 0.0f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < G.plane; i += (long long)gridDim.x * blockDim.x) {
        const float eta = U[i];
        const float h = G.H + eta;
        e = fmaxf(e, fabsf(eta));
        v = fmaxf(v, fmaxf(fabsf(U[G.plane + i]), fabsf(U[2 * G.plane + i])) / h);
        if (!isfinite(eta) || !isfinite(U[G.plane + i]) || !isfinite(U[2 * G.plane + i]) || !(h > 0.0f))
            e = __int_as_float(0x7f800000);
    }
    e = warp_max(e);
    v = warp_max(v);
    __shared__ float red[2][8];
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = e;
        red[1][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            e = fmaxf(e, red[0][w]);
            v = fmaxf(v, red[1][w]);
        }
        atomicMax(reinterpret_cast<int*>(out) + 2 * p, __float_as_int(e));
        atomicMax(reinterpret_cast<int*>(out) + 2 * p + 1, __float_as_int(v));
    }
}

template <int CIN, int COUT, int MODE>
size_t conv_smem()
{
    return (size_t)(9 * COUT * (CIN + 8) + (TROWS + 2) * (TCOLS + 2) * (CIN + 8)) * sizeof(__nv_bfloat16);
}

// the shared-memory limit of conv_kernel<CIN, COUT, MODE> and its resident
// CTAs per SM (set and queried once per device)
template <int CIN, int COUT, int MODE>
cudaError_t conv_setup(int* per_sm)
{
    const size_t sm = conv_smem<CIN, COUT, MODE>();
    cudaError_t e = tc::smem_attr_once<conv_kernel<CIN, COUT, MODE>>((int)sm);
    if (e != cudaSuccess) return e;
    static std::atomic<int> per_dev[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    int per = dev < 64 ? per_dev[dev].load(std::memory_order_relaxed) : 0;
    if (per == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, conv_kernel<CIN, COUT, MODE>, CONV_THREADS, sm);
        per = std::max(per, 1);
        if (dev < 64) per_dev[dev].store(per, std::memory_order_relaxed);
    }
    if (per_sm) *per_sm = per;
    return cudaSuccess;
}

template <int CIN, int COUT, int MODE>
cudaError_t conv(const __nv_bfloat16* in, const __nv_bfloat16* W, const float* bias, int nb, int ny, int nx,
                 __nv_bfloat16* z, __nv_bfloat16* a, float* f, const __nv_bfloat16* zprev, cudaStream_t st)
{
    const size_t sm = conv_smem<CIN, COUT, MODE>();
    int per = 1;
    cudaError_t e = conv_setup<CIN, COUT, MODE>(&per);
    if (e != cudaSuccess) return e;
    const int sms = tc::sm_count();
    const long long tiles = (long long)nb * (nx / TCOLS) * (ny / TROWS);
    const int grid = (int)std::min<long long>(tiles, (long long)sms * std::max(per, 1));
    conv_kernel<CIN, COUT, MODE><<<grid, CONV_THREADS, sm, st>>>(in, W, bias, nb, ny, nx, z, a, f, zprev);
    return cudaGetLastError();
}

template <int CIN, int COUT, bool PAD>
cudaError_t wgrad(const __nv_bfloat16* dz, const __nv_bfloat16* X, int nb, int ny, int nx, int groups, float* partial,
                  float* grad, cudaStream_t st)
{
    const long long tiles = (long long)nb * (nx / TCOLS) * (ny / TROWS);
    const int tpg = (int)((tiles + groups - 1) / groups);
    wgrad_kernel<CIN, COUT, PAD><<<dim3(groups, 9), CONV_THREADS, 0, st>>>(dz, X, nb, ny, nx, tpg, partial);
    const long long n = 9LL * CIN * COUT;
    reduce_groups_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(partial, groups, n, grad);
    return cudaGetLastError();
}

// layer 0's weight gradients (16 -> 64) with all taps per CTA
template <bool PAD>
cudaError_t wgrad9(const __nv_bfloat16* dz, const __nv_bfloat16* X, int nb, int ny, int nx, int groups,
                   float* partial, float* grad, cudaStream_t st)
{
    const long long tiles = (long long)nb * (nx / TCOLS) * (ny / TROWS);
    const int tpg = (int)((tiles + groups - 1) / groups);
    wgrad9_kernel<PAD><<<groups, CONV_THREADS, 0, st>>>(dz, X, nb, ny, nx, tpg, partial);
    const long long n = 9LL * 16 * 64;
    reduce_groups_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(partial, groups, n, grad);
    return cudaGetLastError();
}

cudaError_t bias_grad(const __nv_bfloat16* dz, int nb, int ny, int nx, int C, int pad, float* partial, float* db,
                      cudaStream_t st)
{
    bias_partial_kernel<<<BIAS_BLOCKS, 256, 0, st>>>(dz, nb, ny, nx, C, pad, partial);
    bias_reduce_kernel<<<1, 64, 0, st>>>(partial, BIAS_BLOCKS, C, db);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sur_drift(const float* S0, const float* S1, int ne, int nd, double* xy, const Grid& G, double dx,
                             double dy, double T, cudaStream_t st)
{
    const int n = ne * nd;
    if (n > 0) sur_drift_kernel<<<(n + 127) / 128, 128, 0, st>>>(S0, S1, ne, nd, xy, G, dx, dy, T);
    return cudaGetLastError();
}

cudaError_t launch_sur_stats(const float* S, int ne, const Grid& G, float* out, cudaStream_t st)
{
    cudaMemsetAsync(out, 0, sizeof(float) * 2 * ne, st);
    const long long blocks = (G.plane + 256 * 8 - 1) / (256 * 8);
    dim3 grid((unsigned)std::max<long long>(1, std::min<long long>(blocks, 1024)), ne);
    sur_stats_kernel<<<grid, 256, 0, st>>>(S, G, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// host: the network and its training
// ---------------------------------------------------------------------------
Surrogate::~Surrogate() { release(); }

void Surrogate::release()
{
    for (void* p : owned)
        if (p) cudaFree(p);
    owned.clear();
}

static void sfree(Surrogate& s, void* p)
{
    if (!p) return;
    for (auto& q : s.owned)
        if (q == p) {
            cudaFree(q);
            q = nullptr;
        }
}

template <typename T>
static T* salloc(Surrogate& s, size_t n)
{
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) return nullptr;
    s.owned.push_back(p);
    return static_cast<T*>(p);
}

int Surrogate::layer_cin(int l) const { return l == 0 ? 16 : width; }
int Surrogate::layer_cout(int l) const { return l == depth - 1 ? 16 : width; }
size_t Surrogate::layer_w(int l) const { return 9ull * layer_cin(l) * layer_cout(l); }

int Surrogate::init(int nx_, int ny_, int width_, int depth_)
{
    nx = nx_;
    ny = ny_;
    width = width_;
    depth = depth_;
    if (width != 64 || depth < 2 || depth > 16 || nx % TCOLS || ny % TROWS) return IEWPF_EINVAL;
    n_params = 0;
    for (int l = 0; l < depth; ++l) {
        w_off.push_back(n_params);
        n_params += layer_w(l);
        b_off.push_back(n_params);
        n_params += layer_cout(l);
    }
    dflag = salloc<int>(*this, 1);
    master = salloc<float>(*this, n_params);
    grad = salloc<float>(*this, n_params);
    adam_m = salloc<float>(*this, n_params);
    adam_v = salloc<float>(*this, n_params);
    for (int l = 0; l < depth; ++l) {
        wf.push_back(salloc<__nv_bfloat16>(*this, layer_w(l)));
        wd.push_back(salloc<__nv_bfloat16>(*this, layer_w(l)));
    }
    if (!master || !grad || !adam_m || !adam_v || !dflag) return IEWPF_ENOMEM;
    cudaMemset(dflag, 0, sizeof(int));
    for (auto* p : wf)
        if (!p) return IEWPF_ENOMEM;
    for (auto* p : wd)
        if (!p) return IEWPF_ENOMEM;
    cudaMemset(adam_m, 0, n_params * sizeof(float));
    cudaMemset(adam_v, 0, n_params * sizeof(float));
    // the network's kernels run on non-blocking streams
    return cudaDeviceSynchronize() == cudaSuccess ? IEWPF_OK : IEWPF_ECUDA;
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

// 64-channel halo-padded activations [nb][ny + 2][nx + 2][64] as a 4-D map
// (64 ch, nx + 2, ny + 2, nb) with the 128-byte swizzle, box (64, bw, bh, 1)
static bool map64(CUtensorMap* m, void* p, int nb, int ny, int nx, uint32_t bw, uint32_t bh)
{
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t W2 = (cuuint64_t)nx + 2, H2 = (cuuint64_t)ny + 2;
    const cuuint64_t dims[4] = {64, W2, H2, (cuuint64_t)nb};
    const cuuint64_t strides[3] = {128, W2 * 128, H2 * W2 * 128};
    const cuuint32_t box[4] = {64, bw, bh, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, p, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 16-channel halo-padded arrays [nb][ny + 2][nx + 2][16] as a 5-D map (8 ch,
// nx + 2, ny + 2, channel group, nb) without swizzle, box (8, bw, bh, 2, 1)
static bool map16(CUtensorMap* m, void* p, int nb, int ny, int nx, uint32_t bw, uint32_t bh)
{
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t W2 = (cuuint64_t)nx + 2, H2 = (cuuint64_t)ny + 2;
    const cuuint64_t dims[5] = {8, W2, H2, 2, (cuuint64_t)nb};
    const cuuint64_t strides[4] = {32, W2 * 32, 16, H2 * W2 * 32};
    const cuuint32_t box[5] = {8, bw, bh, 2, 1};
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, p, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool Surrogate::uses_tc_train() const
{
    return path == 0 && conv_tr_supported(nx, ny);
}

int Surrogate::ensure_batch(int nb)
{
    const int pad = uses_tc_train() ? 1 : 0;
    if (nb <= cap_batch && pad == batch_pad) return IEWPF_OK;
    // activations per layer: input (16 ch), then z and a per hidden layer
    for (void* p : {(void*)x_in, (void*)out, (void*)target, (void*)dz_a, (void*)dz_b, (void*)dz_out, (void*)wpartial,
                    (void*)bpartial, (void*)lpartial, (void*)dloss, (void*)eloss})
        sfree(*this, p);
    for (auto* p : z) sfree(*this, p);
    for (auto* p : a) sfree(*this, p);
    cap_batch = 0;
    const size_t pix = (size_t)nb * nx * ny;
    const size_t ppix = pad ? (size_t)nb * (nx + 2) * (ny + 2) : pix;
    x_in = salloc<__nv_bfloat16>(*this, ppix * 16);
    z.assign(depth, nullptr);
    a.assign(depth, nullptr);
    for (int l = 0; l + 1 < depth; ++l) {
        z[l] = salloc<__nv_bfloat16>(*this, pix * width);
        a[l] = salloc<__nv_bfloat16>(*this, ppix * width);
    }
    out = salloc<float>(*this, pix * 3);
    target = salloc<float>(*this, pix * 3);
    dz_a = salloc<__nv_bfloat16>(*this, ppix * width);
    dz_b = salloc<__nv_bfloat16>(*this, ppix * width);
    dz_out = salloc<__nv_bfloat16>(*this, ppix * 16);
    int groups = wgrad_groups(nb);
    if (pad) {
        int g = 0, tpg = 0;
        wgrad_tc_split(nb, ny, nx, &g, &tpg);
        groups = std::max(groups, g);
    }
    wpartial = salloc<float>(*this, std::max((size_t)groups * std::max(9 * width * width, wgrad_tc_partial(width)),
                                             (size_t)wgrad9_groups(nb) * 9 * 16 * width));
    bpartial = salloc<float>(*this, (size_t)BIAS_BLOCKS * width);
    lpartial = salloc<double>(*this, 1024);
    dloss = salloc<double>(*this, 1);
    eloss = salloc<double>(*this, 1);
    if (!x_in || !out || !target || !dz_a || !dz_b || !dz_out || !wpartial || !bpartial || !lpartial || !dloss ||
        !eloss)
        return IEWPF_ENOMEM;
    for (int l = 0; l + 1 < depth; ++l)
        if (!z[l] || !a[l]) return IEWPF_ENOMEM;
    if (pad) {
        // tensor maps of the padded buffers (boxes: conv_tr.cu's stages and tiles)
        tm_fwd.assign(depth, CUtensorMap{});
        tm_wx.assign(depth, CUtensorMap{});
        // forward and data passes: halo patches of 10 x 18 pixels; weight
        // gradients: X halo patches of 66 x 6 and dZ tiles of 64 x 4
        bool ok = map16(&tm_in, x_in, nb, ny, nx, 10, 18) && map16(&tm_dout_f, dz_out, nb, ny, nx, 10, 18) &&
                  map16(&tm_dout_w, dz_out, nb, ny, nx, 64, 4);
        for (int l = 0; l + 1 < depth && ok; ++l)
            ok = map64(&tm_fwd[l], a[l], nb, ny, nx, 10, 18) && map64(&tm_wx[l], a[l], nb, ny, nx, 66, 6);
        __nv_bfloat16* dzs[2] = {dz_a, dz_b};
        for (int k = 0; k < 2 && ok; ++k)
            ok = map64(&tm_dz_f[k], dzs[k], nb, ny, nx, 10, 18) && map64(&tm_dz_w[k], dzs[k], nb, ny, nx, 64, 4);
        if (!ok) return IEWPF_ECUDA;
    }
    // launch attributes set now, outside any capture of a training step
    cudaError_t e = pad ? conv_tr_prepare() : cudaSuccess;
    if (e == cudaSuccess) e = conv_setup<16, 64, MODE_HIDDEN>(nullptr);
    if (e == cudaSuccess) e = conv_setup<64, 64, MODE_HIDDEN>(nullptr);
    if (e == cudaSuccess) e = conv_setup<64, 16, MODE_OUT>(nullptr);
    if (e == cudaSuccess) e = conv_setup<16, 64, MODE_DGRAD>(nullptr);
    if (e == cudaSuccess) e = conv_setup<64, 64, MODE_DGRAD>(nullptr);
    if (e != cudaSuccess) return IEWPF_ECUDA;
    batch_pad = pad;
    cap_batch = nb;
    return IEWPF_OK;
}

int Surrogate::wgrad9_groups(int nb) const
{
    const long long tiles = (long long)nb * (nx / TCOLS) * (ny / TROWS);
    return (int)std::max<long long>(1, std::min<long long>(256, tiles / 4));
}

int Surrogate::wgrad_groups(int nb) const
{
    const long long tiles = (long long)nb * (nx / TCOLS) * (ny / TROWS);
    return (int)std::max<long long>(1, std::min<long long>(256, tiles / 16));
}

static CastPlan cast_plan(const Surrogate& s)
{
    CastPlan P{};
    P.depth = s.depth;
    for (int l = 0; l < s.depth; ++l) {
        P.w_off[l] = (long long)s.w_off[l];
        P.b_off[l] = (long long)s.b_off[l];
        P.cin[l] = s.layer_cin(l);
        P.cout[l] = s.layer_cout(l);
        P.wf[l] = s.wf[l];
        P.wd[l] = s.wd[l];
    }
    return P;
}

cudaError_t Surrogate::cast(cudaStream_t st)
{
    cast_all_kernel<<<(unsigned)((n_params + 255) / 256), 256, 0, st>>>(master, (long long)n_params, cast_plan(*this));
    return cudaGetLastError();
}

bool Surrogate::uses_tc() const
{
    return path == 0 && conv_tc_supported(nx, ny);
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

int Surrogate::ensure_infer(int nb)
{
    if (!uses_tc()) {
        const int rc = ensure_batch(nb);
        y_out = out;
        return rc;
    }
    if (nb <= cap_infer) {
        y_out = out_i;
        return IEWPF_OK;
    }
    for (void* p : {(void*)xp, (void*)ap[0], (void*)ap[1], (void*)out_i}) sfree(*this, p);
    cap_infer = 0;
    const size_t pp = (size_t)nb * (nx + 2) * (ny + 2);
    xp = salloc<__nv_bfloat16>(*this, pp * 16);
    ap[0] = salloc<__nv_bfloat16>(*this, pp * width);
    ap[1] = salloc<__nv_bfloat16>(*this, pp * width);
    out_i = salloc<float>(*this, (size_t)nb * nx * ny * 3);
    if (!xp || !ap[0] || !ap[1] || !out_i) return IEWPF_ENOMEM;
    auto enc = tensor_map_encoder();
    if (!enc) return IEWPF_ECUDA;
    const cuuint64_t W2 = (cuuint64_t)nx + 2, H2 = (cuuint64_t)ny + 2;
    {
        // 16 channels: (8 ch, x, y, channel group, b), no swizzle
        const cuuint64_t dims[5] = {8, W2, H2, 2, (cuuint64_t)nb};
        const cuuint64_t strides[4] = {32, W2 * 32, 16, H2 * W2 * 32};
        const cuuint32_t box[5] = {8, 130, 4, 2, 1};
        const cuuint32_t es[5] = {1, 1, 1, 1, 1};
        if (enc(&map_x, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, xp, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
            CUDA_SUCCESS)
            return IEWPF_ECUDA;
    }
    for (int k = 0; k < 2; ++k) {
        // 64 channels: (64 ch, x, y, b), 128-byte swizzle
        const cuuint64_t dims[4] = {(cuuint64_t)width, W2, H2, (cuuint64_t)nb};
        const cuuint64_t strides[3] = {(cuuint64_t)width * 2, W2 * width * 2, H2 * W2 * width * 2};
        const cuuint32_t box[4] = {(cuuint32_t)width, 130, 4, 1};
        const cuuint32_t es[4] = {1, 1, 1, 1};
        if (enc(&map_a[k], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, ap[k], dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return IEWPF_ECUDA;
    }
    cap_infer = nb;
    y_out = out_i;
    return IEWPF_OK;
}

int Surrogate::infer(const float* U, int nb, cudaStream_t st)
{
    int rc = ensure_infer(nb);
    if (rc) return rc;
    cudaError_t e;
    if (!uses_tc()) {
        if ((e = pack_input(U, nb, st)) != cudaSuccess || (e = forward(nb, st)) != cudaSuccess) return IEWPF_ECUDA;
        return IEWPF_OK;
    }
    const long long n = (long long)nb * (nx + 2) * (ny + 2);
    pack_input_padded_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(U, nullptr, nullptr, nb, ny, nx, in_scale[0], in_scale[1],
                                                                         in_scale[2], xp);
    const int probe = inject_timeouts > 0 ? kInjectedWaitPolls : 0;
    if (inject_timeouts > 0) --inject_timeouts;
    for (int l = 0; l < depth; ++l) {
        const float* bias = master + b_off[l];
        const int kind = l == 0 ? 0 : (l + 1 < depth ? 1 : 2);
        const CUtensorMap& in_map = l == 0 ? map_x : map_a[(l - 1) & 1];
        e = launch_conv_tc(kind, in_map, wf[l], bias, nb, ny, nx, kind < 2 ? ap[l & 1] : nullptr,
                           kind == 2 ? out_i : nullptr, dflag, probe, st);
        if (e != cudaSuccess) return IEWPF_ECUDA;
    }
    return cudaGetLastError() == cudaSuccess ? IEWPF_OK : IEWPF_ECUDA;
}

cudaError_t Surrogate::forward(int nb, cudaStream_t st)
{
    cudaError_t e;
    if (batch_pad) {
        for (int l = 0; l < depth; ++l) {
            const int kind = l == 0 ? 0 : (l + 1 < depth ? 1 : 2);
            e = launch_conv_tr(kind, l == 0 ? tm_in : tm_fwd[l - 1], wf[l], master + b_off[l], nb, ny, nx,
                               kind < 2 ? z[l] : nullptr, kind < 2 ? a[l] : nullptr, kind == 2 ? out : nullptr,
                               nullptr, dflag, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    const __nv_bfloat16* in = x_in;
    for (int l = 0; l < depth; ++l) {
        const float* bias = master + b_off[l];
        if (l == 0) e = conv<16, 64, MODE_HIDDEN>(in, wf[l], bias, nb, ny, nx, z[l], a[l], nullptr, nullptr, st);
        else if (l + 1 < depth) e = conv<64, 64, MODE_HIDDEN>(in, wf[l], bias, nb, ny, nx, z[l], a[l], nullptr, nullptr, st);
        else e = conv<64, 16, MODE_OUT>(in, wf[l], bias, nb, ny, nx, nullptr, nullptr, out, nullptr, st);
        if (e != cudaSuccess) return e;
        if (l + 1 < depth) in = a[l];
    }
    return cudaSuccess;
}

// loss of the current forward pass against `target`, gradients into grad
cudaError_t Surrogate::backward(int nb, cudaStream_t st, bool add_eloss)
{
    const long long pix = (long long)nb * nx * ny;
    loss_kernel<<<1024, 256, 0, st>>>(out, target, pix, ny, nx, batch_pad, 1.0 / (3.0 * pix), dz_out, lpartial);
    sum_kernel<<<1, 256, 0, st>>>(lpartial, 1024, 1.0 / (3.0 * pix), dloss, add_eloss ? eloss : nullptr);
    const int groups = wgrad_groups(nb);
    cudaError_t e;
    const int L = depth - 1;
    if (batch_pad) {
        // tcgen05: weight gradients of layers 1..L, data passes; layer 0's
        // weight gradient (16 input channels) on mma.sync
        int tg = 0, tpg = 0;
        wgrad_tc_split(nb, ny, nx, &tg, &tpg);
        // weights and bias of a layer (contiguous in the parameters)
        auto wg = [&](int cout, const CUtensorMap& xm, const CUtensorMap& dm, float* g) {
            cudaError_t r = launch_wgrad_tc(cout, xm, dm, nb, ny, nx, tg, tpg, wpartial, dflag, st);
            if (r != cudaSuccess) return r;
            const long long n = wgrad_tc_partial(cout);
            reduce_groups_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(wpartial, tg, n, g);
            return cudaGetLastError();
        };
        if ((e = wg(16, tm_wx[L - 1], tm_dout_w, grad + w_off[L])) != cudaSuccess) return e;
        if ((e = launch_conv_tr(3, tm_dout_f, wd[L], nullptr, nb, ny, nx, nullptr, dz_a, nullptr, z[L - 1], dflag,
                                st)) != cudaSuccess)
            return e;
        int cur = 0;
        __nv_bfloat16* dzs[2] = {dz_a, dz_b};
        for (int l = L - 1; l >= 0; --l) {
            if (l > 0) {
                e = wg(64, tm_wx[l - 1], tm_dz_w[cur], grad + w_off[l]);
            } else {
                e = wgrad9<true>(dzs[cur], x_in, nb, ny, nx, wgrad9_groups(nb), wpartial, grad + w_off[0], st);
                if (e == cudaSuccess) e = bias_grad(dzs[cur], nb, ny, nx, 64, 1, bpartial, grad + b_off[0], st);
            }
            if (e != cudaSuccess) return e;
            if (l > 0) {
                if ((e = launch_conv_tr(4, tm_dz_f[cur], wd[l], nullptr, nb, ny, nx, nullptr, dzs[cur ^ 1], nullptr,
                                        z[l - 1], dflag, st)) != cudaSuccess)
                    return e;
                cur ^= 1;
            }
        }
        return cudaGetLastError();
    }
    // last layer (64 -> 16)
    if ((e = wgrad<64, 16, false>(dz_out, a[L - 1], nb, ny, nx, groups, wpartial, grad + w_off[L], st)) != cudaSuccess)
        return e;
    if ((e = bias_grad(dz_out, nb, ny, nx, 16, 0, bpartial, grad + b_off[L], st)) != cudaSuccess) return e;
    // dZ of layer L-1 = conv(dZ_out, Wd_L) * silu'(z[L-1])
    if ((e = conv<16, 64, MODE_DGRAD>(dz_out, wd[L], nullptr, nb, ny, nx, nullptr, dz_a, nullptr, z[L - 1], st)) !=
        cudaSuccess)
        return e;
    __nv_bfloat16* cur = dz_a;
    __nv_bfloat16* nxt = dz_b;
    for (int l = L - 1; l >= 0; --l) {
        const __nv_bfloat16* X = l == 0 ? x_in : a[l - 1];
        if (l == 0) e = wgrad9<false>(cur, X, nb, ny, nx, wgrad9_groups(nb), wpartial, grad + w_off[l], st);
        else e = wgrad<64, 64, false>(cur, X, nb, ny, nx, groups, wpartial, grad + w_off[l], st);
        if (e != cudaSuccess) return e;
        if ((e = bias_grad(cur, nb, ny, nx, 64, 0, bpartial, grad + b_off[l], st)) != cudaSuccess) return e;
        if (l > 0) {
            if ((e = conv<64, 64, MODE_DGRAD>(cur, wd[l], nullptr, nb, ny, nx, nullptr, nxt, nullptr, z[l - 1], st)) !=
                cudaSuccess)
                return e;
            std::swap(cur, nxt);
        }
    }
    return cudaGetLastError();
}

cudaError_t Surrogate::train_step(const float* X, const float* Y, const int* order, int* ctr, const float* bc,
                                  int batch, float lr, cudaStream_t st)
{
    cudaError_t e;
    if ((e = pack_input(X, batch, st, order, ctr)) != cudaSuccess ||
        (e = pack_target(X, Y, batch, st, order, ctr)) != cudaSuccess || (e = forward(batch, st)) != cudaSuccess ||
        (e = backward(batch, st, true)) != cudaSuccess)
        return e;
    const AdamArgs A{master, adam_m, adam_v, grad, (long long)n_params, lr, kAdamB1, kAdamB2, kAdamEps, 1.0f, 1.0f,
                     bc, ctr + 1};
    adam_cast_kernel<<<(unsigned)((n_params + 255) / 256), 256, 0, st>>>(A, cast_plan(*this));
    advance_kernel<<<1, 32, 0, st>>>(ctr, ctr + 1, batch);
    return cudaGetLastError();
}

cudaError_t Surrogate::adam_step(float lr, cudaStream_t st)
{
    ++t_adam;
    const float c1 = 1.0f - std::pow(kAdamB1, (float)t_adam), c2 = 1.0f - std::pow(kAdamB2, (float)t_adam);
    const AdamArgs A{master, adam_m, adam_v, grad, (long long)n_params, lr, kAdamB1, kAdamB2, kAdamEps, c1, c2,
                     nullptr, nullptr};
    adam_cast_kernel<<<(unsigned)((n_params + 255) / 256), 256, 0, st>>>(A, cast_plan(*this));
    return cudaGetLastError();
}

cudaError_t Surrogate::pack_input(const float* U, int nb, cudaStream_t st, const int* idx, const int* cursor)
{
    if (batch_pad) {
        const long long n = (long long)nb * (nx + 2) * (ny + 2);
        pack_input_padded_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(U, idx, cursor, nb, ny, nx, in_scale[0],
                                                                             in_scale[1], in_scale[2], x_in);
        return cudaGetLastError();
    }
    const long long n = (long long)nb * nx * ny;
    pack_input_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(U, idx, cursor, nb, ny, nx, in_scale[0],
                                                                  in_scale[1], in_scale[2], x_in);
    return cudaGetLastError();
}

cudaError_t Surrogate::pack_target(const float* X, const float* Y, int nb, cudaStream_t st, const int* idx,
                                   const int* cursor)
{
    const long long n = (long long)nb * nx * ny;
    pack_target_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(X, Y, idx, cursor, nb, ny, nx, 1.0f / out_scale[0],
                                                                   1.0f / out_scale[1], 1.0f / out_scale[2], target);
    return cudaGetLastError();
}

cudaError_t Surrogate::apply(float* U, int nb, cudaStream_t st)
{
    if (!y_out || nb > std::max(cap_batch, cap_infer)) return cudaErrorInvalidValue;
    const long long n = (long long)nb * nx * ny;
    apply_output_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(U, y_out, nb, ny, nx, out_scale[0],
                                                                    out_scale[1], out_scale[2]);
    return cudaGetLastError();
}

}  // namespace iewpf
