// Training convolutions of the surrogate on the 5th-generation tensor cores:
// the forward pass that keeps the pre-activations z, the backward data pass
// (the flipped, transposed weights with the SiLU derivative fused) and the
// weight gradients.  Operands are staged by TMA, products by tcgen05.mma from
// shared memory with FP32 accumulators in tensor memory.
//
// Forward and data passes (conv_tr_kernel): implicit GEMM over tiles of 16
// output rows x 8 pixels.  The 64-pixel rows of the training fields are half
// an M = 128 accumulator, so the tile is tall instead: each of its 16 rows is
// one 8-row atom of the A operand (128-byte swizzle for 64 channels, one
// core matrix for 16), and consecutive atoms lie one halo-patch row (10
// pixels) apart, the descriptor's uniform atom stride.  One TMA box per tile
// (CIN channels, 10 pixels, 18 rows) holds the tile and its halo, and a
// shifted tap is a shifted start address; 9 taps x CIN / 16 products of
// 128 x COUT x 16 fill one accumulator, two of them alternate in tensor
// memory.  (A tile of 4 rows x 64 pixels needs the three column-shifted
// copies of its patch, 3.1 times the bytes per output pixel.)
//
// Weight gradients (wgrad_tc_kernel): dW[tap][co][ci] = sum_p dZ[p][co]
// X[p + off(tap)][ci] as a GEMM with K = pixels, both operands M/N-major (the
// channels are contiguous in NHWC).  The A operand of one product is the
// halo patch of X seen at two taps: its two 64-channel blocks lie one tap
// offset apart (the descriptor's block stride), so M = 128 = (tap pair,
// channel).  Five products cover the 9 taps: the pairs (0,1) (2,3) (4,5)
// (6,7) and (ones, 8), whose first block is a fixed 2 KB run of BF16 ones in
// shared memory (the descriptor's block stride reaches tap 8 from it), so
// its rows hold the bias gradient db[co] = sum_p dZ[p][co].  N = COUT
// channels of dZ.  Each CTA reduces a contiguous range of pixel tiles into
// partial sums, which a second pass adds in a fixed order.
//
// Every wait is bounded: on a timeout the CTA raises an abort flag, records
// FLAG_TIMEOUT, waits (bounded) for its own copies and products in flight
// and frees its tensor memory.
#include <algorithm>
#include <cstdint>

#include <cuda.h>

#include "common.cuh"
#include "kernels.h"
#include "surrogate.h"
#include "tc_dev.cuh"

#include <cuda_bf16.h>

namespace iewpf {

namespace {

using tc::idesc_bf16;
using tc::mbar_drain;
using tc::mbar_wait;
using tc::mma_bf16_ss;
using tc::mma_commit;
using tc::sdesc;
using tc::su32;
using tc::tmem_ld16;
using tc::tmem_ld32;

constexpr int TR_TW = 8;                   // tile columns: one 8-row swizzle atom (or core matrix) per tile row
constexpr int TR_TH = 16;                  // tile rows: 16 x 8 = 128 pixels = M
constexpr int TR_PW = TR_TW + 2;           // halo patch columns
constexpr int TR_PH = TR_TH + 2;           // halo patch rows
constexpr int TR_NS = 4;                   // shared-memory stages
constexpr int TR_EPI_WARPS = 8;            // 4 lane quarters x 2 column halves
constexpr int TR_WARPS = 2 + TR_EPI_WARPS;
constexpr int TR_THREADS = 32 * TR_WARPS;

enum TrMode : int { TR_HID = 0, TR_OUT = 1, TR_DGRAD = 2 };

template <int CIN, int COUT>
struct TrLayout {
    static constexpr bool SW = CIN == 64;                          // 128-byte swizzle of the patches
    static constexpr int W_BYTES = 9 * COUT * CIN * 2;
    static constexpr int STAGE = TR_PH * TR_PW * CIN * 2;          // bytes of one halo patch
    static constexpr int STAGE_ALLOC = (STAGE + 1023) / 1024 * 1024;
    static constexpr int PLANE = TR_PH * TR_PW * 16;               // bytes of one 8-channel plane (no swizzle)
    static constexpr int A_OFF = (W_BYTES + 1023) / 1024 * 1024;
    static constexpr int BIAS_OFF = A_OFF + TR_NS * STAGE_ALLOC;
    static constexpr int NBARS = 2 * TR_NS + 4;                    // full, empty, tfull[2], tempty[2]
    static constexpr int BAR_OFF = BIAS_OFF + COUT * 4;            // then the abort flag and the tensor-memory slot
    static constexpr int TOTAL = BAR_OFF + 8 * NBARS + 16;
    // at least 120 KB so that one CTA runs per SM
    static constexpr int REQUEST = (TOTAL > 120 * 1024 ? TOTAL : 120 * 1024) + 1024;
    static constexpr int TMEM_COLS = 2 * COUT < 32 ? 32 : 2 * COUT;
};

using tc::stage_weights;

// 32 BF16 channels of one pixel into the padded [b][ny + 2][nx + 2][C]
// array at the pixel and at its periodic halo images
template <int C>
__device__ __forceinline__ void store_padded32(__nv_bfloat16* __restrict__ out, const __nv_bfloat162* hv, int b,
                                               int y, int x, int ny, int nx, int c0)
{
    const size_t pw = (size_t)(nx + 2), plane = (size_t)(ny + 2) * pw;
    const int ys[2] = {y + 1, y == 0 ? ny + 1 : (y == ny - 1 ? 0 : -1)};
    const int xs[2] = {x + 1, x == 0 ? nx + 1 : (x == nx - 1 ? 0 : -1)};
    const uint4* src = reinterpret_cast<const uint4*>(hv);
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 2; ++c)
            if (ys[a] >= 0 && xs[c] >= 0) {
                uint4* p = reinterpret_cast<uint4*>(out + ((size_t)b * plane + (size_t)ys[a] * pw + xs[c]) * C + c0);
#pragma unroll
                for (int u = 0; u < 4; ++u) p[u] = src[u];
            }
}

template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(TR_THREADS, 1)
conv_tr_kernel(const __grid_constant__ CUtensorMap tmap_in, const __nv_bfloat16* __restrict__ W,
               const float* __restrict__ bias, int nb, int ny, int nx, __nv_bfloat16* __restrict__ zout,
               __nv_bfloat16* __restrict__ aout, float* __restrict__ fout, const __nv_bfloat16* __restrict__ zprev,
               int* __restrict__ flag)
{
    using L = TrLayout<CIN, COUT>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float* sbias = reinterpret_cast<float*>(smem + L::BIAS_OFF);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
    volatile int* abort = reinterpret_cast<volatile int*>(smem + L::BAR_OFF + 8 * L::NBARS);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L::BAR_OFF + 8 * L::NBARS + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = su32(smem);

    stage_weights<CIN, COUT, TR_THREADS>(smem, W, tid);
    for (int i = tid; i < COUT; i += TR_THREADS) sbias[i] = MODE == TR_DGRAD ? 0.0f : bias[i];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(tmem_slot)),
                     "r"(L::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        // full[NS], empty[NS]: one arrival; tfull[2]: one commit; tempty[2]: one per epilogue warp
        for (int k = 0; k < L::NBARS; ++k) {
            const int count = (k >= 2 * TR_NS + 2) ? TR_EPI_WARPS : 1;
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(su32(&bars[k])), "r"(count));
        }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t full0 = su32(&bars[0]), empty0 = su32(&bars[TR_NS]), tfull0 = su32(&bars[2 * TR_NS]),
                   tempty0 = su32(&bars[2 * TR_NS + 2]);

    const int tiles_x = nx / TR_TW, tiles_y = ny / TR_TH;
    const long long ntiles = (long long)nb * tiles_x * tiles_y;
    const long long first = blockIdx.x, stride = gridDim.x;
    const int nloc = first < ntiles ? (int)((ntiles - 1 - first) / stride + 1) : 0;
    auto tile_coords = [&](int i, int& b, int& y0, int& x0) {
        const long long t = first + (long long)i * stride;
        b = (int)(t / ((long long)tiles_x * tiles_y));
        const int rem = (int)(t % ((long long)tiles_x * tiles_y));
        y0 = (rem / tiles_x) * TR_TH;
        x0 = (rem % tiles_x) * TR_TW;
    };

    if (warp == 0) {
        // ---- TMA producer: the halo patch of tile i into stage i % NS ----
        int issued = 0;
        if (lane == 0) {
            for (int i = 0; i < nloc; ++i) {
                const int s = i % TR_NS;
                const uint32_t k = (uint32_t)(i / TR_NS);
                if (!mbar_wait(empty0 + 8 * s, (k & 1) ^ 1, abort)) break;
                int b, y0, x0;
                tile_coords(i, b, y0, x0);
                const uint32_t dst = sbase + L::A_OFF + s * L::STAGE_ALLOC;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(full0 + 8 * s),
                             "r"(L::STAGE)
                             : "memory");
                // padded coordinates: patch row 0 = padded row y0, patch column 0 = padded column x0
                if (L::SW)
                    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
                                 " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(dst),
                                 "l"(reinterpret_cast<uint64_t>(&tmap_in)), "r"(0), "r"(x0), "r"(y0), "r"(b),
                                 "r"(full0 + 8 * s)
                                 : "memory");
                else
                    asm volatile("cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
                                 " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];\n" ::"r"(dst),
                                 "l"(reinterpret_cast<uint64_t>(&tmap_in)), "r"(0), "r"(x0), "r"(y0), "r"(0),
                                 "r"(b), "r"(full0 + 8 * s)
                                 : "memory");
                issued = i + 1;
            }
            // after an abort, wait (bounded) for the copies in flight
            if (*abort)
                for (int i = issued >= TR_NS ? issued - TR_NS : 0; i < issued; ++i)
                    mbar_drain(full0 + 8 * (i % TR_NS), (uint32_t)((i / TR_NS) & 1));
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---- MMA issuer: 9 taps x CIN / 16 products of 128 x COUT x 16 per tile ----
        int committed = 0;
        if (lane == 0) {
            constexpr uint32_t IDESC = idesc_bf16(128, COUT);
            const uint64_t bdesc = L::SW ? sdesc(sbase, 16, 1024, 2) : sdesc(sbase, COUT * 16, 128, 0);
            for (int i = 0; i < nloc; ++i) {
                const int s = i % TR_NS, as = i & 1;
                if (!mbar_wait(tempty0 + 8 * as, (uint32_t)(((i >> 1) & 1) ^ 1), abort)) break;
                if (!mbar_wait(full0 + 8 * s, (uint32_t)((i / TR_NS) & 1), abort)) break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t a0 = sbase + L::A_OFF + s * L::STAGE_ALLOC;
                // A: the tile's 128 pixels as 16 rows of 8, one 8-row atom (or core
                // matrix) per tile row, atoms one patch row (TR_PW pixels) apart
                const uint64_t adesc = L::SW ? sdesc(a0, 16, TR_PW * 128, 2) : sdesc(a0, L::PLANE, TR_PW * 16, 0);
                const uint32_t d0 = tmem + (uint32_t)(as * COUT);
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    const int ky = tap / 3, kx = tap % 3;
#pragma unroll
                    for (int kc = 0; kc < CIN / 16; ++kc) {
                        const uint32_t aoff = L::SW ? ((ky * TR_PW + kx) * 128 + kc * 32) >> 4
                                                    : (2 * kc * L::PLANE + (ky * TR_PW + kx) * 16) >> 4;
                        const uint32_t boff = L::SW ? (tap * COUT * 128 + kc * 32) >> 4
                                                    : ((tap * (CIN / 8) + 2 * kc) * COUT * 16) >> 4;
                        mma_bf16_ss(d0, adesc + aoff, bdesc + boff, IDESC, (tap | kc) != 0);
                    }
                }
                // the stage is free and the accumulator is ready once these products complete
                mma_commit(empty0 + 8 * s);
                mma_commit(tfull0 + 8 * as);
                committed = i + 1;
            }
            // after an abort, wait (bounded) for the products in flight: a
            // commit to the next phase of tile `committed`'s barrier completes
            // once every product issued so far has
            if (*abort) {
                mma_commit(tfull0 + 8 * (committed & 1));
                mbar_drain(tfull0 + 8 * (committed & 1), (uint32_t)((committed >> 1) & 1));
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue: warp 2 + e reads lane quarter (warp % 4) of the
        // accumulator and its columns 32 (e / 4) + 0..31 ----
        const int e = warp - 2, q = warp & 3, h = e >> 2;
        const bool active = MODE != TR_OUT || h == 0;     // the last layer has 16 columns
        const int m = 32 * q + lane;                      // tile pixel: row m / 8, column m % 8
        for (int i = 0; i < nloc; ++i) {
            const int as = i & 1;
            bool ok = true;
            if (lane == 0) ok = mbar_wait(tfull0 + 8 * as, (uint32_t)((i >> 1) & 1), abort);
            if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            int b, y0, x0;
            tile_coords(i, b, y0, x0);
            const int y = y0 + (m >> 3), x = x0 + (m & 7);
            const size_t pix = ((size_t)b * ny + y) * nx + x;
            const uint32_t ta = tmem + (uint32_t)(as * COUT + 32 * h) + ((uint32_t)(32 * q) << 16);
            if (MODE == TR_OUT) {
                if (active) {
                    float v[16];
                    tmem_ld16(ta, v);
#pragma unroll
                    for (int c = 0; c < 3; ++c) fout[pix * 3 + c] = v[c] + sbias[c];
                }
            } else {
                uint32_t v[32];
                tmem_ld32(ta, v);
                __align__(16) __nv_bfloat162 hv[16];
                if (MODE == TR_HID) {
                    __align__(16) __nv_bfloat162 zv[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float z0 = __uint_as_float(v[2 * j]) + sbias[32 * h + 2 * j];
                        const float z1 = __uint_as_float(v[2 * j + 1]) + sbias[32 * h + 2 * j + 1];
                        zv[j] = __floats2bfloat162_rn(z0, z1);
                        hv[j] = __floats2bfloat162_rn(silu_act(z0), silu_act(z1));
                    }
                    uint4* zp = reinterpret_cast<uint4*>(zout + pix * COUT + 32 * h);
                    const uint4* zs = reinterpret_cast<const uint4*>(zv);
#pragma unroll
                    for (int u = 0; u < 4; ++u) zp[u] = zs[u];
                } else {
                    // dZ of the previous layer = (W^T dZ) * silu'(z_prev)
                    __align__(16) __nv_bfloat162 zv[16];
                    const uint4* zq = reinterpret_cast<const uint4*>(zprev + pix * COUT + 32 * h);
                    uint4* zd = reinterpret_cast<uint4*>(zv);
#pragma unroll
                    for (int u = 0; u < 4; ++u) zd[u] = zq[u];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float g0 = __uint_as_float(v[2 * j]) * silu_grad(__bfloat162float(zv[j].x));
                        const float g1 = __uint_as_float(v[2 * j + 1]) * silu_grad(__bfloat162float(zv[j].y));
                        hv[j] = __floats2bfloat162_rn(g0, g1);
                    }
                }
                store_padded32<COUT>(aout, hv, b, y, x, ny, nx, 32 * h);
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(tempty0 + 8 * as) : "memory");
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid == 0 && *abort) atomicOr(flag, FLAG_TIMEOUT);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(L::TMEM_COLS));
}

// ---------------------------------------------------------------------------
// weight gradients
// ---------------------------------------------------------------------------
constexpr int WG_PX = 64;                  // pixels of a tile row
constexpr int WG_ROWS = 4;                 // rows per tile
constexpr int WG_PROWS = WG_ROWS + 2;      // halo patch rows of X
constexpr int WG_PCOLS = WG_PX + 2;        // halo patch columns of X
constexpr int WG_NS = 2;
constexpr int WG_PAIRS = 5;
constexpr int WG_THREADS = 32 * (2 + 4);

template <int COUT>
struct WgLayout {
    static constexpr int ONES = 2048;                                  // 16 pixels x 64 channels of BF16 ones
    static constexpr int STAGE0 = ONES;                                // first stage
    static constexpr int XSTAGE = WG_PROWS * WG_PCOLS * 128;           // X halo patch, 64 channels
    static constexpr int XSTAGE_ALLOC = (XSTAGE + 1023) / 1024 * 1024;
    static constexpr int DSTAGE = WG_ROWS * WG_PX * COUT * 2;          // dZ tile
    static constexpr int DPLANE = WG_ROWS * WG_PX * 16;                // one 8-channel plane of dZ (COUT = 16)
    static constexpr int STAGE_ALLOC = XSTAGE_ALLOC + (DSTAGE + 1023) / 1024 * 1024;
    static constexpr int BAR_OFF = STAGE0 + WG_NS * STAGE_ALLOC;       // full[2] empty[2] done, abort, slot
    static constexpr int TOTAL = BAR_OFF + 64;
    static constexpr int REQUEST = (TOTAL > 120 * 1024 ? TOTAL : 120 * 1024) + 1024;
    static constexpr int TMEM_COLS = WG_PAIRS * COUT <= 128 ? 128 : 512;
};

// first tap of pair j; the pair is (t0, t0 + 1); the last one is (ones, 8)
__host__ __device__ constexpr int wg_t0(int j) { return j < 4 ? 2 * j : 7; }
// floats of one group's partial sums: dW[9][COUT][64], then db[COUT]
__host__ __device__ constexpr int wg_partial(int cout) { return 9 * cout * 64 + cout; }
// offset of tap t in the X halo patch, in pixels
__host__ __device__ constexpr int wg_off(int t) { return (t / 3) * WG_PCOLS + t % 3; }

template <int COUT>
__global__ void __launch_bounds__(WG_THREADS, 1)
wgrad_tc_kernel(const __grid_constant__ CUtensorMap tmap_x, const __grid_constant__ CUtensorMap tmap_d, int nb,
                int ny, int nx, int tiles_per_group, float* __restrict__ partial, int* __restrict__ flag)
{
    using L = WgLayout<COUT>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
    volatile int* abort = reinterpret_cast<volatile int*>(smem + L::BAR_OFF + 40);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L::BAR_OFF + 44);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = su32(smem);
    // the ones block of the bias product (BF16 1.0 = 0x3F80)
    for (int i = tid; i < L::ONES / 16; i += WG_THREADS)
        reinterpret_cast<uint4*>(smem)[i] = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(tmem_slot)),
                     "r"(L::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        for (int k = 0; k < 2 * WG_NS + 1; ++k)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(su32(&bars[k])), "r"(1));
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t full0 = su32(&bars[0]), empty0 = su32(&bars[WG_NS]), done = su32(&bars[2 * WG_NS]);

    const int tiles_x = nx / WG_PX, tiles_y = ny / WG_ROWS;
    const long long ntiles = (long long)nb * tiles_x * tiles_y;
    const long long t0 = (long long)blockIdx.x * tiles_per_group;
    const int nloc = t0 < ntiles ? (int)(min(ntiles, t0 + tiles_per_group) - t0) : 0;

    if (warp == 0) {
        // ---- TMA producer: X halo patch and dZ tile of each pixel tile ----
        int issued = 0;
        if (lane == 0) {
            for (int i = 0; i < nloc; ++i) {
                const int s = i % WG_NS;
                const uint32_t k = (uint32_t)(i / WG_NS);
                if (!mbar_wait(empty0 + 8 * s, (k & 1) ^ 1, abort)) break;
                const long long t = t0 + i;
                const int b = (int)(t / ((long long)tiles_x * tiles_y));
                const int rem = (int)(t % ((long long)tiles_x * tiles_y));
                const int y0 = (rem / tiles_x) * WG_ROWS, x0 = (rem % tiles_x) * WG_PX;
                const uint32_t xs = sbase + L::STAGE0 + s * L::STAGE_ALLOC, ds = xs + L::XSTAGE_ALLOC;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(full0 + 8 * s),
                             "r"(L::XSTAGE + L::DSTAGE)
                             : "memory");
                // X: padded rows y0.., columns x0.. (the halo of the tile)
                asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
                             " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(xs),
                             "l"(reinterpret_cast<uint64_t>(&tmap_x)), "r"(0), "r"(x0), "r"(y0), "r"(b),
                             "r"(full0 + 8 * s)
                             : "memory");
                // dZ: the tile's own pixels, padded rows y0 + 1.., columns x0 + 1..
                if (COUT == 64)
                    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
                                 " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(ds),
                                 "l"(reinterpret_cast<uint64_t>(&tmap_d)), "r"(0), "r"(x0 + 1), "r"(y0 + 1), "r"(b),
                                 "r"(full0 + 8 * s)
                                 : "memory");
                else
                    asm volatile("cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
                                 " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];\n" ::"r"(ds),
                                 "l"(reinterpret_cast<uint64_t>(&tmap_d)), "r"(0), "r"(x0 + 1), "r"(y0 + 1), "r"(0),
                                 "r"(b), "r"(full0 + 8 * s)
                                 : "memory");
                issued = i + 1;
            }
            if (*abort)
                for (int i = issued >= WG_NS ? issued - WG_NS : 0; i < issued; ++i)
                    mbar_drain(full0 + 8 * (i % WG_NS), (uint32_t)((i / WG_NS) & 1));
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---- MMA issuer: 16 K steps of 16 pixels per tile, 5 tap pairs each ----
        if (lane == 0) {
            constexpr uint32_t IDESC = idesc_bf16(128, COUT, 1, 1);
            for (int i = 0; i < nloc; ++i) {
                const int s = i % WG_NS;
                if (!mbar_wait(full0 + 8 * s, (uint32_t)((i / WG_NS) & 1), abort)) break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t xs = sbase + L::STAGE0 + s * L::STAGE_ALLOC, ds = xs + L::XSTAGE_ALLOC;
#pragma unroll 1
                for (int st = 0; st < WG_ROWS * WG_PX / 16; ++st) {
                    const int r = st >> 2, xo = (st & 3) * 16;
                    // B = dZ^T (N = COUT channels, K = 16 pixels), M/N-major
                    const uint64_t bdesc = COUT == 64 ? sdesc(ds + (uint32_t)((r * WG_PX + xo) * 128), 0, 1024, 2)
                                                      : sdesc(ds + (uint32_t)((r * WG_PX + xo) * 16), 128, L::DPLANE, 0);
#pragma unroll
                    for (int j = 0; j < WG_PAIRS; ++j) {
                        const int ta = wg_t0(j), tb = ta + 1;
                        // A = the X patch at taps ta and tb (M = 2 x 64 channels, K = 16 pixels);
                        // the last product's first block is the ones block
                        const uint32_t bstart = xs + (uint32_t)(((r + tb / 3) * WG_PCOLS + xo + tb % 3) * 128);
                        const uint32_t aaddr = j < WG_PAIRS - 1
                                                   ? xs + (uint32_t)(((r + ta / 3) * WG_PCOLS + xo + ta % 3) * 128)
                                                   : sbase;
                        const uint64_t adesc = sdesc(aaddr, bstart - aaddr, 1024, 2);
                        mma_bf16_ss(tmem + (uint32_t)(j * COUT), adesc, bdesc, IDESC, (i | st) != 0);
                    }
                }
                mma_commit(empty0 + 8 * s);
            }
            // every product issued so far (all of them, or up to an abort)
            mma_commit(done);
            if (*abort) mbar_drain(done, 0);
        }
        __syncwarp();
    } else {
        // ---- epilogue: warp 2 + q reads tensor-memory lanes 32 (warp % 4) + 0..31 ----
        const int q = warp & 3, m = 32 * q + lane, ci = m & 63;
        bool ok = true;
        if (lane == 0) ok = mbar_wait(done, 0, abort);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (ok) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            float* P = partial + (size_t)blockIdx.x * wg_partial(COUT);
#pragma unroll 1
            for (int j = 0; j < WG_PAIRS; ++j) {
                const int tap = m < 64 ? wg_t0(j) : wg_t0(j) + 1;
                const bool bias = j == WG_PAIRS - 1 && m < 64;         // rows of the ones block
                const uint32_t ta = tmem + (uint32_t)(j * COUT) + ((uint32_t)(32 * q) << 16);
#pragma unroll
                for (int c0 = 0; c0 < COUT; c0 += 16) {
                    float v[16];
                    tmem_ld16(ta + (uint32_t)c0, v);
                    if (!bias) {
#pragma unroll
                        for (int c = 0; c < 16; ++c)
                            P[((size_t)tap * COUT + c0 + c) * 64 + ci] = nloc > 0 ? v[c] : 0.0f;
                    } else if (m == 0) {
#pragma unroll
                        for (int c = 0; c < 16; ++c) P[9 * COUT * 64 + c0 + c] = nloc > 0 ? v[c] : 0.0f;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid == 0 && *abort) atomicOr(flag, FLAG_TIMEOUT);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(L::TMEM_COLS));
}

using tc::sm_count;

template <int CIN, int COUT, int MODE>
cudaError_t conv_tr(const CUtensorMap& map, const __nv_bfloat16* W, const float* bias, int nb, int ny, int nx,
                    __nv_bfloat16* z, __nv_bfloat16* a, float* f, const __nv_bfloat16* zprev, int* flag,
                    cudaStream_t st)
{
    using L = TrLayout<CIN, COUT>;
    static_assert(L::REQUEST <= 227 * 1024, "shared memory");
    static_assert(L::TMEM_COLS >= 32 && (L::TMEM_COLS & (L::TMEM_COLS - 1)) == 0, "tensor memory columns");
    cudaError_t e = tc::smem_attr_once<conv_tr_kernel<CIN, COUT, MODE>>(L::REQUEST);
    if (e != cudaSuccess) return e;
    const long long tiles = (long long)nb * (nx / TR_TW) * (ny / TR_TH);
    const int grid = (int)std::min<long long>(tiles, sm_count());
    if (grid < 1) return cudaSuccess;
    conv_tr_kernel<CIN, COUT, MODE><<<grid, TR_THREADS, L::REQUEST, st>>>(map, W, bias, nb, ny, nx, z, a, f, zprev,
                                                                         flag);
    return cudaGetLastError();
}

template <int COUT>
cudaError_t wgrad_tc(const CUtensorMap& xm, const CUtensorMap& dm, int nb, int ny, int nx, int groups, int tpg,
                     float* partial, int* flag, cudaStream_t st)
{
    using L = WgLayout<COUT>;
    static_assert(L::REQUEST <= 227 * 1024, "shared memory");
    cudaError_t e = tc::smem_attr_once<wgrad_tc_kernel<COUT>>(L::REQUEST);
    if (e != cudaSuccess) return e;
    wgrad_tc_kernel<COUT><<<groups, WG_THREADS, L::REQUEST, st>>>(xm, dm, nb, ny, nx, tpg, partial, flag);
    return cudaGetLastError();
}

}  // namespace

bool conv_tr_supported(int nx, int ny)
{
    return nx > 0 && ny > 0 && nx % WG_PX == 0 && ny % TR_TH == 0 && ny % WG_ROWS == 0 && nx + 2 <= 65536 &&
           ny + 2 <= 65536;
}

cudaError_t launch_conv_tr(int kind, const CUtensorMap& in_map, const __nv_bfloat16* W, const float* bias, int nb,
                           int ny, int nx, __nv_bfloat16* z, __nv_bfloat16* a, float* f, const __nv_bfloat16* zprev,
                           int* flag, cudaStream_t st)
{
    if (!conv_tr_supported(nx, ny)) return cudaErrorInvalidValue;
    switch (kind) {
    case 0: return conv_tr<16, 64, TR_HID>(in_map, W, bias, nb, ny, nx, z, a, f, zprev, flag, st);
    case 1: return conv_tr<64, 64, TR_HID>(in_map, W, bias, nb, ny, nx, z, a, f, zprev, flag, st);
    case 2: return conv_tr<64, 16, TR_OUT>(in_map, W, bias, nb, ny, nx, z, a, f, zprev, flag, st);
    case 3: return conv_tr<16, 64, TR_DGRAD>(in_map, W, bias, nb, ny, nx, z, a, f, zprev, flag, st);
    case 4: return conv_tr<64, 64, TR_DGRAD>(in_map, W, bias, nb, ny, nx, z, a, f, zprev, flag, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t conv_tr_prepare()
{
    cudaError_t e;
    if ((e = tc::smem_attr_once<conv_tr_kernel<16, 64, TR_HID>>(TrLayout<16, 64>::REQUEST)) != cudaSuccess ||
        (e = tc::smem_attr_once<conv_tr_kernel<64, 64, TR_HID>>(TrLayout<64, 64>::REQUEST)) != cudaSuccess ||
        (e = tc::smem_attr_once<conv_tr_kernel<64, 16, TR_OUT>>(TrLayout<64, 16>::REQUEST)) != cudaSuccess ||
        (e = tc::smem_attr_once<conv_tr_kernel<16, 64, TR_DGRAD>>(TrLayout<16, 64>::REQUEST)) != cudaSuccess ||
        (e = tc::smem_attr_once<conv_tr_kernel<64, 64, TR_DGRAD>>(TrLayout<64, 64>::REQUEST)) != cudaSuccess ||
        (e = tc::smem_attr_once<wgrad_tc_kernel<64>>(WgLayout<64>::REQUEST)) != cudaSuccess ||
        (e = tc::smem_attr_once<wgrad_tc_kernel<16>>(WgLayout<16>::REQUEST)) != cudaSuccess)
        return e;
    sm_count();
    return cudaSuccess;
}

int wgrad_tc_partial(int cout)
{
    return wg_partial(cout);
}

void wgrad_tc_split(int nb, int ny, int nx, int* groups, int* tiles_per_group)
{
    const long long tiles = (long long)nb * (nx / WG_PX) * (ny / WG_ROWS);
    const long long g0 = std::max<long long>(1, std::min<long long>(tiles, sm_count()));
    const long long tpg = (tiles + g0 - 1) / g0;
    *tiles_per_group = (int)tpg;
    *groups = (int)((tiles + tpg - 1) / tpg);      // every group holds at least one tile
}

cudaError_t launch_wgrad_tc(int cout, const CUtensorMap& x_map, const CUtensorMap& d_map, int nb, int ny, int nx,
                            int groups, int tiles_per_group, float* partial, int* flag, cudaStream_t st)
{
    if (!conv_tr_supported(nx, ny) || groups < 1 || tiles_per_group < 1) return cudaErrorInvalidValue;
    if (cout == 64) return wgrad_tc<64>(x_map, d_map, nb, ny, nx, groups, tiles_per_group, partial, flag, st);
    if (cout == 16) return wgrad_tc<16>(x_map, d_map, nb, ny, nx, groups, tiles_per_group, partial, flag, st);
    return cudaErrorInvalidValue;
}

}  // namespace iewpf
