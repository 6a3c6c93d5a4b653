// Inference forward 3x3 periodic convolution of the surrogate on the
// 5th-generation tensor cores: operands staged by TMA
// (cp.async.bulk.tensor), products by tcgen05.mma (BF16 from shared memory,
// FP32 accumulators in tensor memory), epilogue through tcgen05.ld.
//
// Implicit GEMM per tile of 2 output rows x 128 pixels: for output row r and
// tap (ky, kx), A is the 128 x CIN block of input pixels shifted by
// (ky - 1, kx - 1) and B the COUT x CIN weights of the tap; each row's
// 128 x COUT accumulator sums 9 taps x CIN/16 MMAs of K = 16.  Activations
// live in HBM with a one-pixel periodic halo ([b][ny + 2][nx + 2][C]), so the
// halo patch of a tile (4 rows x 130 pixels x CIN) is a single TMA box and a
// shifted tap is a shifted start address in the matrix descriptor:
//  * CIN = 64: 128-byte rows (one pixel, 64 channels) in the 128-byte swizzle
//    layout (8-row atoms of 1024 bytes); the swizzle follows the absolute
//    shared-memory address, so starts at any pixel (+128 B) or K step (+32 B)
//    stay consistent with what TMA wrote;
//  * CIN = 16: no swizzle, core matrices of 8 pixels x 16 bytes, staged
//    through a tensor map whose dimensions are permuted to
//    (8 channels, pixels, rows, channel groups).
// Warp roles: warp 0 issues TMA, warp 1 issues MMAs (one thread each), warps
// 2-17 drain the accumulators (warp w reads tensor-memory lanes 32 (w % 4) +
// 0..31, i.e. 32 pixels, of one output row and 32 of its channels).  Two shared-memory stages and two
// accumulator sets connect them through mbarriers.  The epilogue adds the
// bias, applies SiLU, writes BF16 outputs with their periodic halo images (or
// the FP32 output of the last layer).  Every wait is bounded: on a timeout the
// CTA raises an abort flag, records FLAG_TIMEOUT, waits (bounded) for its own
// copies and products in flight and frees its tensor memory.
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

constexpr int TC_PX = 128;                 // pixels of one output row segment (MMA M)
constexpr int TC_ROWS = 2;                 // output rows per tile
constexpr int TC_PROWS = TC_ROWS + 2;      // patch rows
constexpr int TC_PCOLS = TC_PX + 2;        // patch columns
constexpr int TC_EPI_WARPS = 16;           // 4 lane quarters x 2 rows x 2 column halves
constexpr int TC_WARPS = 2 + TC_EPI_WARPS;
constexpr int TC_THREADS = 32 * TC_WARPS;
using tc::idesc_bf16;
using tc::mbar_drain;
using tc::mbar_wait;
using tc::sdesc;
using tc::su32;
using tc::tmem_ld16;
using tc::tmem_ld32;

template <int CIN, int COUT>
struct TcLayout {
    static constexpr bool SW = CIN == 64;                          // 128-byte swizzle for the A patch
    static constexpr int W_BYTES = 9 * COUT * CIN * 2;
    static constexpr int STAGE = TC_PROWS * TC_PCOLS * CIN * 2;    // bytes of one patch
    static constexpr int STAGE_ALLOC = (STAGE + 1023) / 1024 * 1024;
    static constexpr int W_OFF = 0;
    static constexpr int A_OFF = (W_BYTES + 1023) / 1024 * 1024;
    static constexpr int BIAS_OFF = A_OFF + 2 * STAGE_ALLOC;
    static constexpr int BAR_OFF = BIAS_OFF + COUT * 4;            // 8 mbarriers, abort flag, tensor-memory slot
    static constexpr int TOTAL = BAR_OFF + 128;
    // at least 120 KB so that one CTA runs per SM: it keeps its tensor memory
    static constexpr int REQUEST = (TOTAL > 120 * 1024 ? TOTAL : 120 * 1024) + 1024;
    static constexpr int TMEM_COLS = 2 * TC_ROWS * COUT;
};

template <int CIN, int COUT, bool OUT>
__global__ void __launch_bounds__(TC_THREADS, 1)
conv_tc_kernel(const __grid_constant__ CUtensorMap tmap_in, const __nv_bfloat16* __restrict__ W,
               const float* __restrict__ bias, int nb, int ny, int nx, __nv_bfloat16* __restrict__ aout,
               float* __restrict__ fout, int* __restrict__ flag, int probe_polls)
{
    using L = TcLayout<CIN, COUT>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float* sbias = reinterpret_cast<float*>(smem + L::BIAS_OFF);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
    // bars: full[2], empty[2], tfull[2], tempty[2]
    volatile int* abort = reinterpret_cast<volatile int*>(smem + L::BAR_OFF + 64);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L::BAR_OFF + 68);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = su32(smem);

    // weights of every tap, once per CTA (B operand, K-major, rows = output channels)
    tc::stage_weights<CIN, COUT, TC_THREADS, true>(smem + L::W_OFF, W, tid);
    for (int i = tid; i < COUT; i += TC_THREADS) sbias[i] = bias[i];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(tmem_slot)),
                     "r"(L::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        for (int k = 0; k < 8; ++k) {
            const int count = (k >= 6) ? TC_EPI_WARPS : 1;     // tempty: one arrival per epilogue warp
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

    const uint32_t full0 = su32(&bars[0]), empty0 = su32(&bars[2]), tfull0 = su32(&bars[4]), tempty0 = su32(&bars[6]);
    // injected failure (probe_polls > 0): before any copy or product is
    // issued, thread 0 waits on stage 0's full barrier, which nothing can
    // complete yet, for at most probe_polls polls; the wait runs out through
    // the same bounded-wait path as the pipeline's, the CTA aborts and runs
    // no tile, and FLAG_TIMEOUT is recorded below
    if (probe_polls > 0) {
        if (tid == 0) mbar_wait(full0, 0, abort, probe_polls);
        __syncthreads();
    }

    const int tiles_x = nx / TC_PX, tiles_y = ny / TC_ROWS;
    const long long ntiles = (long long)nb * tiles_x * tiles_y;
    const long long first = blockIdx.x, stride = gridDim.x;
    const int nloc = (first < ntiles && !*abort) ? (int)((ntiles - 1 - first) / stride + 1) : 0;
    auto tile_coords = [&](int i, int& b, int& y0, int& x0) {
        const long long t = first + (long long)i * stride;
        b = (int)(t / ((long long)tiles_x * tiles_y));
        const int rem = (int)(t % ((long long)tiles_x * tiles_y));
        y0 = (rem / tiles_x) * TC_ROWS;
        x0 = (rem % tiles_x) * TC_PX;
    };

    if (warp == 0) {
        // ---- TMA producer ----
        int issued = 0;
        if (lane == 0) {
            for (int i = 0; i < nloc; ++i) {
                const int s = i & 1;
                const uint32_t k = (uint32_t)(i >> 1);
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
                                 "l"(reinterpret_cast<uint64_t>(&tmap_in)), "r"(0), "r"(x0), "r"(y0), "r"(0), "r"(b),
                                 "r"(full0 + 8 * s)
                                 : "memory");
                issued = i + 1;
            }
            // after an abort, wait (bounded) for the copies in flight
            if (*abort)
                for (int i = issued >= 2 ? issued - 2 : 0; i < issued; ++i)
                    mbar_drain(full0 + 8 * (i & 1), (uint32_t)((i >> 1) & 1));
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---- MMA issuer ----
        int issued = 0;
        if (lane == 0) {
            constexpr uint32_t IDESC = idesc_bf16(TC_PX, COUT);
            for (int i = 0; i < nloc; ++i) {
                const int s = i & 1;
                const uint32_t k = (uint32_t)(i >> 1);
                if (!mbar_wait(full0 + 8 * s, k & 1, abort)) break;
                if (!mbar_wait(tempty0 + 8 * s, (k & 1) ^ 1, abort)) break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t a0 = sbase + L::A_OFF + s * L::STAGE_ALLOC;
                const uint32_t d0 = tmem + (uint32_t)(s * TC_ROWS * COUT);
                // descriptors of the stage and of the weights; every MMA adds a
                // compile-time offset (in 16-byte units) to the address field
                constexpr uint32_t PLANE = TC_PROWS * TC_PCOLS * 16;
                const uint64_t adesc = L::SW ? sdesc(a0, 16, 1024, 2) : sdesc(a0, PLANE, 128, 0);
                const uint64_t bdesc = L::SW ? sdesc(sbase + L::W_OFF, 16, 1024, 2)
                                             : sdesc(sbase + L::W_OFF, COUT * 16, 128, 0);
                if constexpr (L::SW) {
                    // patch row p feeds output row r at ky = p - r; rows 1 and 2 feed
                    // both output rows at the same pixel alignment, so each is one
                    // product of N = 2 COUT into the two adjacent accumulators with the
                    // weight blocks of ky and ky - 1 ([kx][ky = 2, 1, 0] order); rows 0
                    // and 3 are single products.  The first product of each (kx, K
                    // step) round is the row-1 pair, which at kx = 0, kc = 0
                    // initialises both accumulators.
                    constexpr uint32_t ID1 = idesc_bf16(TC_PX, COUT), ID2 = idesc_bf16(TC_PX, 2 * COUT);
#pragma unroll
                    for (int kx = 0; kx < 3; ++kx)
#pragma unroll
                        for (int kc = 0; kc < CIN / 16; ++kc) {
                            auto aoff = [&](int p) { return (uint32_t)(((p * TC_PCOLS + kx) * 128 + kc * 32) >> 4); };
                            auto boff = [&](int ky_top) {
                                return (uint32_t)((((kx * 3 + 2 - ky_top) * COUT) * 128 + kc * 32) >> 4);
                            };
                            tc::mma_bf16_ss(d0, adesc + aoff(1), bdesc + boff(1), ID2, (kx | kc) != 0);
                            tc::mma_bf16_ss(d0, adesc + aoff(0), bdesc + boff(0), ID1, 1);
                            tc::mma_bf16_ss(d0, adesc + aoff(2), bdesc + boff(2), ID2, 1);
                            tc::mma_bf16_ss(d0 + (uint32_t)COUT, adesc + aoff(3), bdesc + boff(2), ID1, 1);
                        }
                } else {
#pragma unroll
                for (int r = 0; r < TC_ROWS; ++r)
#pragma unroll
                    for (int tap = 0; tap < 9; ++tap) {
                        const int ky = tap / 3, kx = tap % 3;
#pragma unroll
                        for (int kc = 0; kc < CIN / 16; ++kc) {
                            const uint32_t aoff = L::SW ? (((r + ky) * TC_PCOLS + kx) * 128 + kc * 32) >> 4
                                                        : (2 * kc * PLANE + ((r + ky) * TC_PCOLS + kx) * 16) >> 4;
                            const uint32_t boff = L::SW ? (tap * COUT * 128 + kc * 32) >> 4
                                                        : ((tap * (CIN / 8) + 2 * kc) * COUT * 16) >> 4;
                            if ((tap | kc) != 0)
                                asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 1;\n" ::"r"(
                                                 d0 + (uint32_t)(r * COUT)),
                                             "l"(adesc + aoff), "l"(bdesc + boff), "r"(IDESC));
                            else
                                asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 0;\n" ::"r"(
                                                 d0 + (uint32_t)(r * COUT)),
                                             "l"(adesc + aoff), "l"(bdesc + boff), "r"(IDESC));
                        }
                    }
                }
                // the stage is free and the accumulators are ready once these MMAs complete
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                 empty0 + 8 * s)
                             : "memory");
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                 tfull0 + 8 * s)
                             : "memory");
                issued = i + 1;
            }
            if (*abort && issued > 0)
                mbar_drain(tfull0 + 8 * ((issued - 1) & 1), (uint32_t)(((issued - 1) >> 1) & 1));
        }
        __syncwarp();
    } else {
        // ---- epilogue: warp 2 + e reads lane quarter (warp % 4) of output row
        // (e / 8) and accumulator columns 32 ((e / 4) % 2) + 0..31 ----
        const int e = warp - 2, q = warp & 3, r = e >> 3, h = (e >> 2) & 1;
        const bool active = !OUT || h == 0;          // the last layer has 16 columns
        for (int i = 0; i < nloc; ++i) {
            const int s = i & 1;
            const uint32_t k = (uint32_t)(i >> 1);
            bool ok = true;
            if (lane == 0) ok = mbar_wait(tfull0 + 8 * s, k & 1, abort);
            if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            int b, y0, x0;
            tile_coords(i, b, y0, x0);
            const int y = y0 + r, x = x0 + 32 * q + lane;
            const uint32_t ta = tmem + (uint32_t)(s * TC_ROWS * COUT + r * COUT + 32 * h) + ((uint32_t)(32 * q) << 16);
            if (OUT) {
                if (active) {
                    float v[16];
                    tmem_ld16(ta, v);
                    const size_t pix = ((size_t)b * ny + y) * nx + x;
#pragma unroll
                    for (int c = 0; c < 3; ++c) fout[pix * 3 + c] = v[c] + sbias[c];
                }
            } else {
                uint32_t v[32];
                tmem_ld32(ta, v);
                __align__(16) __nv_bfloat162 hv[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float z0 = __uint_as_float(v[2 * j]) + sbias[32 * h + 2 * j];
                    const float z1 = __uint_as_float(v[2 * j + 1]) + sbias[32 * h + 2 * j + 1];
                    hv[j] = __floats2bfloat162_rn(silu_act(z0), silu_act(z1));
                }
                // this pixel and its periodic images in the padded output
                const size_t pw = (size_t)(nx + 2), plane = (size_t)(ny + 2) * pw;
                const int ys[2] = {y + 1, y == 0 ? ny + 1 : (y == ny - 1 ? 0 : -1)};
                const int xs[2] = {x + 1, x == 0 ? nx + 1 : (x == nx - 1 ? 0 : -1)};
                const uint4* src = reinterpret_cast<const uint4*>(hv);
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int c = 0; c < 2; ++c)
                        if (ys[a] >= 0 && xs[c] >= 0) {
                            uint4* p = reinterpret_cast<uint4*>(
                                aout + ((size_t)b * plane + (size_t)ys[a] * pw + xs[c]) * COUT + 32 * h);
#pragma unroll
                            for (int u = 0; u < 4; ++u) p[u] = src[u];
                        }
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(tempty0 + 8 * s) : "memory");
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid == 0 && *abort) atomicOr(flag, FLAG_TIMEOUT);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(L::TMEM_COLS));
}

template <int CIN, int COUT, bool OUT>
cudaError_t conv_tc(const CUtensorMap& map, const __nv_bfloat16* W, const float* bias, int nb, int ny, int nx,
                    __nv_bfloat16* a, float* f, int* flag, int probe_polls, cudaStream_t st)
{
    using L = TcLayout<CIN, COUT>;
    static_assert(L::REQUEST <= 227 * 1024, "shared memory");
    static_assert(L::TMEM_COLS >= 32 && (L::TMEM_COLS & (L::TMEM_COLS - 1)) == 0, "tensor memory columns");
    cudaError_t e = tc::smem_attr_once<conv_tc_kernel<CIN, COUT, OUT>>(L::REQUEST);
    if (e != cudaSuccess) return e;
    const int sms = tc::sm_count();
    const long long tiles = (long long)nb * (nx / TC_PX) * (ny / TC_ROWS);
    const int grid = (int)std::min<long long>(tiles, sms);
    if (grid < 1) return cudaSuccess;
    conv_tc_kernel<CIN, COUT, OUT><<<grid, TC_THREADS, L::REQUEST, st>>>(map, W, bias, nb, ny, nx, a, f, flag,
                                                                         probe_polls);
    return cudaGetLastError();
}

}  // namespace

bool conv_tc_supported(int nx, int ny)
{
    return nx % TC_PX == 0 && ny % TC_ROWS == 0 && nx + 2 <= 65536;
}

cudaError_t launch_conv_tc(int layer_kind, const CUtensorMap& in_map, const __nv_bfloat16* W, const float* bias,
                           int nb, int ny, int nx, __nv_bfloat16* a, float* f, int* flag, int probe_polls,
                           cudaStream_t st)
{
    if (!conv_tc_supported(nx, ny) || probe_polls < 0) return cudaErrorInvalidValue;
    switch (layer_kind) {
    case 0: return conv_tc<16, 64, false>(in_map, W, bias, nb, ny, nx, a, f, flag, probe_polls, st);
    case 1: return conv_tc<64, 64, false>(in_map, W, bias, nb, ny, nx, a, f, flag, probe_polls, st);
    case 2: return conv_tc<64, 16, true>(in_map, W, bias, nb, ny, nx, a, f, flag, probe_polls, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace iewpf
