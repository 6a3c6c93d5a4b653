// Device helpers of the tcgen05 kernels (conv_tc.cu, conv_tr.cu): shared-
// memory matrix descriptors, the instruction descriptor of a BF16 x BF16 ->
// FP32 product, bounded mbarrier waits and tensor-memory loads.
#pragma once
#include <atomic>
#include <cstdint>

#include <cuda_runtime.h>

namespace iewpf {
namespace tc {

// host: the dynamic shared-memory limit of kernel K, set once per device
// (setting it twice from two threads is harmless)
template <auto K>
inline cudaError_t smem_attr_once(int bytes)
{
    static std::atomic<unsigned long long> done{0};     // bit d: set on device d
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 64 && ((done.load(std::memory_order_acquire) >> dev) & 1ull)) return cudaSuccess;
    e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && dev < 64) done.fetch_or(1ull << dev, std::memory_order_release);
    return e;
}

// host: SM count of the current device (cached per device)
inline int sm_count()
{
    static std::atomic<int> cache[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev < 64) {
        const int c = cache[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;
    if (dev < 64) cache[dev].store(sms, std::memory_order_relaxed);
    return sms;
}

constexpr long long WAIT_LIMIT = 1LL << 24;

__device__ __forceinline__ uint32_t su32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor.  layout 0 = no swizzle, 2 = 128-byte
// swizzle, 6 = 32-byte swizzle.  K-major operands: lbo = bytes between core
// matrices along K (no swizzle), sbo = bytes between 8-row groups along M/N.
// M/N-major operands: swizzled, lbo = bytes between 64-element (128-byte
// swizzle) blocks along M/N and sbo = bytes between 8-row groups along K; no
// swizzle, lbo = bytes between 8-row groups along K and sbo = bytes between
// 8-element core matrices along M/N.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo, uint32_t layout)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46) | ((uint64_t)(layout & 7) << 61);
}

// instruction descriptor: BF16 A and B, FP32 D, M x N; a_mn / b_mn select the
// M/N-major (transposed) form of A / B
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int a_mn = 0, int b_mn = 0)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// bounded wait for the phase of `parity`; gives up when the CTA aborted
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort,
                                          long long limit = WAIT_LIMIT)
{
    for (long long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (done) return true;
        if ((it & 255) == 255 && *abort) return false;
    }
    *abort = 1;
    return false;
}

// the same without the abort check (draining after an abort)
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity)
{
    for (long long it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (done) return;
    }
}

__device__ __forceinline__ void tmem_ld16(uint32_t ta, float* v)
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                 "[%16];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// 32 consecutive accumulator columns of the warp's 32 lanes (one register each)
__device__ __forceinline__ void tmem_ld32(uint32_t ta, uint32_t* r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                   "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                   "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ void mma_bf16_ss(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc)
{
    if (acc)
        asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 1;\n" ::"r"(d), "l"(adesc), "l"(bdesc),
                     "r"(idesc));
    else
        asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 0;\n" ::"r"(d), "l"(adesc), "l"(bdesc),
                     "r"(idesc));
}

// stage the weights of every tap once per CTA (B operand, K-major, rows =
// output channels): 128-byte swizzled rows of 64 input channels, or core
// matrices of 8 output channels x 16 bytes ([tap][chunk][co][8 ch]).  Every
// thread issues all its loads before its first store, so the copy costs one
// round trip to L2 rather than one per chunk.  With KXMAJOR (64 input
// channels) the tap blocks are ordered [kx][ky = 2, 1, 0], so that the
// blocks of ky and ky - 1 at one kx are adjacent rows of one operand.
template <int CIN, int COUT, int NTHREADS, bool KXMAJOR = false>
__device__ __forceinline__ void stage_weights(unsigned char* wsm, const void* __restrict__ W, int tid)
{
    constexpr int N = 9 * COUT * (CIN / 8);                 // 16-byte chunks
    constexpr int PER = (N + NTHREADS - 1) / NTHREADS;
    uint4 r[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = tid + k * NTHREADS;
        if (i < N) r[k] = __ldg(reinterpret_cast<const uint4*>(W) + i);
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = tid + k * NTHREADS;
        if (i < N) {
            // chunk i of W: row (tap, co), channels 8 c .. 8 c + 7
            const int c = i % (CIN / 8), co = (i / (CIN / 8)) % COUT, tap = i / ((CIN / 8) * COUT);
            const int blk = KXMAJOR ? (tap % 3) * 3 + 2 - tap / 3 : tap;
            const int off = CIN == 64 ? (blk * COUT + co) * 128 + ((c ^ (co & 7)) << 4)
                                      : ((tap * (CIN / 8) + c) * COUT + co) * 16;
            *reinterpret_cast<uint4*>(wsm + off) = r[k];
        }
    }
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

}  // namespace tc
}  // namespace iewpf
