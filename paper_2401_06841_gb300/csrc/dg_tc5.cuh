// dg_tc5.cuh -- 5th-generation tensor-core (tcgen05) building blocks of the
// x3 kernels on sm_103a: shared-memory matrix descriptors, the instruction
// descriptor of kind::f16 products with FP32 accumulation in tensor memory
// (TMEM), bounded mbarrier waits, TMEM allocation and loads, and the split of
// FP32 data into BF16 components.
//
// Operand layout (no swizzle).  An operand tile is made of 8 x 16-byte core
// matrices.  K-major (rows x K): element (r, k) at
//     (r/8) SBO + (k/8) LBO + (r%8) 16 + (k%8) 2   bytes,
// MN-major (K rows of M contiguous elements): element (m, k) at
//     (m/8) SBO + (k/8) LBO + (k%8) 16 + (m%8) 2   bytes;
// in both LBO is the stride between K-groups of 8 and SBO the stride between
// row (M or N) groups of 8.  A product D[M][N] += A[M][K] B[N][K]^T with
// M = 128 keeps row i of D in TMEM lane i; with M = 64, row 16w + j in lane
// 32w + j (j < 16).
//
// Split-BF16 products: x = x0 + x1 with x0 = bf16(x), x1 = bf16(x - x0); the
// product a b is formed as a0 b0 + a0 b1 + a1 b0 (relative error ~ 2^-16),
// every term accumulated in FP32 in TMEM.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cstdint>

namespace dg {
namespace tc5 {

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor (no swizzle): start address, LBO and SBO in
// units of 16 bytes, descriptor version 1 at bit 46
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// the descriptor of the same layout `off` bytes further (off a multiple of 16;
// shared-memory addresses stay below 2^18, so the start-address field does not
// carry): one add per product instead of a descriptor built from scratch
__device__ __forceinline__ uint64_t dadd(uint64_t d, uint32_t off) { return d + (uint64_t)(off >> 4); }

// instruction descriptor: D FP32, A and B BF16, A/B K-major (0) or MN-major (1)
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int a_mn, int b_mn)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// one product D (+)= A B^T issued by the calling thread
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, bool accumulate)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"((uint32_t)accumulate));
}

// the same with lanes of D left untouched: bit i of word j set = lane 32 j + i not written
__device__ __forceinline__ void mma_masked(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, bool accumulate,
                                           uint32_t m0, uint32_t m1, uint32_t m2, uint32_t m3)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, {%5, %6, %7, %8}, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"((uint32_t)accumulate), "r"(m0), "r"(m1), "r"(m2), "r"(m3));
}

// arrive on the mbarrier once every product this thread has issued so far is complete
__device__ __forceinline__ void commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// wait for phase `parity` of the mbarrier to complete; false after `limit`
// unsuccessful polls (the caller records the failure and leaves)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit = (1u << 24))
{
    const uint32_t a = saddr(bar);
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.b32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// expect `bytes` of bulk-copy transactions on the mbarrier (and arrive once)
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}

// TMA bulk copy global -> shared of `bytes` (multiple of 16, both addresses
// 16-byte aligned), completing its transactions on the mbarrier
__device__ __forceinline__ void bulk_g2s(void* smem, const void* gmem, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(saddr(smem)),
        "l"(gmem), "r"(bytes), "r"(saddr(bar))
        : "memory");
}

// tiled TMA load of the box at (x, y) of a 2D tensor map (the map in kernel
// parameter space: a __grid_constant__ argument), completing on the mbarrier
__device__ __forceinline__ void tma_2d(void* smem, const CUtensorMap* map, int x, int y, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(saddr(smem)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(saddr(bar))
        : "memory");
}

// make generic-proxy shared-memory writes visible to the tensor cores
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// TMEM allocation by one whole warp; the column base lands in *slot
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// warp-collective loads: lane i of the warp reads TMEM lane (taddr.lane + i),
// N consecutive 32-bit columns from taddr.col
__device__ __forceinline__ void ld4(uint32_t taddr, float* v)
{
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t tmem_addr(uint32_t base, int lane0, int col)
{
    return base + ((uint32_t)lane0 << 16) + (uint32_t)col;
}

// split x into BF16 components: x ~ hi + lo
__device__ __forceinline__ void split2(float x, __nv_bfloat16& hi, __nv_bfloat16& lo)
{
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}
// four FP32 values -> 8 bytes of hi and 8 bytes of lo (BF16 pairs, element order kept)
__device__ __forceinline__ void split4(const float* x, uint2& hi, uint2& lo)
{
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(x[0], x[1]), h1 = __floats2bfloat162_rn(x[2], x[3]);
    const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
    const __nv_bfloat162 l0 = __floats2bfloat162_rn(x[0] - f0.x, x[1] - f0.y);
    const __nv_bfloat162 l1 = __floats2bfloat162_rn(x[2] - f1.x, x[3] - f1.y);
    hi.x = *reinterpret_cast<const uint32_t*>(&h0);
    hi.y = *reinterpret_cast<const uint32_t*>(&h1);
    lo.x = *reinterpret_cast<const uint32_t*>(&l0);
    lo.y = *reinterpret_cast<const uint32_t*>(&l1);
}
// eight FP32 values -> 16 bytes of hi and 16 bytes of lo
__device__ __forceinline__ void split8(const float* x, uint4& hi, uint4& lo)
{
    uint2 h0, l0, h1, l1;
    split4(x, h0, l0);
    split4(x + 4, h1, l1);
    hi = make_uint4(h0.x, h0.y, h1.x, h1.y);
    lo = make_uint4(l0.x, l0.y, l1.x, l1.y);
}

// byte offsets of the canonical layouts
__host__ __device__ constexpr int koff(int r, int k, int lbo, int sbo)
{
    return (r >> 3) * sbo + (k >> 3) * lbo + (r & 7) * 16 + (k & 7) * 2;
}
__host__ __device__ constexpr int mnoff(int m, int k, int lbo, int sbo)
{
    return (m >> 3) * sbo + (k >> 3) * lbo + (k & 7) * 16 + (m & 7) * 2;
}

}  // namespace tc5
}  // namespace dg
