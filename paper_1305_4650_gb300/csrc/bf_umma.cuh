// Fifth-generation tensor-core (tcgen05) building blocks, as inline PTX for sm_100-family
// GPUs (compiled for sm_103a): tensor-memory allocation, shared-memory matrix descriptors,
// the instruction descriptors of BF16 x BF16 -> FP32 and TF32 x TF32 -> FP32 MMAs, the MMAs,
// their completion on an mbarrier and the loads of the FP32 accumulator from tensor memory.
//
// Operand layout (both operands K-major, no swizzle).  A matrix of 16-bit elements is
// stored as "core matrices" of 8 rows x 16 bytes (8 elements of K), each 128 contiguous
// bytes, row r of the core matrix at byte 16 r.  Element (row, k) lives at
//     start + (row / 8) * SBO + (k / 8) * LBO + (row % 8) * 16 + (k % 8) * 2,
// where LBO (the "leading dimension byte offset") steps between core matrices along K and
// SBO (the "stride dimension byte offset") between groups of 8 rows.  One MMA of
// kind::f16 consumes K = 16, i.e. two core matrices along K; the next K step starts
// 2 LBO further on.  With 32-bit elements (TF32) a core matrix holds 8 rows x 4 elements
// of K, element (row, k) at start + (row / 8) * SBO + (k / 4) * LBO + (row % 8) * 16 +
// (k % 4) * 4, and one MMA of kind::tf32 consumes K = 8: again two core matrices.
//
// Accumulator layout (cta_group::1, M = 128): row i of D is tensor-memory lane i, column j
// is column base + j, one FP32 value per (lane, column).  A warp can read only the lane
// quarter 32 (warp % 4) .. 32 (warp % 4) + 31 (tcgen05.ld of shape 32x32b: thread i of the
// warp receives lane 32 (warp % 4) + i).
#pragma once

#include <cstdint>

namespace bfk {
namespace umma {

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle, descriptor version 1 (bits 46-48),
// base offset 0, relative leading-dimension offset, swizzle mode 0 (bits 61-63)
__device__ __forceinline__ uint64_t desc_kmajor(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of tcgen05.mma kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 and 10-12 = 1), no negation, both K-major (bits 15, 16 = 0), N / 8 in bits
// 17-22, M / 16 in bits 24-28
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// instruction descriptor of tcgen05.mma kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32
// (bits 7-9 and 10-12 = 2), no negation, both K-major, N / 8 in bits 17-22, M / 16 in bits
// 24-28
__host__ __device__ constexpr uint32_t idesc_tf32_f32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of the 16-byte piece `piece` along K (elements k = piece * (16 / element
// size) ...) of row `row` in a K-major, unswizzled operand
__host__ __device__ constexpr uint32_t kmajor_piece_off(int row, int piece, uint32_t lbo, uint32_t sbo)
{
    return (uint32_t)(row >> 3) * sbo + (uint32_t)piece * lbo + (uint32_t)(row & 7) * 16u;
}

// byte offset of element (row, k) in a K-major, unswizzled operand (see above)
__host__ __device__ constexpr uint32_t kmajor_off(int row, int k, uint32_t lbo, uint32_t sbo)
{
    return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 3) * lbo + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

// D (+)= A B^T over one K step of 16; issued by one thread
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// D (+)= A B^T over one K step of 8 TF32 elements; issued by one thread
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// arrive (once) on the mbarrier when every MMA this thread issued so far has completed
__device__ __forceinline__ void commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}

// tensor-memory allocation of ncols columns (a power of two >= 32) by one whole warp; the
// address is written to *slot in shared memory
__device__ __forceinline__ void alloc(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// ordering of tensor-core operations around thread synchronisation
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// generic-proxy writes to shared memory made visible to the tensor cores (async proxy)
__device__ __forceinline__ void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 8 consecutive FP32 columns of this warp's 32 lanes (warp-collective); the wait for the
// load is part of the same statement, so no use of v can be scheduled before it
__device__ __forceinline__ void ld8(uint32_t taddr, float v[8])
{
    uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
        : "r"(taddr)
        : "memory");
    v[0] = __uint_as_float(r0);
    v[1] = __uint_as_float(r1);
    v[2] = __uint_as_float(r2);
    v[3] = __uint_as_float(r3);
    v[4] = __uint_as_float(r4);
    v[5] = __uint_as_float(r5);
    v[6] = __uint_as_float(r6);
    v[7] = __uint_as_float(r7);
}

// split x into BF16 parts: hi = x rounded to BF16, lo = (x - hi) rounded to BF16, so that
// hi + lo carries 16 significant bits; two values at a time, packed as stored along K
// (the first value at the lower address)
__device__ __forceinline__ void split2(float x0, float x1, uint32_t &hi, uint32_t &lo)
{
    uint32_t h;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(x1), "f"(x0));
    const float h0 = __uint_as_float(h << 16), h1 = __uint_as_float(h & 0xFFFF0000u);
    uint32_t l;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(l) : "f"(__fsub_rn(x1, h1)), "f"(__fsub_rn(x0, h0)));
    hi = h;
    lo = l;
}

// split x into TF32 parts: hi = x rounded to TF32 (10 stored mantissa bits), lo = (x - hi)
// (exact in FP32) rounded to TF32, so that hi + lo carries 22 significant bits; each part
// as the 32-bit word the tensor core reads
__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo)
{
    uint32_t h, l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(__fsub_rn(x, __uint_as_float(h))));
    hi = h;
    lo = l;
}

}  // namespace umma
}  // namespace bfk
