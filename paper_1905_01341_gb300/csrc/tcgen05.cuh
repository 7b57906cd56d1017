// Building blocks of the tcgen05 (5th-generation tensor core) kernels: shared-memory operand
// descriptors for the canonical K-major layout without swizzle, the kind::f16 instruction
// descriptor and MMA issue, mbarrier waits with an iteration limit, cp.async and bulk (TMA
// engine) copies, and the three-piece BF16 split that makes BF16 products as accurate as FP32.
//
// Operand layout: one 16-wide K step of an operand block of `rows` rows is rows x 16 BF16
// elements in 8-row x 16-byte core matrices, K-adjacent core matrices 128 B apart (LBO) and
// 8-row groups 256 B apart (SBO); kmajor_off gives the element offset of (row, kk).
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace bem {
namespace {

constexpr int TC_K = 16;         // K per stage (one kind::f16 MMA)
constexpr uint32_t TC_LBO = 128;  // bytes between K-adjacent core matrices
constexpr uint32_t TC_SBO = 256;  // bytes between 8-row groups
constexpr long long kWaitLimit = 1ll << 20;  // iterations before a wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((TC_LBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((TC_SBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for this architecture; no swizzle, base offset 0
    return d;
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, N and M given.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (long long it = 0; it < kWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 16-byte global -> shared copy; src_bytes = 0 writes zeros without reading.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Bulk copy (the TMA engine, no tensor map) of `bytes` contiguous bytes global -> shared; it
// counts its bytes on `mbar`, whose phase the issuing thread opened with expect_tx. Both
// addresses and the size are multiples of 16 bytes.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// element offset of (row, kk) inside one 16-wide K step of a K-major operand block
__host__ __device__ constexpr int kmajor_off(int row, int kk) {
    return (row >> 3) * 128 + (kk >> 3) * 64 + (row & 7) * 8 + (kk & 7);
}

// three-piece BF16 split of an FP64 value (operator tables)
__device__ __forceinline__ void split3_d(double v, __nv_bfloat16 &b0, __nv_bfloat16 &b1, __nv_bfloat16 &b2) {
    b0 = __double2bfloat16(v);
    double r = v - (double)__bfloat162float(b0);
    b1 = __double2bfloat16(r);
    r -= (double)__bfloat162float(b1);
    b2 = __double2bfloat16(r);
}

// three-piece BF16 split of an FP32 value (each difference is exact in FP32)
__device__ __forceinline__ void split3_f(float v, __nv_bfloat16 &b0, __nv_bfloat16 &b1, __nv_bfloat16 &b2) {
    b0 = __float2bfloat16_rn(v);
    float r = v - __bfloat162float(b0);
    b1 = __float2bfloat16_rn(r);
    r -= __bfloat162float(b1);
    b2 = __float2bfloat16_rn(r);
}

}  // namespace
}  // namespace bem
