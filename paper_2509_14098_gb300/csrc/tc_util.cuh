// tc_util.cuh — small device helpers shared by the tensor-core stage kernels (sm_103a):
// shared-memory addresses, the tcgen05 matrix / instruction descriptors, MMA commit and
// the TF32 rounding used by the split-precision operands.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace svk {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor, K-major, 128-byte swizzle: start >> 4, LBO (unused
// for this layout) 1, SBO = 1024 bytes between 8-row groups, version 1, swizzle mode 2
__device__ __forceinline__ uint64_t mdesc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// instruction descriptor: FP32 accumulator, A / B format (1 = BF16, 2 = TF32), both
// K-major, N, M = 128
__device__ __forceinline__ uint32_t idesc(uint32_t fmt, uint32_t N) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((128u >> 4) << 24);
}
__device__ __forceinline__ void cp_async16g(uint32_t saddr, const void* g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// round to the nearest TF32 value (10 mantissa bits, ties to even): both halves of the
// split are then exactly representable, whatever the MMA does with the low bits
__device__ __forceinline__ float rn_tf32(float x) {
    const uint32_t b = __float_as_uint(x);
    return __uint_as_float((b + 0x0FFFu + ((b >> 13) & 1u)) & 0xFFFFE000u);
}

// one poll of an mbarrier phase
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile("{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, q;\n\t}"
                 : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    return done != 0;
}

}  // namespace svk
