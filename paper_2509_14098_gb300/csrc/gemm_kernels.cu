// gemm_kernels.cu — a fused stage applied as a split-precision tensor-core GEMM:
// D (2^(k+1) x columns) = Ut (2^(k+1) x 2^(k+1)) * B (the tile's columns), with
// Ut ~ Ahi + Alo, B ~ Bhi + Blo and D ~ Ahi Bhi + Ahi Blo + Alo Bhi accumulated in
// FP32 in tensor memory (TF32x3, Ootomo-Yokota style; BF16x3, Henry et al. style).
//
// sm_103a: operands in shared memory in the canonical no-swizzle K-major layout
// (core matrix = 8 rows x 16 bytes), tcgen05.mma issued by one thread, completion via
// tcgen05.commit -> mbarrier (bounded wait: on time-out the kernel raises an error flag,
// frees its tensor memory and returns), accumulators read with tcgen05.ld.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "gemm.h"

namespace svk {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start >> 4, LBO >> 4, SBO >> 4, version 1, no swizzle
__device__ __forceinline__ uint64_t mdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor: FP32 accumulator, A/B format (1 = BF16, 2 = TF32), K-major, N, M
__device__ __forceinline__ uint32_t idesc(uint32_t fmt, uint32_t M, uint32_t N) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}
__device__ __forceinline__ void cp_async8(void* smem, const void* g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(smem)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async16g(void* smem, const void* g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(g) : "memory");
}

// round to the nearest TF32 value (10 mantissa bits, ties to even): both halves of the
// split are then exactly representable, whatever the MMA does with the low bits
__device__ __forceinline__ float rn_tf32(float x) {
    const uint32_t b = __float_as_uint(x);
    return __uint_as_float((b + 0x0FFFu + ((b >> 13) & 1u)) & 0xFFFFE000u);
}

constexpr int kThreads = 128;
constexpr uint32_t kWaitLimit = 1u << 24;

template <int PREC>   // 1 = TF32x3, 2 = BF16x3
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_stage(float2* __restrict__ psi, const GemmStage* __restrict__ stp, const uint8_t* __restrict__ ablob,
                 int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ int s_fail;
    const GemmStage& st = *stp;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t M_total = 2u << st.keff;           // rows of Ut
    const uint32_t ncols = 1u << st.ncol_bits;         // N of the MMA
    const uint32_t nacc = st.nacc;
    // shared memory: A chunk (hi | lo), B staging (fp32, 16 KB for 128 columns), B lo
    // (TF32) or B hi | lo (BF16).  After the K loop the same space holds the output
    // staging (16 KB per warp).
    const uint32_t abytes = st.a_chunk_bytes;
    unsigned char* sA = sm;
    float* sB = reinterpret_cast<float*>(sm + abytes);                     // fp32 chunk, 128 x 32
    unsigned char* sB2 = sm + abytes + 16384;                               // TF32: lo; BF16: hi | lo
    const uint32_t B2bytes = PREC == 1 ? 16384 : 16384;
    (void)B2bytes;
    float* stg = reinterpret_cast<float*>(sm);                              // [warp][32 rows][128 cols]

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        s_fail = 0;
    }
    const uint32_t tcols = nacc * 128;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    uint32_t phase = 0;
    const uint64_t ntiles = 1ull << st.n_glob;
    const uint32_t nvar = st.nvar;
    const uint32_t namp = 1u << nvar;                 // amplitudes per chunk (16 x columns)
    const uint32_t id = idesc(PREC == 1 ? 2u : 1u, 128u, ncols);
    const uint32_t LBO = 128;
    const uint32_t SBO_A = PREC == 1 ? 1024u : 512u;  // 32 K elements per row
    const int KSTEPS = PREC == 1 ? 4 : 2;             // MMA K-steps per 32-element chunk

    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        uint64_t base = 0;
        for (uint32_t i = 0; i < st.n_glob; ++i)
            if ((tile >> i) & 1) base |= 1ull << st.glob_pos[i];
        for (uint32_t c = 0; c < st.nchunk; ++c) {
            uint64_t cbase = base;
            for (uint32_t j = 0; 4 + j < st.keff; ++j)
                if ((c >> j) & 1) cbase |= st.hi_local[j];
            // A chunk: contiguous, preformatted
            {
                const uint8_t* src = ablob + st.a_off + (uint64_t)c * abytes;
                for (uint32_t o = (uint32_t)tid * 16; o < abytes; o += kThreads * 16) cp_async16g(sA + o, src + o);
            }
            // state chunk: amplitude (jj, n) -> canonical fp32 position of floats 2jj, 2jj+1 of row n
            for (uint32_t t = tid; t < namp; t += kThreads) {
                uint64_t p = cbase;
                uint32_t jj = 0, n = 0;
                for (uint32_t b = 0; b < nvar; ++b)
                    if ((t >> b) & 1) {
                        p |= st.var_phys[b];
                        const uint32_t r = st.var_role[b];
                        if (r < 8) jj |= 1u << r;
                        else n |= 1u << (r - 8);
                    }
                unsigned char* dst = reinterpret_cast<unsigned char*>(sB) + (n >> 3) * 1024 + (jj >> 1) * 128 +
                                     (n & 7) * 16 + (jj & 1) * 8;
                cp_async8(dst, psi + p);
            }
            asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
            __syncthreads();
            // split B in shared memory
            for (uint32_t e = tid; e < ncols * 32; e += kThreads) {
                // e walks the fp32 canonical buffer (only the first ncols rows are used)
                const uint32_t row = e >> 5, kk = e & 31;
                const uint32_t off32 = (row >> 3) * 1024 + (kk >> 2) * 128 + (row & 7) * 16 + (kk & 3) * 4;
                const float x = *reinterpret_cast<const float*>(reinterpret_cast<const unsigned char*>(sB) + off32);
                if (PREC == 1) {
                    const float hi = rn_tf32(x);
                    *reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(sB) + off32) = hi;
                    *reinterpret_cast<float*>(sB2 + off32) = rn_tf32(x - hi);
                } else {
                    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
                    const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
                    const uint32_t off16 = (row >> 3) * 512 + (kk >> 3) * 128 + (row & 7) * 16 + (kk & 7) * 2;
                    *reinterpret_cast<__nv_bfloat16*>(sB2 + off16) = hi;
                    *reinterpret_cast<__nv_bfloat16*>(sB2 + 8192 + off16) = lo;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t aH = smem_u32(sA), aL = smem_u32(sA + abytes / 2);
                const uint32_t bH = PREC == 1 ? smem_u32(sB) : smem_u32(sB2);
                const uint32_t bL = PREC == 1 ? smem_u32(sB2) : smem_u32(sB2 + 8192);
                const uint32_t SBO_B = SBO_A;
                for (uint32_t a = 0; a < nacc; ++a) {
                    const uint32_t aoff = a * 16 * SBO_A;   // 128 rows = 16 row groups
                    for (int p = 0; p < 3; ++p) {
                        const uint32_t As = (p == 2 ? aL : aH) + aoff;
                        const uint32_t Bs = (p == 1 ? bL : bH);
                        for (int s = 0; s < KSTEPS; ++s) {
                            const uint64_t da = mdesc(As + s * 2 * LBO, LBO, SBO_A);
                            const uint64_t db = mdesc(Bs + s * 2 * LBO, LBO, SBO_B);
                            const uint32_t acc = (c > 0 || p > 0 || s > 0) ? 1u : 0u;
                            const uint32_t d = tmem + a * 128;
                            if (PREC == 1)
                                asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                                             "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q;\n\t}"
                                             ::"r"(d), "l"(da), "l"(db), "r"(id), "r"(acc));
                            else
                                asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n\t}"
                                             ::"r"(d), "l"(da), "l"(db), "r"(id), "r"(acc));
                        }
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(smem_u32(&mbar)) : "memory");
            }
            // bounded wait for the MMAs (they read sA / sB before the next chunk overwrites them)
            uint32_t done = 0;
            for (uint32_t it = 0; it < kWaitLimit && !done; ++it)
                asm volatile("{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
                             "selp.u32 %0, 1, 0, q;\n\t}"
                             : "=r"(done) : "r"(smem_u32(&mbar)), "r"(phase) : "memory");
            if (!done) s_fail = 1;
            phase ^= 1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            __syncthreads();
            if (s_fail) break;
        }
        if (s_fail) break;
        // readback: warp w owns TMEM lanes 32w..32w+31 = rows 128a + 32w + lane of Ut,
        // i.e. output chunk c_out = 4a + w (16 amplitudes, re/im in adjacent rows)
        float* my = stg + (size_t)warp * 32 * 128;
        for (uint32_t a = 0; a < nacc; ++a) {
            for (uint32_t n0 = 0; n0 < ncols; n0 += 32) {
                uint32_t r[32];
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + a * 128 + n0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                      "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                      "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                for (int j = 0; j < 32; ++j)
                    if (n0 + j < ncols) my[lane * 128 + ((n0 + j + lane) & 127)] = __uint_as_float(r[j]);
            }
            __syncwarp();
            const uint32_t cout = 4 * a + (uint32_t)warp;
            uint64_t cbase = base;
            for (uint32_t j = 0; 4 + j < st.keff; ++j)
                if ((cout >> j) & 1) cbase |= st.hi_local[j];
            for (uint32_t t = lane; t < namp; t += 32) {
                uint64_t p = cbase;
                uint32_t jj = 0, n = 0;
                for (uint32_t b = 0; b < nvar; ++b)
                    if ((t >> b) & 1) {
                        p |= st.var_phys[b];
                        const uint32_t rr = st.var_role[b];
                        if (rr < 8) jj |= 1u << rr;
                        else n |= 1u << (rr - 8);
                    }
                float2 v;
                v.x = my[(2 * jj) * 128 + ((n + 2 * jj) & 127)];
                v.y = my[(2 * jj + 1) * 128 + ((n + 2 * jj + 1) & 127)];
                psi[p] = v;
            }
            __syncwarp();
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();   // staging overlaps the operand buffers of the next tile
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (s_fail && tid == 0) atomicExch(status, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
}

}  // namespace

size_t gemm_smem_bytes(const GemmStage& st) {
    // A chunk + B fp32 staging + B second buffer, at least the output staging
    return std::max<size_t>((size_t)st.a_chunk_bytes + 16384 + 16384, (size_t)4 * 32 * 128 * 4);
}

cudaError_t launch_gemm_stage(int prec, void* psi, const GemmStage* d_stage, const GemmStage& hst,
                              const uint8_t* d_ablob, int* d_status, cudaStream_t s) {
    const size_t smem = gemm_smem_bytes(hst);
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t ntiles = 1ull << hst.n_glob;
    // one CTA per SM: each holds up to 256 tensor-memory columns
    const unsigned grid = (unsigned)std::min<uint64_t>(ntiles, (uint64_t)nsm);
    // the kernel also holds ~1 KB of static shared memory: request only what it can use
    constexpr int kMaxDyn = 128 * 1024;
    if (smem > (size_t)kMaxDyn) return cudaErrorInvalidConfiguration;
    if (prec == 1) {
        static bool cfg = false;
        if (!cfg) {
            cudaError_t e = cudaFuncSetAttribute(k_gemm_stage<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn);
            if (e != cudaSuccess) return e;
            cfg = true;
        }
        k_gemm_stage<1><<<grid, kThreads, smem, s>>>((float2*)psi, d_stage, d_ablob, d_status);
    } else {
        static bool cfg = false;
        if (!cfg) {
            cudaError_t e = cudaFuncSetAttribute(k_gemm_stage<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn);
            if (e != cudaSuccess) return e;
            cfg = true;
        }
        k_gemm_stage<2><<<grid, kThreads, smem, s>>>((float2*)psi, d_stage, d_ablob, d_status);
    }
    return cudaGetLastError();
}

}  // namespace svk
