// hier_kernels.cu — the hierarchical tensor-core stage (hier.h), sm_103a.
//
// One CTA of 256 threads per tile of T = k + 7 qubits, persistent over the tiles, several
// CTAs per SM (their phases interleave on the SM's tensor core and memory pipes):
//  1. the tile's 2^T amplitudes are read from HBM once (16-byte pairs: qubits 0..3 are
//     tile bits, so a warp reads whole 128-byte runs), split into hi / lo halves and
//     stored as sub-partition 0's A operand (128 rows = the columns of its k qubits);
//  2. per sub-partition s: one thread issues the 3 x (K / 32 bytes) tcgen05.mma of
//     D = Ahi Bhi + Alo Bhi + Ahi Blo into tensor memory and commits them; the B operand
//     (the fused unitary, pre-split by the host) arrives by one bulk copy that is issued
//     as soon as the previous sub-partition's MMAs are done; every thread then reads half
//     a row of D (tcgen05.ld) and stores it, split again, as sub-partition s + 1's A
//     operand, or after the last one into the FP32 output tile (same shared memory);
//  3. the tile is written back to HBM once.
// Every wait is bounded: on time-out the kernel raises the status flag, waits (bounded)
// for the copies and MMAs it issued, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>

#include "hier.h"
#include "tc_util.cuh"

namespace svk {

namespace {

constexpr int kHT = 256;                 // threads: two per A row / tensor-memory lane (each half the columns)
constexpr uint32_t kHWait = 1u << 22;    // polls of a bounded wait

// an amplitude (re, im) split into hi / lo halves at A offset o (lo 16384 bytes above)
template <int PREC>
__device__ __forceinline__ void put_amp(unsigned char* A, uint32_t o, float re, float im) {
    if (PREC == 1) {
        const float hr = rn_tf32(re), hi = rn_tf32(im);
        *reinterpret_cast<float2*>(A + o) = make_float2(hr, hi);
        *reinterpret_cast<float2*>(A + o + 16384) = make_float2(rn_tf32(re - hr), rn_tf32(im - hi));
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
        const float2 f = __bfloat1622float2(h);
        *reinterpret_cast<__nv_bfloat162*>(A + o) = h;
        *reinterpret_cast<__nv_bfloat162*>(A + o + 16384) = __floats2bfloat162_rn(re - f.x, im - f.y);
    }
}

template <int PREC, int KS>
__global__ void __launch_bounds__(kHT, 4)
    k_hier_stage(float2* __restrict__ psi, const HierStage* __restrict__ stp, const uint8_t* __restrict__ ublob,
                 int* __restrict__ status) {
    constexpr uint32_t T = KS + 7, N = 2u << KS, K2 = 1u << KS;
    constexpr uint32_t CAMP = PREC == 1 ? 4 : 5;                 // log2 amplitudes per K chunk
    constexpr uint32_t NCHUNK = 1u << (KS - CAMP);
    constexpr uint32_t NROUND = 1u << (T - 9);                  // 16-byte pairs per thread
    constexpr uint32_t A_BYTES = NCHUNK * 32768, B_BYTES = NCHUNK * 2 * N * 128;
    extern __shared__ unsigned char sm_raw[];
    __shared__ HierStage s_st;
    __shared__ uint64_t s_gr[NROUND];                           // round -> physical offset
    __shared__ uint32_t s_ar[NROUND], s_tr[NROUND];             // round -> layout-0 / output-tile offset
    __shared__ __align__(8) uint64_t bar_b[2], bar_mma, bar_fin;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_fail;
    static_assert(sizeof(HierStage) % 4 == 0, "stage copy");

    const uint32_t tid = threadIdx.x, warp = tid >> 5;
    for (uint32_t i = tid; i < sizeof(HierStage) / 4; i += kHT)
        reinterpret_cast<uint32_t*>(&s_st)[i] = reinterpret_cast<const uint32_t*>(stp)[i];
    if (tid == 0) s_fail = 0;
    __syncthreads();
    const HierStage& st = s_st;
    const uint32_t nsub = st.n_sub;
    const uint32_t sbase = (smem_u32(sm_raw) + 1023u) & ~1023u;
    unsigned char* const Ab = sm_raw + (sbase - smem_u32(sm_raw));
    const uint32_t Aaddr = sbase, Baddr = sbase + A_BYTES;
    uint32_t* const oj = reinterpret_cast<uint32_t*>(Ab + A_BYTES + st.b_slots * B_BYTES);   // [nsub][2^k]

    // amplitude-offset tables: oj[s][j] = XOR over the bits of j of the next layout's term
    // of sub-partition s's amplitude bit
    for (uint32_t i = tid; i < nsub * K2; i += kHT) {
        const uint32_t s = i / K2, j = i % K2;
        uint32_t o = 0;
        for (uint32_t b = 0; b < (uint32_t)KS; ++b)
            if ((j >> b) & 1) o ^= st.ao[s + 1][st.amp_bits[s][b]];
        oj[i] = o;
    }
    if (tid < NROUND) {
        uint64_t g = 0;
        uint32_t a = 0, t = 0;
        for (uint32_t b = 0; b + 9 < T; ++b)
            if ((tid >> b) & 1) {
                const uint32_t tb = st.ld_bits[8 + b];
                g |= 1ull << st.tile_pos[tb];
                a ^= st.ao[0][tb];
                t ^= st.ao[nsub][tb];
            }
        s_gr[tid] = g;
        s_ar[tid] = a;
        s_tr[tid] = t;
    }
    // this thread's part of a pair index: thread bit b <- tile bit ld_bits[b]
    uint64_t gthr = 0;
    uint32_t athr = 0, tthr = 0;
    for (uint32_t b = 0; b < 8; ++b)
        if ((tid >> b) & 1) {
            const uint32_t tb = st.ld_bits[b];
            gthr |= 1ull << st.tile_pos[tb];
            athr ^= st.ao[0][tb];
            tthr ^= st.ao[nsub][tb];
        }
    const uint32_t a0b = st.ao[0][0];   // the pair's second amplitude (tile bit 0) in layout 0
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_b[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_b[1])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_mma)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_fin)));
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint64_t ntiles = 1ull << st.n_glob;

    // B operands in st.b_slots buffers (thread 0 manages them).  When the launch's
    // sub-partitions fit, each keeps its own buffer for the whole launch (one copy per
    // CTA).  Otherwise MMA group g (sub-partition g mod n_sub) uses buffer g mod b_slots:
    // with two buffers the copy for group g + 1 is issued just before group g's MMAs (its
    // buffer's previous group has completed), with one after group g's MMAs complete.
    const uint32_t NBS = st.b_slots;
    const bool resident = nsub <= NBS;
    uint32_t nload0 = 0, nload1 = 0;   // copies issued per buffer
    uint32_t pendm = 0;                // buffers with a copy not yet waited for (bit mask)
    auto load_b = [&](uint32_t slot, uint32_t s) {
        const uint32_t bar = smem_u32(&bar_b[slot]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(B_BYTES) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(Baddr + slot * B_BYTES), "l"(ublob + st.b_off + (size_t)s * B_BYTES), "r"(B_BYTES),
                     "r"(bar)
                     : "memory");
        if (slot) ++nload1;
        else ++nload0;
        pendm |= 1u << slot;
    };
    // bounded wait; gives up at once when another thread already failed
    auto wait = [&](uint64_t& bar, uint32_t parity) -> bool {
        const uint32_t a = smem_u32(&bar);
        for (uint32_t it = 0; it < kHWait; ++it) {
            if (mbar_test(a, parity)) return true;
            if (s_fail) return false;
        }
        s_fail = 1;
        return false;
    };
    uint32_t nm = 0;          // MMA groups committed (every thread counts them)
    if (tid == 0 && (uint64_t)blockIdx.x < ntiles) {
        if (resident)
            for (uint32_t s = 0; s < nsub; ++s) load_b(s, s);
        else
            load_b(0, 0);
    }

    bool ok = true;
    for (uint64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        uint64_t base = 0;
        for (uint32_t i = 0; i < st.n_glob; ++i)
            if ((t >> i) & 1) base |= 1ull << st.glob_pos[i];
        // 1. the tile from HBM into sub-partition 0's A operand
        {
            float4 v[NROUND];
#pragma unroll
            for (uint32_t r = 0; r < NROUND; ++r) v[r] = *reinterpret_cast<const float4*>(psi + (base | gthr | s_gr[r]));
#pragma unroll
            for (uint32_t r = 0; r < NROUND; ++r) {
                const uint32_t o = athr ^ s_ar[r];
                put_amp<PREC>(Ab, o, v[r].x, v[r].y);
                put_amp<PREC>(Ab, o ^ a0b, v[r].z, v[r].w);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the tensor core
        __syncthreads();
        // 2. the sub-partitions, one GEMM each
        for (uint32_t s = 0; s < nsub; ++s) {
            if (tid == 0) {
                bool go = !s_fail;
                const uint32_t slot = resident ? s : nm % NBS;
                if (go && !resident && NBS == 2 && (s + 1 < nsub || t + gridDim.x < ntiles))
                    load_b((nm + 1) % NBS, (s + 1) % nsub);   // the next group's operand
                if (go && ((pendm >> slot) & 1u)) {
                    go = wait(bar_b[slot], ((slot ? nload1 : nload0) - 1) & 1u);
                    pendm &= ~(1u << slot);
                }
                if (go) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t id = idesc(PREC == 1 ? 2u : 1u, N);
#pragma unroll
                    for (uint32_t c = 0; c < NCHUNK; ++c)
#pragma unroll
                        for (int p = 0; p < 3; ++p) {   // hi*hi, lo*hi, hi*lo
                            const uint32_t As = Aaddr + c * 32768u + (p == 1 ? 16384u : 0u);
                            const uint32_t Bs = Baddr + slot * B_BYTES + c * (2u * N * 128u) + (p == 2 ? N * 128u : 0u);
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const uint64_t da = mdesc(As + 32u * q), db = mdesc(Bs + 32u * q);
                                const uint32_t acc = (c > 0 || p > 0 || q > 0) ? 1u : 0u;
                                if (PREC == 1)
                                    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                                                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q;\n\t}"
                                                 ::"r"(tmem), "l"(da), "l"(db), "r"(id), "r"(acc));
                                else
                                    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                                                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n\t}"
                                                 ::"r"(tmem), "l"(da), "l"(db), "r"(id), "r"(acc));
                            }
                        }
                }
                // committed even when nothing was issued: the barrier phase then completes
                // at once and every thread's count stays in step
                mma_commit(smem_u32(&bar_mma));
            }
            ++nm;
            const bool mine = wait(bar_mma, (nm - 1) & 1u);
            if (__syncthreads_or(!mine || s_fail)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // one buffer: the next group's operand streams in while this one's results are
            // read out
            if (tid == 0 && !resident && NBS == 1 && (s + 1 < nsub || t + gridDim.x < ntiles)) load_b(0, (s + 1) % nsub);
            // epilogue: row m of D (warp w reads tensor-memory lanes 32 (w & 3) ..; warps
            // 0..3 take the first half of the columns, 4..7 the second), stored through the
            // next layout
            const bool last = s + 1 == nsub;
            const uint32_t L = s + 1;
            const uint32_t m = 32u * (warp & 3u) + (tid & 31u), nh = (warp >> 2) * (N / 2);
            uint32_t om = 0;
            for (uint32_t i = 0; i < 7; ++i)
                if ((m >> i) & 1) om ^= st.ao[L][st.col_bits[s][i]];
            const uint32_t* ojs = oj + s * K2;
#pragma unroll
            for (uint32_t n1 = 0; n1 < N / 2; n1 += 32) {
                const uint32_t n0 = nh + n1;
                uint32_t r[32];
                const uint32_t taddr = tmem + ((32u * (warp & 3u)) << 16) + n0;
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
#pragma unroll
                for (uint32_t i = 0; i < 16; ++i) {
                    const uint32_t o = om ^ ojs[(n0 >> 1) + i];
                    const float re = __uint_as_float(r[2 * i]), im = __uint_as_float(r[2 * i + 1]);
                    if (last) *reinterpret_cast<float2*>(Ab + o) = make_float2(re, im);
                    else put_amp<PREC>(Ab, o, re, im);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
        }
        if (!ok) break;
        // 3. the output tile back to HBM
#pragma unroll
        for (uint32_t r = 0; r < NROUND; ++r)
            *reinterpret_cast<float4*>(psi + (base | gthr | s_gr[r])) =
                *reinterpret_cast<const float4*>(Ab + (tthr ^ s_tr[r]));
        __syncthreads();
    }

    // a failed run: wait (bounded) for the MMAs and the bulk copy this CTA issued before
    // its shared and tensor memory go away
    if (s_fail && tid == 0) {
        mma_commit(smem_u32(&bar_fin));
        for (uint32_t it = 0; it < kHWait && !mbar_test(smem_u32(&bar_fin), 0); ++it) {
        }
        for (uint32_t sl = 0; sl < 2; ++sl)
            if ((pendm >> sl) & 1u)
                for (uint32_t it = 0; it < kHWait && !mbar_test(smem_u32(&bar_b[sl]), ((sl ? nload1 : nload0) - 1) & 1u);
                     ++it) {
                }
        atomicExch(status, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(N));
}

template <int PREC, int KS>
cudaError_t launch_one(float2* psi, const HierStage* d_st, const HierStage& hst, const uint8_t* d_ublob,
                       int* d_status, cudaStream_t s) {
    const size_t smem = svh::hier_smem_bytes(hst);
    static bool cfg = false;
    if (!cfg) {
        cudaError_t e = cudaFuncSetAttribute(k_hier_stage<PREC, KS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             220 * 1024);
        if (e != cudaSuccess) return e;
        // the whole unified L1 / shared array as shared memory: several CTAs per SM
        e = cudaFuncSetAttribute(k_hier_stage<PREC, KS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        cfg = true;
    }
    if (smem > 220 * 1024) return cudaErrorInvalidConfiguration;
    // CTAs per SM from the SM's shared memory (each CTA: dynamic + static + the 1 KB the
    // driver reserves), registers and threads, capped by tensor memory (512 columns per
    // SM, N per CTA).  (The occupancy calculator answers 1 here once the kernel's dynamic
    // shared-memory limit is raised above what one launch uses.)
    static int smem_sm = 0, reserved = 0, static_smem = 0, regs = 0;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (!smem_sm) {
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, k_hier_stage<PREC, KS>);
        if (e != cudaSuccess) return e;
        static_smem = (int)fa.sharedSizeBytes;
        regs = std::max(1, fa.numRegs);
    }
    int per_sm = smem_sm / (int)(smem + (size_t)static_smem + (size_t)reserved);
    per_sm = std::min(per_sm, 65536 / (regs * kHT));
    per_sm = std::min(per_sm, 2048 / kHT);
    per_sm = std::max(1, std::min(per_sm, (int)(512 / (2u << KS))));
    if (const char* v = getenv("SVGB_HIER_CTAS")) per_sm = std::max(1, std::min(atoi(v), (int)(512 / (2u << KS))));
    if (getenv("SVGB_HIER_VERBOSE"))
        fprintf(stderr, "k_hier_stage<%d,%d>: smem %zu + %d static, CTAs per SM %d\n", PREC, KS, smem, static_smem, per_sm);
    const uint64_t ntiles = 1ull << hst.n_glob;
    const unsigned grid = (unsigned)std::min<uint64_t>(ntiles, (uint64_t)nsm * (uint64_t)per_sm);
    k_hier_stage<PREC, KS><<<grid, kHT, smem, s>>>(psi, d_st, d_ublob, d_status);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_hier_stage(int prec, void* psi, const HierStage* d_st, const HierStage& hst, const uint8_t* d_ublob,
                              int* d_status, cudaStream_t s) {
    if (hst.n_sub == 0 || hst.n_sub > (uint32_t)kHierMaxSub) return cudaErrorInvalidValue;
    if (prec == 2 && hst.k == 5) return launch_one<2, 5>((float2*)psi, d_st, hst, d_ublob, d_status, s);
    if (prec == 2 && hst.k == 6) return launch_one<2, 6>((float2*)psi, d_st, hst, d_ublob, d_status, s);
    if (prec == 1 && hst.k == 5) return launch_one<1, 5>((float2*)psi, d_st, hst, d_ublob, d_status, s);
    return cudaErrorInvalidValue;
}

}  // namespace svk
