// gemm_kernels.cu — a fused stage applied as a split-precision tensor-core GEMM,
// D (128 columns x N) = X (128 columns x K) * Ut^T, with X ~ Xhi + Xlo, Ut ~ Uhi + Ulo
// and D ~ Xhi Uhi + Xlo Uhi + Xhi Ulo accumulated in FP32 in tensor memory (TF32x3,
// Ootomo-Yokota style; BF16x3, Henry et al. style).
//
// sm_103a, one CTA of 512 threads per SM, persistent over tiles:
//  - B (the stage's fused unitary, pre-split and pre-swizzled by the host) is copied
//    into shared memory once per CTA when it fits (k = 6), else streamed per K chunk;
//  - A (the tile's state columns) is produced per K chunk by all threads: 8-byte
//    loads whose warps cover contiguous >= 128-byte runs, the hi / lo split, and
//    stores into a two-slot ring in the 128-byte-swizzled K-major layout; the loads
//    run two chunks ahead (a ring of three register sets);
//  - one thread issues the 3 x 4 tcgen05.mma of a chunk and commits them to the
//    slot's mbarrier (the slot is refilled once they complete) and, after a tile's
//    last chunk, to the accumulator's mbarrier;
//  - accumulators are double-buffered in tensor memory: a tile's epilogue
//    (tcgen05.ld, in-place stores) runs after the next tile's first chunk is issued.
// Every wait is bounded: on time-out the kernel raises the status flag, waits (bounded)
// for the MMAs it issued, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "gemm.h"

namespace svk {

namespace {

constexpr int kT = 512;
constexpr int kLogT = 9;
constexpr uint32_t kWaitLimit = 1u << 22;
constexpr uint32_t kOpBlock = 16384;     // one 128-row operand block of 128-byte rows
constexpr uint32_t kASlot = 2 * kOpBlock;

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
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t it = 0; it < kWaitLimit; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, q;\n\t}"
                     : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
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

// byte offset of amplitude jj of a chunk (its (re, im) pair) in row m of an A block:
// XOR-linear in the bits of jj and m, so a thread's part and a round's part combine
// with XOR
template <int PREC>
__device__ __forceinline__ uint32_t a_offset(uint32_t jj, uint32_t m) {
    const uint32_t rowo = (m >> 3) * 1024 + (m & 7) * 128;
    return PREC == 1 ? rowo + ((((jj >> 1) ^ m) & 7u) << 4) + ((jj & 1u) << 3)
                     : rowo + ((((jj >> 2) ^ m) & 7u) << 4) + ((jj & 3u) << 2);
}

template <int PREC>   // 1 = TF32x3, 2 = BF16x3
__global__ void __launch_bounds__(kT, 1)
    k_gemm_stage(float2* __restrict__ psi, const GemmStage* __restrict__ stp, const uint8_t* __restrict__ ublob,
                 int* __restrict__ status) {
    extern __shared__ unsigned char sm_raw[];
    __shared__ GemmStage s_st;
    __shared__ uint64_t s_ltab[128];                 // local index -> physical offset
    __shared__ uint64_t s_roff[32];                  // producer round -> physical offset
    __shared__ uint32_t s_rsoff[32];                 // producer round -> swizzled A offset part
    __shared__ __align__(8) uint64_t bar_mma[2], bar_acc[2], bar_fin;
    __shared__ uint32_t tmem_slot;
    static_assert(sizeof(GemmStage) % 4 == 0, "stage copy");

    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (uint32_t i = tid; i < sizeof(GemmStage) / 4; i += kT)
        reinterpret_cast<uint32_t*>(&s_st)[i] = reinterpret_cast<const uint32_t*>(stp)[i];
    __syncthreads();
    const GemmStage& st = s_st;
    const uint32_t N = st.N, nchunk = st.nchunk, cb = st.camp_bits, nvar = st.nvar;
    const uint32_t ncols = 1u << st.ncol_bits;
    const uint32_t namp = 1u << nvar;                 // amplitudes per chunk
    const uint32_t npair = namp >> 1;                 // 16-byte pairs (physical bit 0 is var bit 0)
    const uint32_t rounds = npair > (uint32_t)kT ? npair / kT : 1u;
    const bool resident = st.resident != 0;
    const uint32_t bcb = st.b_chunk_bytes;

    // operand regions (1024-byte aligned for the swizzle pattern)
    const uint32_t sbase = (smem_u32(sm_raw) + 1023u) & ~1023u;
    unsigned char* gbase = sm_raw + (sbase - smem_u32(sm_raw));
    auto a_slot = [&](uint32_t s) -> uint32_t {
        return resident ? sbase + nchunk * bcb + s * kASlot : sbase + s * (kASlot + bcb);
    };
    auto b_chunk = [&](uint32_t c, uint32_t s) -> uint32_t {
        return resident ? sbase + c * bcb : sbase + s * (kASlot + bcb) + kASlot;
    };

    // tables: local index -> physical bits; producer mapping: a thread loads amplitude
    // pairs (var bit 0 is always physical bit 0, so a pair is 16 contiguous bytes); var
    // bit v >= 1 of pair tp = tid + 512 r comes from tid bit v - 1 (v <= 9) or r bit v - 10
    for (uint32_t i = tid; i < (1u << st.keff); i += kT) {
        uint64_t p = 0;
        for (uint32_t j = 0; j < st.keff; ++j)
            if ((i >> j) & 1) p |= 1ull << st.local_pos[j];
        s_ltab[i] = p;
    }
    uint64_t p_tid = 0;
    uint32_t jm_tid = 0;
    for (uint32_t v = 1; v < nvar && v <= (uint32_t)kLogT; ++v)
        if ((tid >> (v - 1)) & 1) {
            p_tid |= 1ull << st.var_pos[v];
            const uint32_t r = st.var_role[v];
            jm_tid |= 1u << r;   // role j < 8: amplitude bit j; role 8 + c: column bit c (bit 8 + c)
        }
    if (tid < rounds) {
        uint64_t p = 0;
        uint32_t jm = 0;
        for (uint32_t v = kLogT + 1; v < nvar; ++v)
            if ((tid >> (v - kLogT - 1)) & 1) {
                p |= 1ull << st.var_pos[v];
                const uint32_t r = st.var_role[v];
                jm |= 1u << r;
            }
        s_roff[tid] = p;
        s_rsoff[tid] = a_offset<PREC>(jm & 0xFFu, jm >> 8);
    }
    const uint32_t soff_tid = a_offset<PREC>(jm_tid & 0xFFu, jm_tid >> 8);
    const uint32_t jm_b0 = 1u << st.var_role[0];                  // the pair's second amplitude
    const uint32_t soff_b0 = a_offset<PREC>(jm_b0 & 0xFFu, jm_b0 >> 8);
    // epilogue: this thread's column (TMEM lane) and the quarter of N its warp reads
    const uint32_t m_ep = 32u * (warp & 3u) + lane;
    uint64_t cpart = 0;
    for (uint32_t c = 0; c < st.ncol_bits; ++c)
        if ((m_ep >> c) & 1) cpart |= 1ull << st.col_pos[c];

    // rows beyond the columns (narrow states only) stay zero in both A slots
    if (ncols < 128)
        for (uint32_t s = 0; s < 2; ++s)
            for (uint32_t o = tid * 16; o < kASlot; o += kT * 16) {
                const uint32_t row = (o % kOpBlock) / 128 % 8 + (o % kOpBlock) / 1024 * 8;
                if (row >= ncols) *reinterpret_cast<uint4*>(gbase + (a_slot(s) - sbase) + o) = make_uint4(0, 0, 0, 0);
            }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_mma[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_acc[i])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_fin)));
    }
    const uint32_t tcols = 2 * N;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (resident) {
        const uint8_t* src = ublob + st.b_off;
        for (uint32_t o = tid * 16; o < nchunk * bcb; o += kT * 16) cp_async16g(sbase + o, src + o);
        asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t id = idesc(PREC == 1 ? 2u : 1u, N);
    bool myfail = false;   // this thread's bounded waits
    const uint64_t ntiles = 1ull << st.n_glob;

    // epilogue of the tile with global bits pbase from accumulator buffer ab
    auto epilogue = [&](uint64_t pbase, uint32_t ab, uint32_t parity) {
        const bool ok = mbar_wait(smem_u32(&bar_acc[ab]), parity);
        if (!ok) myfail = true;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t part = N >> 2;
        for (uint32_t n0 = (warp >> 2) * part; n0 < ((warp >> 2) + 1) * part; n0 += 32) {
            uint32_t r[32];
            const uint32_t taddr = tmem + ((32u * (warp & 3u)) << 16) + ab * N + n0;
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
            if (ok && m_ep < ncols) {
                const uint64_t pc = pbase | cpart;
                if (st.local_pos[0] == 0) {   // local index pairs (2i, 2i + 1) are adjacent: 16-byte stores
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        *reinterpret_cast<float4*>(psi + (pc | s_ltab[(n0 >> 1) + 2 * q])) =
                            make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                        __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        psi[pc | s_ltab[(n0 >> 1) + q]] = make_float2(__uint_as_float(r[2 * q]), __uint_as_float(r[2 * q + 1]));
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    };

    // This CTA's tiles are blockIdx.x + t * gridDim.x (tile bases advance by an addition
    // in the masked space of the global bits); its chunks are numbered g = t * nchunk + c.
    // Every per-amplitude offset is a per-thread constant.  Three register sets form a
    // ring: while chunk g is split, stored and multiplied, chunks g + 1 and g + 2 are in
    // flight (their loads were issued one and two steps earlier).
    constexpr int RMAX = PREC == 1 ? 2 : 4;   // amplitude pairs per thread and chunk
    const uint64_t my_tiles = (uint64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const uint64_t total = my_tiles * nchunk;
    uint64_t gmask = 0, pstep = 0, base = 0;
    for (uint32_t i = 0; i < st.n_glob; ++i) {
        const uint64_t b = 1ull << st.glob_pos[i];
        gmask |= b;
        if ((gridDim.x >> i) & 1) pstep |= b;
        if ((blockIdx.x >> i) & 1) base |= b;
    }
    uint32_t vmask = 0;
#pragma unroll
    for (int r = 0; r < RMAX; ++r)
        if ((uint32_t)r < rounds && tid + (uint32_t)r * kT < npair) vmask |= 1u << r;
    auto load_chunk = [&](uint64_t cb0, float4 (&v)[RMAX]) {
        const uint64_t b = cb0 | p_tid;
#pragma unroll
        for (int r = 0; r < RMAX; ++r)
            if ((vmask >> r) & 1) v[r] = *reinterpret_cast<const float4*>(psi + (b | s_roff[r]));
    };
    auto next_tile = [&](uint64_t b) -> uint64_t { return ((b | ~gmask) + pstep) & gmask; };
    float4 va[RMAX], vb[RMAX], vc3[RMAX];
    // lookahead position: the chunk two steps ahead of the current one
    uint32_t cl = 0;
    uint64_t bl = base;
    auto advance_look = [&]() {
        if (++cl == nchunk) {
            cl = 0;
            bl = next_tile(bl);
        }
    };
    if (total) load_chunk(bl | s_ltab[cl << cb], va);
    advance_look();
    if (total > 1) load_chunk(bl | s_ltab[cl << cb], vb);
    advance_look();
    bool failed = false;   // uniform (from __syncthreads_or)
    uint64_t prev_base = 0, t = 0, g = 0;
    uint32_t c = 0;
    // One chunk step: load chunk g + 2 into vl, split / store chunk g from vc, issue its
    // MMAs, then advance (g, t, c, base).  Returns false when a bounded wait gave up
    // (uniformly across the CTA).
    auto step = [&](float4 (&vc)[RMAX], float4 (&vl)[RMAX]) -> bool {
        const uint32_t slot = (uint32_t)(g & 1u), ab = (uint32_t)(t & 1u);
        uint32_t cn = c + 1;
        uint64_t bn = base;
        if (cn == nchunk) {
            cn = 0;
            bn = next_tile(base);
        }
        if (g + 2 < total) load_chunk(bl | s_ltab[cl << cb], vl);
        advance_look();
        if (g >= 2 && !mbar_wait(smem_u32(&bar_mma[slot]), (uint32_t)((g - 2) >> 1) & 1u)) myfail = true;
        if (!resident) {
            const uint8_t* src = ublob + st.b_off + (size_t)c * bcb;
            const uint32_t dst = b_chunk(c, slot);
            for (uint32_t o = tid * 16; o < bcb; o += kT * 16) cp_async16g(dst + o, src + o);
            asm volatile("cp.async.commit_group;\n" ::: "memory");
        }
        // A chunk: split and store (swizzled K-major, rows = columns)
        unsigned char* aH = gbase + (a_slot(slot) - sbase);
        unsigned char* aL = aH + kOpBlock;
#pragma unroll
        for (int r = 0; r < RMAX; ++r) {
            if (!((vmask >> r) & 1)) continue;
            const uint32_t so = soff_tid ^ s_rsoff[r];
#pragma unroll
            for (int h = 0; h < 2; ++h) {   // the pair's two amplitudes
                const float re = h ? vc[r].z : vc[r].x, im = h ? vc[r].w : vc[r].y;
                const uint32_t o2 = h ? so ^ soff_b0 : so;
                if (PREC == 1) {
                    const float hr = rn_tf32(re), hi_ = rn_tf32(im);
                    *reinterpret_cast<float2*>(aH + o2) = make_float2(hr, hi_);
                    *reinterpret_cast<float2*>(aL + o2) = make_float2(rn_tf32(re - hr), rn_tf32(im - hi_));
                } else {
                    const __nv_bfloat162 h2 = __floats2bfloat162_rn(re, im);
                    const float2 hf = __bfloat1622float2(h2);
                    const __nv_bfloat162 l2 = __floats2bfloat162_rn(re - hf.x, im - hf.y);
                    *reinterpret_cast<__nv_bfloat162*>(aH + o2) = h2;
                    *reinterpret_cast<__nv_bfloat162*>(aL + o2) = l2;
                }
            }
        }
        if (!resident) asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (__syncthreads_or(myfail ? 1 : 0)) return false;   // a uniform verdict
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t A0 = a_slot(slot), B0 = b_chunk(c, slot);
            const uint32_t d = tmem + ab * N;
#pragma unroll
            for (int p = 0; p < 3; ++p) {   // hi*hi, lo*hi, hi*lo
                const uint32_t As = A0 + (p == 1 ? kOpBlock : 0u);
                const uint32_t Bs = B0 + (p == 2 ? N * 128u : 0u);
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    const uint64_t da = mdesc(As + 32u * s), db = mdesc(Bs + 32u * s);
                    const uint32_t acc = (c > 0 || p > 0 || s > 0) ? 1u : 0u;
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
            mma_commit(smem_u32(&bar_mma[slot]));
            if (c + 1 == nchunk) mma_commit(smem_u32(&bar_acc[ab]));
        }
        if (c == 0 && t > 0) epilogue(prev_base, ab ^ 1u, (uint32_t)((t - 1) >> 1) & 1u);
        // advance
        ++g;
        if (cn == 0) {
            prev_base = base;
            ++t;
        }
        c = cn;
        base = bn;
        return true;
    };
    // three steps per iteration so the register sets rotate without copies
    while (g < total && !failed) {
        if (!step(va, vc3)) failed = true;
        else if (g < total && !step(vb, va)) failed = true;
        else if (g < total && !step(vc3, vb)) failed = true;
    }
    __syncthreads();
    if (!failed && my_tiles > 0)   // the last tile (prev_base after the final advance)
        epilogue(prev_base, (uint32_t)((my_tiles - 1) & 1u), (uint32_t)((my_tiles - 1) >> 1) & 1u);
    failed = __syncthreads_or(myfail ? 1 : 0) != 0;
    if (failed && tid == 0) {
        // wait (bounded) for every MMA this CTA issued before freeing tensor memory
        mma_commit(smem_u32(&bar_fin));
        mbar_wait(smem_u32(&bar_fin), 0);
        atomicExch(status, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
}

}  // namespace

size_t gemm_smem_bytes(const GemmStage& st) {
    const size_t ops = st.resident ? (size_t)st.nchunk * st.b_chunk_bytes + 2 * kASlot
                                   : 2 * ((size_t)kASlot + st.b_chunk_bytes);
    return 1024 + ops;   // + alignment of the swizzled operand regions
}

cudaError_t launch_gemm_stage(int prec, void* psi, const GemmStage* d_stage, const GemmStage& hst,
                              const uint8_t* d_ublob, int* d_status, cudaStream_t s) {
    const size_t smem = gemm_smem_bytes(hst);
    constexpr int kMaxDyn = 200 * 1024;   // the kernel also holds ~1.8 KB of static shared memory
    if (smem > (size_t)kMaxDyn) return cudaErrorInvalidConfiguration;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t ntiles = 1ull << hst.n_glob;
    // one CTA per SM: it holds up to 512 tensor-memory columns
    const unsigned grid = (unsigned)std::min<uint64_t>(ntiles, (uint64_t)nsm);
    if (prec == 1) {
        static bool cfg = false;
        if (!cfg) {
            cudaError_t e = cudaFuncSetAttribute(k_gemm_stage<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn);
            if (e != cudaSuccess) return e;
            cfg = true;
        }
        k_gemm_stage<1><<<grid, kT, smem, s>>>((float2*)psi, d_stage, d_ublob, d_status);
    } else {
        static bool cfg = false;
        if (!cfg) {
            cudaError_t e = cudaFuncSetAttribute(k_gemm_stage<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn);
            if (e != cudaSuccess) return e;
            cfg = true;
        }
        k_gemm_stage<2><<<grid, kT, smem, s>>>((float2*)psi, d_stage, d_ublob, d_status);
    }
    return cudaGetLastError();
}

}  // namespace svk
