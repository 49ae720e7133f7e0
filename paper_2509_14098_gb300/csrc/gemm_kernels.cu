// gemm_kernels.cu — a fused stage applied as a split-precision tensor-core GEMM,
// D (128 columns x N) = X (128 columns x K) * Ut^T, with X ~ Xhi + Xlo, Ut ~ Uhi + Ulo
// and D ~ Xhi Uhi + Xlo Uhi + Xhi Ulo accumulated in FP32 in tensor memory (TF32x3,
// Ootomo-Yokota style; BF16x3, Henry et al. style).
//
// sm_103a, one CTA per SM, persistent over tiles, warp-specialised (the roles hand off
// through mbarriers; no CTA-wide barrier in the main loop):
//  - 16 producer warps gather each K chunk of a tile's state columns (16-byte amplitude
//    pairs, lane bits chosen per stage for conflict-free operand stores, the next chunk's
//    loads in flight and the chunk two beyond it prefetched into L2 unless a BF16x3 stage
//    streams B), split them into hi / lo halves and store them into a ring of operand slots in
//    the 128-byte-swizzled K-major layout (A operand, M = 128 columns); when B (the
//    stage's fused unitary, pre-split and pre-swizzled by the host) does not stay in
//    shared memory for the whole launch (k = 7), one of them starts a bulk copy of its K
//    chunk that completes on the slot's own transaction barrier;
//  - one thread issues the 3 x 4 tcgen05.mma of a chunk and commits them to the slot's
//    "empty" barrier, and after a tile's last chunk to the accumulator's "full" barrier;
//  - 4 epilogue warps (one per 32-lane quarter of tensor memory) read a finished
//    accumulator with tcgen05.ld and store the columns in place; accumulators are
//    double-buffered in tensor memory.
// Every wait is bounded: on time-out the kernel raises the status flag, waits (bounded)
// for the MMAs it issued, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "gemm.h"
#include "tc_util.cuh"

namespace svk {

namespace {

constexpr int kP = 512;          // producer threads (warps 0..15)
constexpr int kLogP = 9;
constexpr int kEpiWarp0 = 16;    // epilogue warps 16..19 (tensor-memory lane quarter = warp & 3)
constexpr int kMmaWarp = 20;     // MMA issue (lane 0), tensor-memory allocation
constexpr int kT = 21 * 32;
constexpr uint32_t kWaitLimit = 1u << 22;
constexpr uint32_t kOpBlock = 16384;     // one 128-row operand block of 128-byte rows
constexpr uint32_t kASlot = 2 * kOpBlock;

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
    __shared__ __align__(8) uint64_t bar_full[3], bar_empty[3], bar_accf[2], bar_acce[2], bar_fin, bar_bfull[3];
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_fail;
    static_assert(sizeof(GemmStage) % 4 == 0, "stage copy");

    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (uint32_t i = tid; i < sizeof(GemmStage) / 4; i += kT)
        reinterpret_cast<uint32_t*>(&s_st)[i] = reinterpret_cast<const uint32_t*>(stp)[i];
    if (tid == 0) s_fail = 0;
    __syncthreads();
    const GemmStage& st = s_st;
    const uint32_t N = st.N, nchunk = st.nchunk, cb = st.camp_bits, nvar = st.nvar, NS = st.nslot;
    const uint32_t ncols = 1u << st.ncol_bits;
    const uint32_t namp = 1u << nvar;                 // amplitudes per chunk
    const uint32_t npair = namp >> 1;                 // 16-byte pairs (physical bit 0 is var bit 0)
    const uint32_t rounds = npair > (uint32_t)kP ? npair / kP : 1u;
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

    // tables: local index -> physical bits; producer mapping: a producer loads amplitude
    // pairs (var bit 0 is always physical bit 0, so a pair is 16 contiguous bytes); producer
    // bit i of pair tp = tid + kP r (tid bits, then round bits) is var bit pperm[i]
    for (uint32_t i = tid; i < (1u << st.keff); i += kT) {
        uint64_t p = 0;
        for (uint32_t j = 0; j < st.keff; ++j)
            if ((i >> j) & 1) p |= 1ull << st.local_pos[j];
        s_ltab[i] = p;
    }
    if (tid < rounds) {
        uint64_t p = 0;
        uint32_t jm = 0;
        for (uint32_t i = kLogP; i + 1 < nvar; ++i)
            if ((tid >> (i - kLogP)) & 1) {
                const uint32_t v = st.pperm[i];
                p |= 1ull << st.var_pos[v];
                jm |= 1u << st.var_role[v];
            }
        s_roff[tid] = p;
        s_rsoff[tid] = a_offset<PREC>(jm & 0xFFu, jm >> 8);
    }
    // rows beyond the columns (narrow states only) stay zero in every A slot
    if (ncols < 128)
        for (uint32_t s = 0; s < NS; ++s)
            for (uint32_t o = tid * 16; o < kASlot; o += kT * 16) {
                const uint32_t row = (o % kOpBlock) / 128 % 8 + (o % kOpBlock) / 1024 * 8;
                if (row >= ncols) *reinterpret_cast<uint4*>(gbase + (a_slot(s) - sbase) + o) = make_uint4(0, 0, 0, 0);
            }
    if (tid == 0) {
        for (int i = 0; i < 3; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_full[i])), "r"(kP / 32));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_empty[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_bfull[i])));
        }
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_accf[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_u32(&bar_acce[i])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_fin)));
    }
    const uint32_t tcols = 2 * N;
    if (warp == kMmaWarp) {
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
    const uint64_t ntiles = 1ull << st.n_glob;
    const uint64_t my_tiles = (uint64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const uint64_t total = my_tiles * nchunk;
    uint64_t gmask = 0, pstep = 0, base0 = 0;
    for (uint32_t i = 0; i < st.n_glob; ++i) {
        const uint64_t b = 1ull << st.glob_pos[i];
        gmask |= b;
        if ((gridDim.x >> i) & 1) pstep |= b;
        if ((blockIdx.x >> i) & 1) base0 |= b;
    }
    auto next_tile = [&](uint64_t b) -> uint64_t { return ((b | ~gmask) + pstep) & gmask; };
    // bounded wait that also gives up once another role has failed
    auto wait = [&](const uint64_t& bar, uint32_t parity) -> bool {
        const uint32_t a = smem_u32(&bar);
        for (uint32_t it = 0; it < kWaitLimit; ++it) {
            uint32_t done;
            asm volatile("{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
                         "selp.u32 %0, 1, 0, q;\n\t}"
                         : "=r"(done) : "r"(a), "r"(parity) : "memory");
            if (done) return true;
            if (s_fail) return false;
        }
        s_fail = 1;
        return false;
    };

    if (warp < kP / 32) {
        // ------------------------------------------------------------ producers
        constexpr int RMAX = PREC == 1 ? 2 : 4;   // amplitude pairs per thread and chunk
        uint64_t p_tid = 0;
        uint32_t jm_tid = 0;
        for (uint32_t i = 0; i + 1 < nvar && i < (uint32_t)kLogP; ++i)
            if ((tid >> i) & 1) {
                const uint32_t v = st.pperm[i];
                p_tid |= 1ull << st.var_pos[v];
                jm_tid |= 1u << st.var_role[v];   // role j < 8: amplitude bit j; 8 + c: column bit c
            }
        const uint32_t soff_tid = a_offset<PREC>(jm_tid & 0xFFu, jm_tid >> 8);
        const bool pair_amp = st.var_role[0] == 0;                    // pair = amplitudes 2i, 2i + 1 of one row
        const uint32_t jm_b0 = 1u << st.var_role[0];                  // the pair's second amplitude
        const uint32_t soff_b0 = a_offset<PREC>(jm_b0 & 0xFFu, jm_b0 >> 8);
        uint32_t vmask = 0;
#pragma unroll
        for (int r = 0; r < RMAX; ++r)
            if ((uint32_t)r < rounds && tid + (uint32_t)r * kP < npair) vmask |= 1u << r;
        auto load_chunk = [&](uint64_t cb0, float4 (&v)[RMAX]) {
            const uint64_t b = cb0 | p_tid;
#pragma unroll
            for (int r = 0; r < RMAX; ++r)
                if ((vmask >> r) & 1) v[r] = *reinterpret_cast<const float4*>(psi + (b | s_roff[r]));
        };
        // lookahead position: the chunk after the current one
        uint32_t cl = 0;
        uint64_t bl = base0;
        auto advance_look = [&]() {
            if (++cl == nchunk) {
                cl = 0;
                bl = next_tile(bl);
            }
        };
        // L2 prefetch two chunks beyond the register lookahead (the loads then hit L2),
        // except for BF16x3 stages whose B streams through L2 every chunk (measured slower)
        uint32_t cpf = cl;
        uint64_t bpf = bl;
        auto advance_pf = [&]() {
            if (++cpf == nchunk) {
                cpf = 0;
                bpf = next_tile(bpf);
            }
        };
        const uint32_t pfd = (resident || PREC == 1) ? 2u : 0u;
        for (uint32_t i = 0; i < pfd + 1; ++i) advance_pf();
        auto prefetch_chunk = [&]() {
            const uint64_t b = bpf | s_ltab[cpf << cb] | p_tid;
#pragma unroll
            for (int r = 0; r < RMAX; ++r)
                if ((vmask >> r) & 1) asm volatile("prefetch.global.L2 [%0];" ::"l"(psi + (b | s_roff[r])));
        };
        uint64_t nbulk = 0;   // B bulk copies issued (thread 0)
        float4 va[RMAX], vb[RMAX];
        if (total) load_chunk(bl | s_ltab[cl << cb], va);
        advance_look();
        uint64_t g = 0;
        uint32_t c = 0;
        auto step = [&](float4 (&vc)[RMAX], float4 (&vl)[RMAX]) -> bool {
            const uint32_t slot = (uint32_t)(g % NS), use = (uint32_t)(g / NS);
            if (g + 1 < total) load_chunk(bl | s_ltab[cl << cb], vl);
            advance_look();
            if (pfd && g + 1 + pfd < total) prefetch_chunk();
            advance_pf();
            if (g >= NS && !wait(bar_empty[slot], (use - 1) & 1u)) return false;
            if (!resident && tid == 0) {   // B chunk: one bulk copy, completing on bar_bfull[slot]
                const uint8_t* src = ublob + st.b_off + (size_t)c * bcb;
                const uint32_t bar = smem_u32(&bar_bfull[slot]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bcb) : "memory");
                asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                             ::"r"(b_chunk(c, slot)), "l"(src), "r"(bcb), "r"(bar) : "memory");
                ++nbulk;
            }
            unsigned char* aH = gbase + (a_slot(slot) - sbase);
            unsigned char* aL = aH + kOpBlock;
#pragma unroll
            for (int r = 0; r < RMAX; ++r) {
                if (!((vmask >> r) & 1)) continue;
                const uint32_t so = soff_tid ^ s_rsoff[r];
                if (pair_amp) {   // the pair's amplitudes are adjacent in the operand row: one store each for hi, lo
                    if (PREC == 1) {
                        const float4 v = vc[r];
                        const float4 hv = make_float4(rn_tf32(v.x), rn_tf32(v.y), rn_tf32(v.z), rn_tf32(v.w));
                        *reinterpret_cast<float4*>(aH + so) = hv;
                        *reinterpret_cast<float4*>(aL + so) = make_float4(rn_tf32(v.x - hv.x), rn_tf32(v.y - hv.y),
                                                                          rn_tf32(v.z - hv.z), rn_tf32(v.w - hv.w));
                    } else {
                        const __nv_bfloat162 h0 = __floats2bfloat162_rn(vc[r].x, vc[r].y);
                        const __nv_bfloat162 h1 = __floats2bfloat162_rn(vc[r].z, vc[r].w);
                        const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
                        const __nv_bfloat162 l0 = __floats2bfloat162_rn(vc[r].x - f0.x, vc[r].y - f0.y);
                        const __nv_bfloat162 l1 = __floats2bfloat162_rn(vc[r].z - f1.x, vc[r].w - f1.y);
                        uint2 hw, lw;
                        memcpy(&hw.x, &h0, 4);
                        memcpy(&hw.y, &h1, 4);
                        memcpy(&lw.x, &l0, 4);
                        memcpy(&lw.y, &l1, 4);
                        *reinterpret_cast<uint2*>(aH + so) = hw;
                        *reinterpret_cast<uint2*>(aL + so) = lw;
                    }
                    continue;
                }
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
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the tensor core
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar_full[slot])) : "memory");
            ++g;
            if (++c == nchunk) c = 0;
            return true;
        };
        while (g < total) {
            if (!step(va, vb)) break;
            if (g < total && !step(vb, va)) break;
        }
        // bulk copies still in flight (a failed run): wait, bounded, for the last one of
        // each slot before the CTA can exit
        if (tid == 0)
            for (uint64_t gg = nbulk > NS ? nbulk - NS : 0; gg < nbulk; ++gg) {
                const uint32_t a = smem_u32(&bar_bfull[gg % NS]), par = (uint32_t)(gg / NS) & 1u;
                uint32_t done = 0;
                for (uint32_t it = 0; it < kWaitLimit && !done; ++it)
                    asm volatile("{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
                                 "selp.u32 %0, 1, 0, q;\n\t}"
                                 : "=r"(done) : "r"(a), "r"(par) : "memory");
                if (!done) s_fail = 1;
            }
    } else if (warp < kEpiWarp0 + 4) {
        // ------------------------------------------------------------ epilogue
        const uint32_t q = warp & 3u, m = 32u * q + lane;
        uint64_t cpart = 0;
        for (uint32_t cc = 0; cc < st.ncol_bits; ++cc)
            if ((m >> cc) & 1) cpart |= 1ull << st.col_pos[cc];
        uint64_t base = base0;
        for (uint64_t tl = 0; tl < my_tiles; ++tl, base = next_tile(base)) {
            const uint32_t ab = (uint32_t)(tl & 1u);
            const bool ok = wait(bar_accf[ab], (uint32_t)(tl >> 1) & 1u);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t pc = base | cpart;
            for (uint32_t n0 = 0; n0 < N; n0 += 32) {
                uint32_t r[32];
                const uint32_t taddr = tmem + ((32u * q) << 16) + ab * N + n0;
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
                if (ok && m < ncols) {
                    if (st.local_pos[0] == 0) {   // local index pairs (2i, 2i + 1) are adjacent: 16-byte stores
#pragma unroll
                        for (int k = 0; k < 8; ++k)
                            *reinterpret_cast<float4*>(psi + (pc | s_ltab[(n0 >> 1) + 2 * k])) =
                                make_float4(__uint_as_float(r[4 * k]), __uint_as_float(r[4 * k + 1]),
                                            __uint_as_float(r[4 * k + 2]), __uint_as_float(r[4 * k + 3]));
                    } else {
#pragma unroll
                        for (int k = 0; k < 16; ++k)
                            psi[pc | s_ltab[(n0 >> 1) + k]] = make_float2(__uint_as_float(r[2 * k]), __uint_as_float(r[2 * k + 1]));
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar_acce[ab])) : "memory");
            if (!ok) break;
        }
    } else if (lane == 0) {
        // ------------------------------------------------------------ MMA issue
        const uint32_t id = idesc(PREC == 1 ? 2u : 1u, N);
        uint64_t g = 0;
        for (uint64_t tl = 0; tl < my_tiles && !s_fail; ++tl) {
            const uint32_t ab = (uint32_t)(tl & 1u);
            if (tl >= 2 && !wait(bar_acce[ab], (uint32_t)((tl >> 1) - 1) & 1u)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t d = tmem + ab * N;
            bool ok = true;
            for (uint32_t c = 0; c < nchunk; ++c, ++g) {
                const uint32_t slot = (uint32_t)(g % NS);
                if (!wait(bar_full[slot], (uint32_t)(g / NS) & 1u) ||
                    (!resident && !wait(bar_bfull[slot], (uint32_t)(g / NS) & 1u))) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t A0 = a_slot(slot), B0 = b_chunk(c, slot);
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
                mma_commit(smem_u32(&bar_empty[slot]));
                if (c + 1 == nchunk) mma_commit(smem_u32(&bar_accf[ab]));
            }
            if (!ok) break;
        }
    }
    __syncthreads();
    if (s_fail && tid == kMmaWarp * 32) {
        // wait (bounded) for every MMA this CTA issued before freeing tensor memory
        mma_commit(smem_u32(&bar_fin));
        uint32_t done = 0;
        for (uint32_t it = 0; it < kWaitLimit && !done; ++it)
            asm volatile("{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], 0;\n\t"
                         "selp.u32 %0, 1, 0, q;\n\t}"
                         : "=r"(done) : "r"(smem_u32(&bar_fin)) : "memory");
        atomicExch(status, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == kMmaWarp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
}

}  // namespace

size_t gemm_smem_bytes(const GemmStage& st) {
    const size_t ops = st.resident ? (size_t)st.nchunk * st.b_chunk_bytes + (size_t)st.nslot * kASlot
                                   : (size_t)st.nslot * ((size_t)kASlot + st.b_chunk_bytes);
    return 1024 + ops;   // + alignment of the swizzled operand regions
}

cudaError_t launch_gemm_stage(int prec, void* psi, const GemmStage* d_stage, const GemmStage& hst,
                              const uint8_t* d_ublob, int* d_status, cudaStream_t s) {
    const size_t smem = gemm_smem_bytes(hst);
    constexpr int kMaxDyn = 225 * 1024;   // the kernel also holds ~1.8 KB of static shared memory
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
