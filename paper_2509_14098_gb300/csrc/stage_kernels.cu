// stage_kernels.cu — one HBM sweep per partition (Sec. 4.3, single-device case:
// pack a tile from global memory into shared memory, compute, unpack).
//
// Forward: each CTA owns one tile, i.e. one assignment of the stage's global bits.
// It stages the 2^T amplitudes whose local bits vary into shared memory with
// 16-byte cp.async copies (the tile always contains the lowest physical bits, so
// every HBM access is a contiguous run of >= 128 B), then walks the stage's register
// groups: each thread pulls 2^R amplitudes into registers, applies the group's ops,
// and writes them back; finally the tile is written back in place.
//
// Backward (adjoint): the same sweep over psi and lambda together, with the stage's
// gates conjugate-transposed in reverse order, and gradient ops accumulating
// Im <lambda|G|psi> per parametric rotation into per-tile partial sums (FP32 inside a
// warp, FP64 across warps and tiles, in a fixed order).
#include <algorithm>

#include "kdev.cuh"
#include "kernels.h"

namespace svk {

// per-group thread-offset table in shared memory only while it stays small
__host__ __device__ __forceinline__ bool group_table_fits(uint32_t n_groups, uint32_t nthr) {
    return (size_t)n_groups * nthr * 12 <= 24 * 1024;
}

// Persistent: CTA b handles tiles b, b + gridDim.x, ... and prefetches the next tile
// into the second buffer (cp.async) while it computes the current one.  Everything
// that does not depend on the tile (chunk offsets, each group's thread offsets) is
// computed once; the tile base advances by an addition in the masked bit space of
// the global bits: base(t + G) = ((base(t) | ~gmask) + pdep(G)) & gmask.
template <typename Real, int R, int MAXT>
__global__ void __launch_bounds__(MAXT, (MAXT >= 512 ? 1 : 2)) k_stage_fwd(typename CT<Real>::C* __restrict__ psi,
                                                    const Stage* __restrict__ stp,
                                                    const Group* __restrict__ groups,
                                                    const DevOp<Real>* __restrict__ gops,
                                                    const DevTerm<Real>* __restrict__ terms,
                                                    const PhaseSlot<Real>* __restrict__ slots) {
    using C = typename CT<Real>::C;
    constexpr int APC = 16 / (int)sizeof(C);
    constexpr int LA = APC == 2 ? 1 : 0;
    constexpr int NCH = (1 << R) / APC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Stage& st = *stp;
    const int T = (int)st.T;
    const int TR = T - R;
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
    const uint32_t ng = st.n_groups;
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + (1u << T);
    Group* sgr = reinterpret_cast<Group*>(buf1 + (1u << T));
    DevOp<Real>* sops = reinterpret_cast<DevOp<Real>*>(sgr + ng);
    PhaseSlot<Real>* ssl = reinterpret_cast<PhaseSlot<Real>*>(sops + st.n_ops);
    typename AngT<Real>::type* sang = reinterpret_cast<typename AngT<Real>::type*>(ssl + st.n_phase);
    const bool gtab = group_table_fits(st.n_groups, nthr);
    const uint32_t ngt = gtab ? ng : 0;
    uint64_t* gfix = reinterpret_cast<uint64_t*>(
        (reinterpret_cast<uintptr_t>(sang + st.n_phase) + 15) & ~(uintptr_t)15);   // [ngt][nthr]
    uint64_t* chp = gfix + (size_t)ngt * nthr;                                      // [NCH]
    uint32_t* gsoff = reinterpret_cast<uint32_t*>(chp + NCH);                         // [ngt][nthr]
    uint32_t* chs = gsoff + (size_t)ngt * nthr;                                       // [NCH]
    const uint64_t ntiles = 1ull << st.n_glob;

    uint64_t t = blockIdx.x;
    if (t >= ntiles) return;
    // tile-independent offsets
    uint64_t gmask = 0, pstep = 0, base = 0;
    for (uint32_t i = 0; i < st.n_glob; ++i) {
        const uint64_t b = 1ull << st.glob_pos[i];
        gmask |= b;
        if ((gridDim.x >> i) & 1) pstep |= b;
        if ((t >> i) & 1) base |= b;
    }
    uint64_t ptid = 0;
    uint32_t stid = 0;
    for (int b = 0; b < TR; ++b)
        if ((tid >> b) & 1) {
            ptid ^= st.ptile[b + LA];
            stid ^= st.swbit[b + LA];
        }
    // first load (chunk offsets for i computed inline once; tables for later tiles)
#pragma unroll
    for (int i = 0; i < NCH; ++i) {
        uint64_t pi = 0;
        uint32_t si = 0;
#pragma unroll
        for (int b = 0; (1 << b) < NCH; ++b)
            if ((i >> b) & 1) {
                pi ^= st.ptile[TR + LA + b];
                si ^= st.swbit[TR + LA + b];
            }
        cp_async16(buf0 + (stid ^ si), psi + (base | (ptid ^ pi)));
        if (tid == 0) {
            chp[i] = pi;
            chs[i] = si;
        }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    stage_prologue<Real>(sgr, sops, ssl, st, groups, gops, slots, tid, nthr);
    for (uint32_t g = 0; g < ngt; ++g) {
        const Group& G = groups[st.group_off + g];
        uint64_t f = 0;
        uint32_t so = 0;
        for (int i = 0; i < TR; ++i)
            if ((tid >> i) & 1) {
                f ^= G.pthr[i];
                so ^= G.sthr[i];
            }
        gfix[g * nthr + tid] = f;
        gsoff[g * nthr + tid] = so;
    }
    __syncthreads();

    OpCtx<Real> x;
    x.slots = ssl;
    x.ang = sang;
    x.tid = tid;
    x.TR = TR;
    x.terms = terms;
    for (uint32_t it = 0; t < ntiles; t += gridDim.x, ++it) {
        C* cur = (it & 1) ? buf1 : buf0;
        C* nxt = (it & 1) ? buf0 : buf1;
        const uint64_t tn = t + gridDim.x;
        const uint64_t bn = ((base | ~gmask) + pstep) & gmask;
        if (tn < ntiles) {
#pragma unroll
            for (int i = 0; i < NCH; ++i) cp_async16(nxt + (stid ^ chs[i]), psi + (bn | (ptid ^ chp[i])));
            asm volatile("cp.async.commit_group;\ncp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        if (st.n_phase) tile_angles<Real>(sang, slots, terms, st, base, tid, nthr);
        __syncthreads();
        for (uint32_t g = 0; g < ng; ++g) {
            const Group& G = sgr[g];
            uint64_t f = 0;
            uint32_t soff = 0;
            if (gtab) {
                f = gfix[g * nthr + tid];
                soff = gsoff[g * nthr + tid];
            } else {
                for (int i = 0; i < TR; ++i)
                    if ((tid >> i) & 1) {
                        f ^= G.pthr[i];
                        soff ^= G.sthr[i];
                    }
            }
            x.fix = base ^ f;
            uint32_t sr[R];
#pragma unroll
            for (int j = 0; j < R; ++j) sr[j] = G.sreg[j];
            const bool pairs = G.pairs != 0;
            typename RegT<Real>::type a[1 << R];
            load_regs<typename RegT<Real>::type, C, R>(a, cur, soff, sr, pairs);
            const DevOp<Real>* op = sops + G.op_off;
            const uint32_t nops = G.n_ops;
            for (uint32_t oi = 0; oi < nops; ++oi) apply_op<Real, R>(a, load_op<Real>(op + oi), x);
            store_regs<typename RegT<Real>::type, C, R>(a, cur, soff, sr, pairs);
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < NCH; ++i) {
            const float4 v = *reinterpret_cast<const float4*>(cur + (stid ^ chs[i]));
            *reinterpret_cast<float4*>(psi + (base | (ptid ^ chp[i]))) = v;
        }
        base = bn;
        __syncthreads();   // cur is refilled by the prefetch of the next iteration but one
    }
}

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------
template <typename Real>
__device__ __forceinline__ Real im_conj_mul(typename CT<Real>::C l, typename CT<Real>::C p) {
    return l.x * p.y - l.y * p.x;   // Im(conj(l) p)
}
template <typename Real>
__device__ __forceinline__ Real re_conj_mul(typename CT<Real>::C l, typename CT<Real>::C p) {
    return l.x * p.x + l.y * p.y;   // Re(conj(l) p)
}

template <typename Real> __device__ __forceinline__ typename CT<Real>::C to_c(typename RegT<Real>::type v);
template <> __device__ __forceinline__ float2 to_c<float>(u64 v) { return unpack2(v); }
template <> __device__ __forceinline__ double2 to_c<double>(double2 v) { return v; }

template <typename Real, int R, int J>
__device__ __forceinline__ Real grad_pairs(const typename RegT<Real>::type (&ps)[1 << R],
                                           const typename RegT<Real>::type (&la)[1 << R], uint8_t type) {
    Real acc = 0;
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) {
        if (k & (1 << J)) continue;
        const int k1 = k | (1 << J);
        const auto l0 = to_c<Real>(la[k]), l1 = to_c<Real>(la[k1]);
        const auto p0 = to_c<Real>(ps[k]), p1 = to_c<Real>(ps[k1]);
        if (type == OP_GRAD_X) {
            acc += im_conj_mul<Real>(l0, p1) + im_conj_mul<Real>(l1, p0);
        } else if (type == OP_GRAD_Y) {
            // Y|0> = i|1>, Y|1> = -i|0>:  Im(conj(l0)(-i p1)) + Im(conj(l1)(i p0))
            acc += -re_conj_mul<Real>(l0, p1) + re_conj_mul<Real>(l1, p0);
        } else {
            acc += im_conj_mul<Real>(l0, p0) - im_conj_mul<Real>(l1, p1);
        }
    }
    return acc;
}

template <typename Real, int R, int MAXT>
__global__ void __launch_bounds__(MAXT, (MAXT >= 512 ? 1 : 2)) k_stage_bwd(typename CT<Real>::C* __restrict__ psi,
                                                   typename CT<Real>::C* __restrict__ lam,
                                                   const Stage* __restrict__ stp,
                                                   const Group* __restrict__ groups,
                                                   const DevOp<Real>* __restrict__ gops,
                                                   const DevTerm<Real>* __restrict__ terms,
                                                   const PhaseSlot<Real>* __restrict__ slots,
                                                   double* __restrict__ partial) {
    using C = typename CT<Real>::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Stage& st = *stp;
    const int T = (int)st.T;
    const int TR = T - R;
    C* tp = reinterpret_cast<C*>(smem_raw);
    C* tl = tp + (1u << T);
    Group* sgr = reinterpret_cast<Group*>(tl + (1u << T));
    DevOp<Real>* sops = reinterpret_cast<DevOp<Real>*>(sgr + st.n_groups);
    PhaseSlot<Real>* ssl = reinterpret_cast<PhaseSlot<Real>*>(sops + st.n_ops);
    typename AngT<Real>::type* sang = reinterpret_cast<typename AngT<Real>::type*>(ssl + st.n_phase);
    float* gsm = reinterpret_cast<float*>(sang + st.n_phase);
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
    const uint32_t nw = (nthr + 31) >> 5;
    const uint32_t warp = tid >> 5, lane = tid & 31;
    const uint32_t nslots = st.n_slots;
    const uint64_t base = tile_base(blockIdx.x, st.glob_pos);

    tile_load<C, R>(tp, psi, base, st.ptile, st.swbit, TR, tid);
    tile_load<C, R>(tl, lam, base, st.ptile, st.swbit, TR, tid);
    stage_prologue<Real>(sgr, sops, ssl, st, groups, gops, slots, tid, nthr);
    tile_angles<Real>(sang, slots, terms, st, base, tid, nthr);
    for (uint32_t i = tid; i < nslots * nw; i += nthr) gsm[i] = 0.f;
    cp_async_commit_wait_all();
    __syncthreads();

    OpCtx<Real> x;
    x.slots = ssl;
    x.ang = sang;
    x.tid = tid;
    x.TR = TR;
    x.terms = terms;
    const uint32_t wmask = nthr >= 32 ? 0xffffffffu : ((1u << nthr) - 1u);
    for (uint32_t g = 0; g < st.n_groups; ++g) {
        const Group& G = sgr[g];
        uint64_t fix = base;
        uint32_t soff = 0;
        for (int i = 0; i < TR; ++i)
            if ((tid >> i) & 1) {
                fix ^= G.pthr[i];
                soff ^= G.sthr[i];
            }
        x.fix = fix;
        uint32_t sr[R];
#pragma unroll
        for (int j = 0; j < R; ++j) sr[j] = G.sreg[j];
        const bool pairs = G.pairs != 0;
        typename RegT<Real>::type ps[1 << R], la[1 << R];
        load_regs<typename RegT<Real>::type, C, R>(ps, tp, soff, sr, pairs);
        load_regs<typename RegT<Real>::type, C, R>(la, tl, soff, sr, pairs);
        const DevOp<Real>* op = sops + G.op_off;
        for (uint32_t oi = 0; oi < G.n_ops; ++oi) {
            const DevOp<Real> o = load_op<Real>(op + oi);
            if (o.type >= OP_GRAD_X) {
                Real acc = 0;
                if (o.type == OP_GRAD_Z && o.u) {
                    // Z on a non-register bit: a sign per thread
#pragma unroll
                    for (int k = 0; k < (1 << R); ++k) acc += im_conj_mul<Real>(to_c<Real>(la[k]), to_c<Real>(ps[k]));
                    if ((fix & o.ctrl_fix) != 0) acc = -acc;
                } else {
                    SVK_SWITCH_J(o.j, R, (acc = grad_pairs<Real, R, J_>(ps, la, o.type)));
                }
                float v = (float)acc;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
                    if ((uint32_t)off < nthr) v += __shfl_xor_sync(wmask, v, off);
                if (lane == 0) gsm[o.slot * nw + warp] += v;
            } else {
                apply_op<Real, R>(ps, o, x);
                apply_op<Real, R>(la, o, x);
            }
        }
        store_regs<typename RegT<Real>::type, C, R>(ps, tp, soff, sr, pairs);
        store_regs<typename RegT<Real>::type, C, R>(la, tl, soff, sr, pairs);
        __syncthreads();
    }
    tile_store<C, R>(tp, psi, base, st.ptile, st.swbit, TR, tid);
    tile_store<C, R>(tl, lam, base, st.ptile, st.swbit, TR, tid);
    for (uint32_t s = tid; s < nslots; s += nthr) {
        double sum = 0.0;
        for (uint32_t w = 0; w < nw; ++w) sum += (double)gsm[s * nw + w];
        partial[(size_t)blockIdx.x * nslots + s] = sum;
    }
}

// ---------------------------------------------------------------------------
// launch wrappers
// ---------------------------------------------------------------------------
size_t stage_smem_bytes(int elem_bytes, const Stage& st, bool backward) {
    const size_t opb = elem_bytes == 8 ? sizeof(DevOp<float>) : sizeof(DevOp<double>);
    const size_t slb = elem_bytes == 8 ? sizeof(PhaseSlot<float>) : sizeof(PhaseSlot<double>);
    const uint32_t nthr = 1u << (st.T - st.R);
    // two tiles (forward: double buffer; backward: psi and lambda) + staged program
    size_t b = ((size_t)elem_bytes << st.T) * 2 + st.n_groups * sizeof(Group) + st.n_ops * opb +
               st.n_phase * (slb + (size_t)elem_bytes);
    if (!backward)   // per-group thread offsets (when they fit) and chunk tables (+ slack)
        b += 16 + (group_table_fits(st.n_groups, nthr) ? (size_t)st.n_groups * nthr * 12 : 0) + 32 * 12;
    if (backward) b += (size_t)st.n_slots * ((nthr + 31) / 32) * sizeof(float);
    return b;
}

template <typename Real, int R, int MAXT>
static cudaError_t launch_fwd_RT(const StageLaunch& L, const Stage& hst, cudaStream_t s) {
    using C = typename CT<Real>::C;
    const size_t smem = stage_smem_bytes(sizeof(C), hst, false);
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_stage_fwd<Real, R, MAXT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const uint64_t ntiles = 1ull << hst.n_glob;
    const int nthr = 1 << (hst.T - R);
    int per_sm = 0, dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stage_fwd<Real, R, MAXT>, nthr, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const uint64_t grid = std::min<uint64_t>(ntiles, (uint64_t)per_sm * (uint64_t)nsm);
    k_stage_fwd<Real, R, MAXT><<<(unsigned)grid, nthr, smem, s>>>(
        (C*)L.psi, L.stage, L.groups, (const DevOp<Real>*)L.ops, (const DevTerm<Real>*)L.terms,
        (const PhaseSlot<Real>*)L.slots);
    return cudaGetLastError();
}
// 256-thread bound (up to 255 registers) unless the tile needs 512 threads
template <typename Real, int R>
static cudaError_t launch_fwd_R(const StageLaunch& L, const Stage& hst, cudaStream_t s) {
    if ((hst.T - R) <= 8) return launch_fwd_RT<Real, R, 256>(L, hst, s);
    if ((hst.T - R) == 9) return launch_fwd_RT<Real, R, 512>(L, hst, s);
    return cudaErrorInvalidConfiguration;
}

cudaError_t launch_stage_fwd(int elem_bytes, const StageLaunch& L, const Stage& hst, cudaStream_t s) {
    if (elem_bytes == 8) {
        switch (hst.R) {
            case 1: return launch_fwd_R<float, 1>(L, hst, s);
            case 2: return launch_fwd_R<float, 2>(L, hst, s);
            case 3: return launch_fwd_R<float, 3>(L, hst, s);
            case 4: return launch_fwd_R<float, 4>(L, hst, s);
            case 5: return launch_fwd_R<float, 5>(L, hst, s);
        }
    } else {
        switch (hst.R) {
            case 1: return launch_fwd_R<double, 1>(L, hst, s);
            case 2: return launch_fwd_R<double, 2>(L, hst, s);
            case 3: return launch_fwd_R<double, 3>(L, hst, s);
            case 4: return launch_fwd_R<double, 4>(L, hst, s);
        }
    }
    return cudaErrorInvalidValue;
}

template <typename Real, int R, int MAXT>
static cudaError_t launch_bwd_RT(const StageLaunch& L, const Stage& hst, cudaStream_t s) {
    using C = typename CT<Real>::C;
    const size_t smem = stage_smem_bytes(sizeof(C), hst, true);
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_stage_bwd<Real, R, MAXT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const uint64_t ntiles = 1ull << hst.n_glob;
    k_stage_bwd<Real, R, MAXT><<<(unsigned)ntiles, 1u << (hst.T - R), smem, s>>>(
        (C*)L.psi, (C*)L.lam, L.stage, L.groups, (const DevOp<Real>*)L.ops, (const DevTerm<Real>*)L.terms,
        (const PhaseSlot<Real>*)L.slots, L.partial);
    return cudaGetLastError();
}
template <typename Real, int R>
static cudaError_t launch_bwd_R(const StageLaunch& L, const Stage& hst, cudaStream_t s) {
    if ((hst.T - R) <= 8) return launch_bwd_RT<Real, R, 256>(L, hst, s);
    if ((hst.T - R) == 9) return launch_bwd_RT<Real, R, 512>(L, hst, s);
    return cudaErrorInvalidConfiguration;
}

cudaError_t launch_stage_bwd(int elem_bytes, const StageLaunch& L, const Stage& hst, cudaStream_t s) {
    if (elem_bytes == 8) {
        switch (hst.R) {
            case 1: return launch_bwd_R<float, 1>(L, hst, s);
            case 2: return launch_bwd_R<float, 2>(L, hst, s);
            case 3: return launch_bwd_R<float, 3>(L, hst, s);
            case 4: return launch_bwd_R<float, 4>(L, hst, s);
        }
    } else {
        switch (hst.R) {
            case 1: return launch_bwd_R<double, 1>(L, hst, s);
            case 2: return launch_bwd_R<double, 2>(L, hst, s);
            case 3: return launch_bwd_R<double, 3>(L, hst, s);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace svk
