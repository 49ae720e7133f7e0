// stage_impl.cuh — one HBM sweep per partition (Sec. 4.3, single-device case:
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
// Im <lambda|G|psi> per parametric rotation: one warp's sum over its amplitudes of one
// tile is formed in the kernel's precision (FP32 for complex64, FP64 for complex128),
// then added in FP64 to that warp's per-CTA slot sum, across tiles; the warps' sums are
// added in FP64, in a fixed order, once at the end.
//
// This header holds the kernel template and its launchers; stage_inst.cu compiles one
// (precision, direction, register width) subset per object so the instantiations
// build in parallel.
#pragma once
#include <algorithm>

#include "kdev.cuh"
#include "kernels.h"
#include "stage_layout.cuh"

// Occupancy of <= 256-thread launches.  The sweep is issue-latency bound, so the
// forward kernel trades registers for resident warps (64 registers, single-buffered
// tiles: measured 10 % faster on the QFT30 stages than 128 registers with
// double-buffered tiles); the adjoint kernel, which holds psi and lambda in
// registers, keeps 128 registers and double buffering.
#ifndef SVK_MINB_FWD
#define SVK_MINB_FWD 4
#endif
#ifndef SVK_MINB_BWD
#define SVK_MINB_BWD 2
#endif

namespace svk {

// ---------------------------------------------------------------------------
// The stage sweep.  NV = 1: forward (psi).  NV = 2: adjoint (psi and lambda together,
// gradient ops accumulate Im <lambda|G|psi>).
// Persistent: CTA b handles tiles b, b + gridDim.x, ... and prefetches the next tile
// into the second buffer (cp.async) while it computes the current one.  Everything
// that does not depend on the tile (chunk offsets, each group's thread offsets) is
// computed once; the tile base advances by an addition in the masked bit space of
// the global bits: base(t + G) = ((base(t) | ~gmask) + pdep(G)) & gmask.  Gradient
// partial sums accumulate per CTA in FP64 (per warp, fixed order) and are written once.
// ---------------------------------------------------------------------------
template <typename Real, int R, int MAXT, int NV, int NB, bool CPLX>
__global__ void __launch_bounds__(MAXT, (MAXT >= 512 ? 1 : (NV == 1 ? SVK_MINB_FWD : SVK_MINB_BWD)))
    k_stage(typename CT<Real>::C* __restrict__ psi, typename CT<Real>::C* __restrict__ lam,
            const Stage* __restrict__ stp, const Group* __restrict__ groups,
            const DevOp<Real>* __restrict__ gops, const DevTerm<Real>* __restrict__ terms,
            const PhaseSlot<Real>* __restrict__ slots, double* __restrict__ partial) {
    using C = typename CT<Real>::C;
    using A = typename RegT<Real>::type;
    using Ang = typename AngT<Real>::type;
    constexpr int APC = 16 / (int)sizeof(C);
    constexpr int LA = APC == 2 ? 1 : 0;
    constexpr int NCH = (1 << R) / APC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Stage& st = *stp;
    const int T = (int)st.T;
    const int TR = T - R;
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
    const uint32_t nw = (nthr + 31) >> 5, warp = tid >> 5, lane = tid & 31;
    const uint32_t ng = st.n_groups;
    const uint32_t nslots = st.n_slots;
    const SmemLayout Ly = smem_layout((int)sizeof(C), NV, NB, st.T, ng, st.n_ops, st.n_phase, nslots, nthr, NCH);
    C* tiles = reinterpret_cast<C*>(smem_raw);              // tile (v, b) at (v * NB + b) << T
    Group* sgr = reinterpret_cast<Group*>(smem_raw + Ly.groups);
    DevOp<Real>* sops = reinterpret_cast<DevOp<Real>*>(smem_raw + Ly.ops);
    PhaseSlot<Real>* ssl = reinterpret_cast<PhaseSlot<Real>*>(smem_raw + Ly.slots);
    Ang* sang = reinterpret_cast<Ang*>(smem_raw + Ly.ang);
    uint64_t* gfix = reinterpret_cast<uint64_t*>(smem_raw + Ly.gfix);
    uint64_t* chp = reinterpret_cast<uint64_t*>(smem_raw + Ly.chp);
    uint32_t* gsoff = reinterpret_cast<uint32_t*>(smem_raw + Ly.gsoff);
    uint32_t* chs = reinterpret_cast<uint32_t*>(smem_raw + Ly.chs);
    double* gsm = reinterpret_cast<double*>(smem_raw + Ly.gsm);
    Ang* tang = reinterpret_cast<Ang*>(smem_raw + Ly.tang);
    const bool ttab = angle_table_fits(st.n_phase, nthr, sizeof(Ang));
    const bool gtab = group_table_fits(ng, nthr);
    const uint64_t ntiles = 1ull << st.n_glob;
    C* vec[2] = {psi, lam};

    uint64_t t = blockIdx.x;
    if (t >= ntiles) return;
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
#pragma unroll
        for (int v = 0; v < NV; ++v) cp_async16(tiles + ((size_t)(v * NB) << T) + (stid ^ si), vec[v] + (base | (ptid ^ pi)));
        if (tid == 0) {
            chp[i] = pi;
            chs[i] = si;
        }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    stage_prologue<Real>(sgr, sops, ssl, st, groups, gops, slots, tid, nthr);
    if (gtab)
        for (uint32_t g = 0; g < ng; ++g) {
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
    if (NV == 2)
        for (uint32_t i = tid; i < nslots * nw; i += nthr) gsm[i] = 0.0;
    if (ttab)   // each thread's own column: the thread-bit part of every phase slot
        for (uint32_t p = 0; p < st.n_phase; ++p) {
            const PhaseSlot<Real>& ps = slots[st.phase_off + p];
            Ang a = 0;
            for (int i = 0; i < TR; ++i)
                if ((tid >> i) & 1) a += ps.J[i];
            tang[p * nthr + tid] = a;
        }
    __syncthreads();

    OpCtx<Real> x;
    x.slots = ssl;
    x.ang = sang;
    x.tid = tid;
    x.nthr = nthr;
    x.tang = ttab ? tang : nullptr;
    x.TR = TR;
    x.terms = terms;
    const uint32_t wmask = nthr >= 32 ? 0xffffffffu : ((1u << nthr) - 1u);
    for (uint32_t it = 0; t < ntiles; t += gridDim.x, ++it) {
        const int cb = NB == 2 ? (int)(it & 1) : 0;
        const uint64_t tn = t + gridDim.x;
        const uint64_t bn = ((base | ~gmask) + pstep) & gmask;
        if (NB == 2 && tn < ntiles) {   // prefetch the next tile into the other buffer
#pragma unroll
            for (int i = 0; i < NCH; ++i)
#pragma unroll
                for (int v = 0; v < NV; ++v)
                    cp_async16(tiles + ((size_t)(v * NB + (cb ^ 1)) << T) + (stid ^ chs[i]),
                               vec[v] + (bn | (ptid ^ chp[i])));
            asm volatile("cp.async.commit_group;\ncp.async.wait_group 1;\n" ::: "memory");
        } else {
            if (NB == 1 && it > 0) {       // one buffer: load this tile now (the first came with the prologue)
#pragma unroll
                for (int i = 0; i < NCH; ++i)
#pragma unroll
                    for (int v = 0; v < NV; ++v)
                        cp_async16(tiles + ((size_t)(v * NB) << T) + (stid ^ chs[i]), vec[v] + (base | (ptid ^ chp[i])));
                asm volatile("cp.async.commit_group;\n" ::: "memory");
            }
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        if (st.n_phase) tile_angles<Real>(sang, slots, terms, st, base, tid, nthr);
        __syncthreads();
        C* cur0 = tiles + ((size_t)cb << T);
        C* cur1 = tiles + ((size_t)(NB + cb) << T);
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
            const DevOp<Real>* op = sops + G.op_off;
            const uint32_t nops = G.n_ops;
            A a[NV][1 << R];
            load_regs<A, C, R>(a[0], cur0, soff, sr, pairs);
            if constexpr (NV == 2) load_regs<A, C, R>(a[NV - 1], cur1, soff, sr, pairs);
            for (uint32_t oi = 0; oi < nops; ++oi) {
                const DevOp<Real> o = load_op<Real>(op + oi);
                if (NV == 2 && o.type >= OP_GRAD_X) {
                    const auto& ps = a[0];
                    const auto& la = a[NV - 1];
                    Real acc = 0;
                    if (o.type == OP_GRAD_Z && o.u) {   // Z on a non-register bit: a sign per thread
#pragma unroll
                        for (int k = 0; k < (1 << R); ++k) acc += im_conj_mul<Real>(to_c<Real>(la[k]), to_c<Real>(ps[k]));
                        if ((x.fix & o.ctrl_fix) != 0) acc = -acc;
                    } else {
                        SVK_SWITCH_J(o.j, R, (acc = grad_pairs<Real, R, J_>(ps, la, o.type)));
                    }
                    Real v = acc;   // over the warp in the kernel's precision, then FP64 across tiles
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1)
                        if ((uint32_t)off < nthr) v += __shfl_xor_sync(wmask, v, off);
                    if (lane == 0) gsm[o.slot * nw + warp] += (double)v;
                } else {
                    apply_op<Real, R, NV, CPLX>(a, o, x);
                }
            }
            store_regs<A, C, R>(a[0], cur0, soff, sr, pairs);
            if constexpr (NV == 2) store_regs<A, C, R>(a[NV - 1], cur1, soff, sr, pairs);
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < NCH; ++i)
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const float4 val = *reinterpret_cast<const float4*>(tiles + ((size_t)(v * NB + cb) << T) + (stid ^ chs[i]));
                *reinterpret_cast<float4*>(vec[v] + (base | (ptid ^ chp[i]))) = val;
            }
        base = bn;
        __syncthreads();   // the current buffers are refilled by the prefetch after next
    }
    if (NV == 2)
        for (uint32_t s = tid; s < nslots; s += nthr) {
            double sum = 0.0;
            for (uint32_t w = 0; w < nw; ++w) sum += gsm[s * nw + w];
            partial[(size_t)blockIdx.x * nslots + s] = sum;
        }
}

// ---------------------------------------------------------------------------
// launch wrappers
// ---------------------------------------------------------------------------
template <typename Real, int R, int MAXT, int NV, int NB, bool CPLX>
static cudaError_t try_launch(const StageLaunch& L, const Stage& hst, cudaStream_t s, uint32_t* grid_out,
                              int min_per_sm, bool* launched) {
    using C = typename CT<Real>::C;
    *launched = false;
    const size_t smem = smem_bytes_nb(sizeof(C), hst, NV, NB);
    if (smem > 227 * 1024) return cudaSuccess;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_stage<Real, R, MAXT, NV, NB, CPLX>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const uint64_t ntiles = 1ull << hst.n_glob;
    const int nthr = 1 << (hst.T - R);
    int per_sm = 0, dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stage<Real, R, MAXT, NV, NB, CPLX>, nthr, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < min_per_sm || per_sm < 1) return cudaSuccess;
    const uint64_t grid = std::min<uint64_t>(ntiles, (uint64_t)per_sm * (uint64_t)nsm);
    if (grid_out) *grid_out = (uint32_t)grid;
    k_stage<Real, R, MAXT, NV, NB, CPLX><<<(unsigned)grid, nthr, smem, s>>>(
        (C*)L.psi, (C*)L.lam, L.stage, L.groups, (const DevOp<Real>*)L.ops, (const DevTerm<Real>*)L.terms,
        (const PhaseSlot<Real>*)L.slots, L.partial);
    *launched = true;
    return cudaGetLastError();
}

// adjoint: double-buffered tiles while that still leaves >= 2 CTAs per SM, else single-
// buffered; forward: single-buffered (occupancy hides the loads, see SVK_MINB_FWD)
template <typename Real, int R, int MAXT, int NV, bool CPLX>
static cudaError_t launch_RT(const StageLaunch& L, const Stage& hst, cudaStream_t s, uint32_t* grid_out) {
    bool ok = false;
    cudaError_t e = cudaSuccess;
    if constexpr (NV == 2) {
        e = try_launch<Real, R, MAXT, NV, 2, CPLX>(L, hst, s, grid_out, 2, &ok);
        if (e != cudaSuccess || ok) return e;
    }
    e = try_launch<Real, R, MAXT, NV, 1, CPLX>(L, hst, s, grid_out, 1, &ok);
    if (e != cudaSuccess) return e;
    return ok ? cudaSuccess : cudaErrorInvalidConfiguration;
}
// 256-thread bound unless the tile needs 512 threads
template <typename Real, int R, int NV>
cudaError_t launch_R(const StageLaunch& L, const Stage& hst, cudaStream_t s, uint32_t* grid_out) {
    // complex64 forward stages without complex dense ops run an interpreter without them
    if constexpr (sizeof(Real) == 4 && NV == 1) {
        if (!hst.has_complex) {
            if ((hst.T - R) <= 8) return launch_RT<Real, R, 256, NV, false>(L, hst, s, grid_out);
            if ((hst.T - R) == 9) return launch_RT<Real, R, 512, NV, false>(L, hst, s, grid_out);
            return cudaErrorInvalidConfiguration;
        }
    }
    if ((hst.T - R) <= 8) return launch_RT<Real, R, 256, NV, true>(L, hst, s, grid_out);
    if ((hst.T - R) == 9) return launch_RT<Real, R, 512, NV, true>(L, hst, s, grid_out);
    return cudaErrorInvalidConfiguration;
}

}  // namespace svk
