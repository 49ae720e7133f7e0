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
#include "kdev.cuh"
#include "kernels.h"

namespace svk {

template <typename Real, int R>
__global__ void __launch_bounds__(512) k_stage_fwd(typename CT<Real>::C* __restrict__ psi,
                                                   const Stage* __restrict__ stp,
                                                   const Group* __restrict__ groups,
                                                   const Op* __restrict__ ops,
                                                   const Term* __restrict__ terms) {
    using C = typename CT<Real>::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tile = reinterpret_cast<C*>(smem_raw);
    const Stage& st = *stp;
    const int TR = (int)st.T - R;
    const uint32_t tid = threadIdx.x;
    const uint64_t base = tile_base(blockIdx.x, st.glob_pos);

    tile_load<C, R>(tile, psi, base, st.ptile, st.swbit, TR, tid);
    cp_async_commit_wait_all();
    __syncthreads();

    const uint32_t ng = st.n_groups;
    for (uint32_t g = 0; g < ng; ++g) {
        const Group& G = groups[st.group_off + g];
        uint64_t fix = base;
        uint32_t soff = 0;
        for (int i = 0; i < TR; ++i)
            if ((tid >> i) & 1) {
                fix ^= G.pthr[i];
                soff ^= G.sthr[i];
            }
        uint32_t sr[R];
#pragma unroll
        for (int j = 0; j < R; ++j) sr[j] = G.sreg[j];
        const bool pairs = G.pairs != 0;
        C a[1 << R];
        load_regs<C, R>(a, tile, soff, sr, pairs);
        const uint32_t nops = G.n_ops;
        for (uint32_t oi = 0; oi < nops; ++oi) apply_op<Real, R>(a, ops[G.op_off + oi], fix, terms);
        store_regs<C, R>(a, tile, soff, sr, pairs);
        __syncthreads();
    }
    tile_store<C, R>(tile, psi, base, st.ptile, st.swbit, TR, tid);
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

template <typename Real, int R, int J>
__device__ __forceinline__ Real grad_pairs(const typename CT<Real>::C (&ps)[1 << R],
                                           const typename CT<Real>::C (&la)[1 << R], uint8_t type) {
    Real acc = 0;
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) {
        if (k & (1 << J)) continue;
        const int k1 = k | (1 << J);
        if (type == OP_GRAD_X) {
            acc += im_conj_mul<Real>(la[k], ps[k1]) + im_conj_mul<Real>(la[k1], ps[k]);
        } else if (type == OP_GRAD_Y) {
            // Y|0> = i|1>, Y|1> = -i|0>:  Im(conj(l0)(-i p1)) + Im(conj(l1)(i p0))
            acc += -re_conj_mul<Real>(la[k], ps[k1]) + re_conj_mul<Real>(la[k1], ps[k]);
        } else {
            acc += im_conj_mul<Real>(la[k], ps[k]) - im_conj_mul<Real>(la[k1], ps[k1]);
        }
    }
    return acc;
}

template <typename Real, int R>
__global__ void __launch_bounds__(512) k_stage_bwd(typename CT<Real>::C* __restrict__ psi,
                                                   typename CT<Real>::C* __restrict__ lam,
                                                   const Stage* __restrict__ stp,
                                                   const Group* __restrict__ groups,
                                                   const Op* __restrict__ ops,
                                                   const Term* __restrict__ terms,
                                                   double* __restrict__ partial) {
    using C = typename CT<Real>::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Stage& st = *stp;
    const int T = (int)st.T;
    const int TR = T - R;
    C* tp = reinterpret_cast<C*>(smem_raw);
    C* tl = tp + (1u << T);
    float* gsm = reinterpret_cast<float*>(tl + (1u << T));
    const uint32_t tid = threadIdx.x;
    const uint32_t nw = (blockDim.x + 31) >> 5;
    const uint32_t warp = tid >> 5, lane = tid & 31;
    const uint32_t nslots = st.n_slots;
    const uint64_t base = tile_base(blockIdx.x, st.glob_pos);

    tile_load<C, R>(tp, psi, base, st.ptile, st.swbit, TR, tid);
    tile_load<C, R>(tl, lam, base, st.ptile, st.swbit, TR, tid);
    cp_async_commit_wait_all();
    for (uint32_t i = tid; i < nslots * nw; i += blockDim.x) gsm[i] = 0.f;
    __syncthreads();

    for (uint32_t g = 0; g < st.n_groups; ++g) {
        const Group& G = groups[st.group_off + g];
        uint64_t fix = base;
        uint32_t soff = 0;
        for (int i = 0; i < TR; ++i)
            if ((tid >> i) & 1) {
                fix ^= G.pthr[i];
                soff ^= G.sthr[i];
            }
        uint32_t sr[R];
#pragma unroll
        for (int j = 0; j < R; ++j) sr[j] = G.sreg[j];
        const bool pairs = G.pairs != 0;
        C ps[1 << R], la[1 << R];
        load_regs<C, R>(ps, tp, soff, sr, pairs);
        load_regs<C, R>(la, tl, soff, sr, pairs);
        for (uint32_t oi = 0; oi < G.n_ops; ++oi) {
            const Op& o = ops[G.op_off + oi];
            if (o.type >= OP_GRAD_X) {
                Real acc = 0;
                if (o.type == OP_GRAD_Z && o.u) {
                    // Z on a non-register bit: a sign per thread
#pragma unroll
                    for (int k = 0; k < (1 << R); ++k) acc += im_conj_mul<Real>(la[k], ps[k]);
                    if ((fix & o.ctrl_fix) != 0) acc = -acc;
                } else {
                    SVK_SWITCH_J(o.j, R, (acc = grad_pairs<Real, R, J_>(ps, la, o.type)));
                }
                float v = (float)acc;
                const uint32_t wmask = blockDim.x >= 32 ? 0xffffffffu : ((1u << blockDim.x) - 1u);
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
                    if ((uint32_t)off < blockDim.x) v += __shfl_xor_sync(wmask, v, off);
                if (lane == 0) gsm[o.slot * nw + warp] += v;
            } else {
                apply_op<Real, R>(ps, o, fix, terms);
                apply_op<Real, R>(la, o, fix, terms);
            }
        }
        store_regs<C, R>(ps, tp, soff, sr, pairs);
        store_regs<C, R>(la, tl, soff, sr, pairs);
        __syncthreads();
    }
    tile_store<C, R>(tp, psi, base, st.ptile, st.swbit, TR, tid);
    tile_store<C, R>(tl, lam, base, st.ptile, st.swbit, TR, tid);
    for (uint32_t s = tid; s < nslots; s += blockDim.x) {
        double sum = 0.0;
        for (uint32_t w = 0; w < nw; ++w) sum += (double)gsm[s * nw + w];
        partial[(size_t)blockIdx.x * nslots + s] = sum;
    }
}

// ---------------------------------------------------------------------------
// launch wrappers
// ---------------------------------------------------------------------------
template <typename Real, int R>
static cudaError_t launch_fwd_R(void* psi, const Stage* st, const Group* gr, const Op* op,
                                const Term* te, int T, uint64_t ntiles, cudaStream_t s) {
    using C = typename CT<Real>::C;
    const size_t smem = (size_t)sizeof(C) << T;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_stage_fwd<Real, R>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    k_stage_fwd<Real, R><<<(unsigned)ntiles, 1u << (T - R), smem, s>>>((C*)psi, st, gr, op, te);
    return cudaGetLastError();
}

cudaError_t launch_stage_fwd(int elem_bytes, int R, void* psi, const Stage* st, const Group* gr,
                             const Op* op, const Term* te, int T, uint64_t ntiles, cudaStream_t s) {
    if (elem_bytes == 8) {
        switch (R) {
            case 1: return launch_fwd_R<float, 1>(psi, st, gr, op, te, T, ntiles, s);
            case 2: return launch_fwd_R<float, 2>(psi, st, gr, op, te, T, ntiles, s);
            case 3: return launch_fwd_R<float, 3>(psi, st, gr, op, te, T, ntiles, s);
            case 4: return launch_fwd_R<float, 4>(psi, st, gr, op, te, T, ntiles, s);
            case 5: return launch_fwd_R<float, 5>(psi, st, gr, op, te, T, ntiles, s);
        }
    } else {
        switch (R) {
            case 1: return launch_fwd_R<double, 1>(psi, st, gr, op, te, T, ntiles, s);
            case 2: return launch_fwd_R<double, 2>(psi, st, gr, op, te, T, ntiles, s);
            case 3: return launch_fwd_R<double, 3>(psi, st, gr, op, te, T, ntiles, s);
            case 4: return launch_fwd_R<double, 4>(psi, st, gr, op, te, T, ntiles, s);
        }
    }
    return cudaErrorInvalidValue;
}

template <typename Real, int R>
static cudaError_t launch_bwd_R(void* psi, void* lam, const Stage* st, const Group* gr,
                                const Op* op, const Term* te, double* partial, int T,
                                uint32_t nslots, uint64_t ntiles, cudaStream_t s) {
    using C = typename CT<Real>::C;
    const uint32_t nthr = 1u << (T - R);
    const uint32_t nw = (nthr + 31) / 32;
    const size_t smem = ((size_t)sizeof(C) << (T + 1)) + (size_t)nslots * nw * sizeof(float);
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_stage_bwd<Real, R>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    k_stage_bwd<Real, R><<<(unsigned)ntiles, nthr, smem, s>>>((C*)psi, (C*)lam, st, gr, op, te, partial);
    return cudaGetLastError();
}

cudaError_t launch_stage_bwd(int elem_bytes, int R, void* psi, void* lam, const Stage* st,
                             const Group* gr, const Op* op, const Term* te, double* partial, int T,
                             uint32_t nslots, uint64_t ntiles, cudaStream_t s) {
    if (elem_bytes == 8) {
        switch (R) {
            case 1: return launch_bwd_R<float, 1>(psi, lam, st, gr, op, te, partial, T, nslots, ntiles, s);
            case 2: return launch_bwd_R<float, 2>(psi, lam, st, gr, op, te, partial, T, nslots, ntiles, s);
            case 3: return launch_bwd_R<float, 3>(psi, lam, st, gr, op, te, partial, T, nslots, ntiles, s);
            case 4: return launch_bwd_R<float, 4>(psi, lam, st, gr, op, te, partial, T, nslots, ntiles, s);
        }
    } else {
        switch (R) {
            case 1: return launch_bwd_R<double, 1>(psi, lam, st, gr, op, te, partial, T, nslots, ntiles, s);
            case 2: return launch_bwd_R<double, 2>(psi, lam, st, gr, op, te, partial, T, nslots, ntiles, s);
            case 3: return launch_bwd_R<double, 3>(psi, lam, st, gr, op, te, partial, T, nslots, ntiles, s);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace svk
