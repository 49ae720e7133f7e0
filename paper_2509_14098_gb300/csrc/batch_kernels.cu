// batch_kernels.cu — many small circuits, forward + observable + adjoint gradient, in
// one persistent launch (complex64).
//
// One CTA takes one circuit at a time from a queue (largest first) and runs it to the
// end; the stage machinery is the one of the single-circuit sweep (Sec. 4.3 tiles in
// shared memory, the register-level partition inside them), but the tile width,
// register width and thread count vary per circuit, so the CTA loops its threads
// over the 2^(T-R) "virtual threads" of each register group.
//
// Per circuit (S = number of forward stages):
//   stage 0 .. S-2 : tiles start from |0...0> (stage 0) or are loaded, forward ops,
//                    stored to the circuit's workspace;
//   stage S-1      : forward ops, then per amplitude h = <x|O|x> (O diagonal: Z strings),
//                    E += h |psi_x|^2 and lambda_x = h psi_x, then the adjoint program's
//                    first stage (the same tile bits) on psi and lambda with gradient ops;
//                    psi and lambda stored only if more adjoint stages follow;
//   adjoint 1 .. S-1: psi and lambda loaded, adjoint ops, stored except by the last.
// A single-stage circuit therefore never touches HBM (whole-tile circuits live in
// shared memory; wider single-stage circuits process their tiles independently).
#include <algorithm>

#include "batch.h"
#include "kdev.cuh"
#include "kernels.h"

namespace svk {

namespace {

constexpr int kNT = 512;            // threads per CTA
constexpr int kNW = kNT / 32;
constexpr int kLogNT = 9;
static_assert(sizeof(Stage) % 8 == 0, "Stage copies use 8-byte words");

struct Ctx {
    float2* tiles;
    Stage* st[2];
    Group* grp[2];
    DevOp<float>* ops[2];
    PhaseSlot<float>* sl[2];
    uint32_t* ang[2];
    float* gsm;
    double* gacc;
    double* red;
};

__device__ __forceinline__ void copy_stage(Stage* dst, const Stage* __restrict__ src, uint32_t tid) {
    const uint64_t* s = reinterpret_cast<const uint64_t*>(src);
    uint64_t* d = reinterpret_cast<uint64_t*>(dst);
    for (uint32_t i = tid; i < sizeof(Stage) / 8; i += kNT) d[i] = s[i];
}

// Form the matrices of bound parametric rotations (same row-major (re, im) layout as
// the host lowering: RX = [[c, -is], [-is, c]], RY = [[c, -s], [s, c]],
// RZ = diag(c - is, c + is), c = cos(theta/2), s = sin(theta/2); the adjoint program
// holds the conjugate transposes).
__device__ __forceinline__ void bind_ops(DevOp<float>* sops, uint32_t n_ops, const double* __restrict__ prm,
                                         uint32_t tid) {
    for (uint32_t i = tid; i < n_ops; i += kNT) {
        DevOp<float>& o = sops[i];
        if (!(o.flags & F_BIND)) continue;
        double sd, cd;
        sincos(0.5 * prm[o.term_off], &sd, &cd);
        const float c = (float)cd;
        const float s = (o.u & BK_DAGGER) ? -(float)sd : (float)sd;
        float m[8] = {c, 0.f, 0.f, 0.f, 0.f, 0.f, c, 0.f};
        switch (o.u & 3) {
            case BK_RX: m[3] = -s; m[5] = -s; break;
            case BK_RY: m[2] = -s; m[4] = s; break;
            default: m[1] = -s; m[7] = s; break;   // BK_RZ
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) o.m[k] = m[k];
    }
}

// 16-byte chunk c of a tile: tile element 2c (tile bit 0 is physical bit 0).
struct ChunkMap {
    uint64_t ptid;
    uint32_t stid;
};
__device__ __forceinline__ ChunkMap chunk_map(const Stage* S, uint32_t tid) {
    ChunkMap m{0, 0};
    const int nb = min((int)S->T - 1, kLogNT);
    for (int b = 0; b < nb; ++b)
        if ((tid >> b) & 1) {
            m.ptid ^= S->ptile[b + 1];
            m.stid ^= S->swbit[b + 1];
        }
    return m;
}
__device__ __forceinline__ void chunk_hi(const Stage* S, uint32_t i, uint64_t* p, uint32_t* s) {
    for (int b = 0; (i >> b) != 0; ++b)
        if ((i >> b) & 1) {
            *p ^= S->ptile[kLogNT + b + 1];
            *s ^= S->swbit[kLogNT + b + 1];
        }
}
__device__ __forceinline__ void tile_load(float2* buf, const float2* __restrict__ g, uint64_t base, const Stage* S,
                                          const ChunkMap& cm, uint32_t tid) {
    const uint32_t nch = 1u << (S->T - 1);
    for (uint32_t i = 0; (i << kLogNT) + tid < nch; ++i) {
        uint64_t p = cm.ptid;
        uint32_t s = cm.stid;
        chunk_hi(S, i, &p, &s);
        cp_async16(buf + s, g + (base | p));
    }
}
__device__ __forceinline__ void tile_store(const float2* buf, float2* g, uint64_t base, const Stage* S,
                                           const ChunkMap& cm, uint32_t tid) {
    const uint32_t nch = 1u << (S->T - 1);
    for (uint32_t i = 0; (i << kLogNT) + tid < nch; ++i) {
        uint64_t p = cm.ptid;
        uint32_t s = cm.stid;
        chunk_hi(S, i, &p, &s);
        *reinterpret_cast<float4*>(g + (base | p)) = *reinterpret_cast<const float4*>(buf + s);
    }
}
// |0...0> restricted to the tile with global bits `base`
__device__ __forceinline__ void tile_zero(float2* buf, uint64_t base, int T, uint32_t tid) {
    const uint32_t nch = 1u << (T - 1);
    for (uint32_t c = tid; c < nch; c += kNT) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c == 0 && base == 0) v.x = 1.f;   // element 0 sits at storage 0 (the swizzle is linear)
        *reinterpret_cast<float4*>(buf + 2 * c) = v;
    }
}

// Apply the register groups of one stage to the tile(s): the CTA's threads loop over
// the 2^(T-R) virtual threads of each group.  NV = 2: psi and lambda, gradient ops add
// Im <lambda|G|psi> into gsm[slot][warp] (every warp is either wholly active or idle,
// because 2^(T-R) is a multiple of 32).
template <int R, int NV>
__device__ __noinline__ void run_groups(float2* cur0, float2* cur1, const Stage* S, const Group* sgr,
                                        const DevOp<float>* sops, const PhaseSlot<float>* ssl, const uint32_t* sang,
                                        const DevTerm<float>* __restrict__ terms, uint64_t base, float* gsm,
                                        uint32_t tid) {
    using A = RegT<float>::type;
    const int TR = (int)S->T - R;
    const uint32_t nvt = 1u << TR;
    const uint32_t warp = tid >> 5, lane = tid & 31;
    OpCtx<float> x;
    x.slots = ssl;
    x.ang = sang;
    x.tang = nullptr;   // virtual threads: the thread-bit terms are summed per op
    x.nthr = nvt;
    x.TR = TR;
    x.terms = terms;
    for (uint32_t g = 0; g < S->n_groups; ++g) {
        const Group& G = sgr[g];
        uint32_t sr[R];
#pragma unroll
        for (int j = 0; j < R; ++j) sr[j] = G.sreg[j];
        const bool pairs = G.pairs != 0;
        const DevOp<float>* op = sops + G.op_off;
        const uint32_t nops = G.n_ops;
        for (uint32_t vt = tid; vt < nvt; vt += kNT) {
            uint64_t f = 0;
            uint32_t soff = 0;
            for (int i = 0; i < TR; ++i)
                if ((vt >> i) & 1) {
                    f ^= G.pthr[i];
                    soff ^= G.sthr[i];
                }
            x.fix = base ^ f;
            x.tid = vt;
            A a[NV][1 << R];
            load_regs<A, float2, R>(a[0], cur0, soff, sr, pairs);
            if constexpr (NV == 2) load_regs<A, float2, R>(a[1], cur1, soff, sr, pairs);
            for (uint32_t oi = 0; oi < nops; ++oi) {
                const DevOp<float> o = load_op<float>(op + oi);
                if (NV == 2 && o.type >= OP_GRAD_X) {
                    float acc = 0.f;
                    if (o.type == OP_GRAD_Z && o.u) {
#pragma unroll
                        for (int k = 0; k < (1 << R); ++k)
                            acc += im_conj_mul<float>(to_c<float>(a[NV - 1][k]), to_c<float>(a[0][k]));
                        if ((x.fix & o.ctrl_fix) != 0) acc = -acc;
                    } else {
                        SVK_SWITCH_J(o.j, R, (acc = grad_pairs<float, R, J_>(a[0], a[NV - 1], o.type)));
                    }
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
                    if (lane == 0) gsm[o.slot * kNW + warp] += acc;
                } else {
                    apply_op<float, R, NV>(a, o, x);
                }
            }
            store_regs<A, float2, R>(a[0], cur0, soff, sr, pairs);
            if constexpr (NV == 2) store_regs<A, float2, R>(a[1], cur1, soff, sr, pairs);
        }
        __syncthreads();
    }
}

template <int NV>
__device__ __forceinline__ void run_groups_R(int R, float2* c0, float2* c1, const Stage* S, const Group* g,
                                             const DevOp<float>* o, const PhaseSlot<float>* sl, const uint32_t* ang,
                                             const DevTerm<float>* terms, uint64_t base, float* gsm, uint32_t tid) {
    switch (R) {
        case 2: run_groups<2, NV>(c0, c1, S, g, o, sl, ang, terms, base, gsm, tid); break;
        case 3: run_groups<3, NV>(c0, c1, S, g, o, sl, ang, terms, base, gsm, tid); break;
        default: run_groups<4, NV>(c0, c1, S, g, o, sl, ang, terms, base, gsm, tid); break;
    }
}

// E += sum_x h(x) |psi_x|^2 and lambda_x = h(x) psi_x over one tile (h in FP32, the
// tile's partial sum in FP64, added by thread 0 in a fixed order).
__device__ __forceinline__ void observe(const float2* psi, float2* lam, const Stage* S, uint64_t base,
                                        const ObsTerm* __restrict__ obs, uint32_t n_obs, double* red, double* E,
                                        uint32_t tid) {
    const int T = (int)S->T;
    float acc = 0.f;
    for (uint32_t e = tid; e < (1u << T); e += kNT) {
        uint64_t p = base;
        uint32_t s = 0;
        for (int b = 0; b < T; ++b)
            if ((e >> b) & 1) {
                p |= S->ptile[b];
                s ^= S->swbit[b];
            }
        float h = 0.f;
        for (uint32_t t = 0; t < n_obs; ++t) {
            const float c = (float)obs[t].coeff;
            h += (__popcll(p & obs[t].zmask) & 1) ? -c : c;
        }
        const float2 v = psi[s];
        acc = fmaf(h, v.x * v.x + v.y * v.y, acc);
        lam[s] = make_float2(h * v.x, h * v.y);
    }
    double d = (double)acc;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
    if ((tid & 31) == 0) red[tid >> 5] = d;
    __syncthreads();
    if (tid == 0) {
        double sum = 0.0;
        for (int w = 0; w < kNW; ++w) sum += red[w];
        *E += sum;
    }
}

// sum the per-warp FP32 gradient partials of this tile into the FP64 slot sums
__device__ __forceinline__ void grad_flush(float* gsm, double* gacc, uint32_t n_slots, uint32_t tid) {
    for (uint32_t s = tid; s < n_slots; s += kNT) {
        double sum = 0.0;
        for (int w = 0; w < kNW; ++w) {
            sum += (double)gsm[s * kNW + w];
            gsm[s * kNW + w] = 0.f;
        }
        gacc[s] += sum;
    }
}

enum SweepKind { SW_FWD = 0, SW_FUSED = 1, SW_BWD = 2 };

// One pass over the tiles of a stage (see the file comment for the three kinds).
__device__ void sweep(const Ctx& c, const BatchArgs& a, const BatchProg& P, const BatchCirc& C, int kind,
                      bool zero_init, bool store, float2* psi_g, float2* lam_g, double* E, uint32_t tid) {
    const Stage* S = kind == SW_BWD ? c.st[1] : c.st[0];
    const int T = (int)S->T;
    const uint32_t ng = S->n_glob;
    const uint64_t ntiles = 1ull << ng;
    const int NV = kind == SW_FWD ? 1 : 2;
    const int nload = kind == SW_BWD ? 2 : 1;
    const int NB = (ntiles > 1 && ((size_t)NV * 2 * (8ull << T)) <= a.sm.tiles) ? 2 : 1;
    uint64_t gmask = 0;
    for (uint32_t i = 0; i < ng; ++i) gmask |= 1ull << S->glob_pos[i];
    const uint64_t low = ng ? (1ull << S->glob_pos[0]) : 0;
    float2* vec[2] = {psi_g, lam_g};
    auto buf = [&](int v, int b) { return c.tiles + ((size_t)(v * NB + b) << T); };
    const ChunkMap cm = chunk_map(S, tid);
    const DevTerm<float>* fterms = a.terms + P.f_term;
    const DevTerm<float>* bterms = a.terms + P.b_term;

    uint64_t base = 0;
    if (!zero_init) {
        for (int v = 0; v < nload; ++v) tile_load(buf(v, 0), vec[v], base, S, cm, tid);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    for (uint64_t t = 0; t < ntiles; ++t) {
        const int cb = NB == 2 ? (int)(t & 1) : 0;
        const uint64_t bn = ((base | ~gmask) + low) & gmask;
        if (zero_init) {
            tile_zero(buf(0, cb), base, T, tid);
        } else if (NB == 2 && t + 1 < ntiles) {
            for (int v = 0; v < nload; ++v) tile_load(buf(v, cb ^ 1), vec[v], bn, S, cm, tid);
            asm volatile("cp.async.commit_group;\ncp.async.wait_group 1;\n" ::: "memory");
        } else {
            if (NB == 1 && t > 0) {
                for (int v = 0; v < nload; ++v) tile_load(buf(v, 0), vec[v], base, S, cm, tid);
                asm volatile("cp.async.commit_group;\n" ::: "memory");
            }
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        if (kind != SW_BWD && c.st[0]->n_phase)
            tile_angles<float>(c.ang[0], a.slots + P.f_slot, fterms, *c.st[0], base, tid, kNT);
        if (kind != SW_FWD && c.st[1]->n_phase)
            tile_angles<float>(c.ang[1], a.slots + P.b_slot, bterms, *c.st[1], base, tid, kNT);
        __syncthreads();
        float2* p0 = buf(0, cb);
        float2* p1 = NV == 2 ? buf(1, cb) : nullptr;
        if (kind != SW_BWD)
            run_groups_R<1>((int)c.st[0]->R, p0, nullptr, c.st[0], c.grp[0], c.ops[0], c.sl[0], c.ang[0], fterms,
                            base, c.gsm, tid);
        if (kind == SW_FUSED) {
            observe(p0, p1, S, base, a.obs + C.obs_off, C.n_obs, c.red, E, tid);
            __syncthreads();
        }
        if (kind != SW_FWD) {
            run_groups_R<2>((int)c.st[1]->R, p0, p1, c.st[1], c.grp[1], c.ops[1], c.sl[1], c.ang[1], bterms, base,
                            c.gsm, tid);
            grad_flush(c.gsm, c.gacc, c.st[1]->n_slots, tid);
        }
        if (store)
            for (int v = 0; v < NV; ++v) tile_store(buf(v, cb), vec[v], base, S, cm, tid);
        base = bn;
        __syncthreads();
    }
}

// Stage the program of one stage (direction d) into shared memory and bind its
// parametric ops to this circuit's parameters.
__device__ __forceinline__ void load_stage(const Ctx& c, int d, const BatchArgs& a, const BatchProg& P,
                                           const double* prm, uint32_t s, uint32_t tid) {
    const uint32_t st_idx = (d == 0 ? P.f_stage : P.b_stage) + s;
    copy_stage(c.st[d], a.stages + st_idx, tid);
    __syncthreads();
    const Stage& S = *c.st[d];
    stage_prologue<float>(c.grp[d], c.ops[d], c.sl[d], S, a.groups + (d == 0 ? P.f_group : P.b_group),
                          a.ops + (d == 0 ? P.f_op : P.b_op), a.slots + (d == 0 ? P.f_slot : P.b_slot), tid, kNT);
    __syncthreads();
    bind_ops(c.ops[d], S.n_ops, prm, tid);
}

// the adjoint stage's FP64 slot sums -> this circuit's gradient entries (one thread,
// fixed order: several slots may feed one parameter)
__device__ __forceinline__ void grad_commit(const Ctx& c, const BatchArgs& a, const BatchProg& P, const BatchCirc& C,
                                            uint32_t tid) {
    __syncthreads();
    if (tid == 0) {
        const Stage& S = *c.st[1];
        for (uint32_t s = 0; s < S.n_slots; ++s)
            a.grad[C.param_off + a.slot_param[P.slot_param + S.slot_off + s]] += c.gacc[s];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kNT, 1) k_batch(const BatchArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ uint32_t s_circ;
    __shared__ double s_E;
    const uint32_t tid = threadIdx.x;
    Ctx c;
    c.tiles = reinterpret_cast<float2*>(sm);
    for (int d = 0; d < 2; ++d) {
        c.st[d] = reinterpret_cast<Stage*>(sm + a.sm.st[d]);
        c.grp[d] = reinterpret_cast<Group*>(sm + a.sm.grp[d]);
        c.ops[d] = reinterpret_cast<DevOp<float>*>(sm + a.sm.ops[d]);
        c.sl[d] = reinterpret_cast<PhaseSlot<float>*>(sm + a.sm.slots[d]);
        c.ang[d] = reinterpret_cast<uint32_t*>(sm + a.sm.ang[d]);
    }
    c.gsm = reinterpret_cast<float*>(sm + a.sm.gsm);
    c.gacc = reinterpret_cast<double*>(sm + a.sm.gacc);
    c.red = reinterpret_cast<double*>(sm + a.sm.red);

    for (;;) {
        if (tid == 0) s_circ = atomicAdd(a.queue, 1u);
        __syncthreads();
        const uint32_t ci = s_circ;
        if (ci >= a.n_circ) break;
        const BatchCirc C = a.circs[ci];
        const BatchProg P = a.progs[C.prog];
        const double* prm = a.params + C.param_off;
        float2* psi_g = reinterpret_cast<float2*>(a.ws) + C.ws;
        float2* lam_g = psi_g + (1ull << P.n);
        if (tid == 0) s_E = 0.0;
        for (uint32_t i = tid; i < a.sm.max_slots * kNW; i += kNT) c.gsm[i] = 0.f;
        for (uint32_t i = tid; i < a.sm.max_slots; i += kNT) c.gacc[i] = 0.0;
        for (uint32_t s = 0; s < P.n_f; ++s) {
            const bool last = s + 1 == P.n_f;
            load_stage(c, 0, a, P, prm, s, tid);
            if (last) load_stage(c, 1, a, P, prm, 0, tid);
            __syncthreads();
            sweep(c, a, P, C, last ? SW_FUSED : SW_FWD, s == 0, last ? P.n_b > 1 : true, psi_g, lam_g, &s_E, tid);
        }
        grad_commit(c, a, P, C, tid);
        for (uint32_t s = 1; s < P.n_b; ++s) {
            for (uint32_t i = tid; i < a.sm.max_slots; i += kNT) c.gacc[i] = 0.0;
            load_stage(c, 1, a, P, prm, s, tid);
            __syncthreads();
            sweep(c, a, P, C, SW_BWD, false, s + 1 < P.n_b, psi_g, lam_g, &s_E, tid);
            grad_commit(c, a, P, C, tid);
        }
        if (tid == 0) a.expval[C.out] = s_E;
        __syncthreads();   // s_circ / s_E are rewritten by the next claim
    }
}

}  // namespace

cudaError_t launch_batch(const BatchArgs& a, int grid, cudaStream_t s) {
    static bool cfg = false;
    if (!cfg) {
        cudaError_t e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024 - 2048);
        if (e != cudaSuccess) return e;
        cfg = true;
    }
    k_batch<<<grid, kNT, a.sm.total, s>>>(a);
    return cudaGetLastError();
}

cudaError_t batch_occupancy(size_t smem, int* per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024 - 2048);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_batch, kNT, smem);
}

int batch_threads() { return kNT; }

// ---------------------------------------------------------------------------
// Wide circuits of a batch run as generated stage kernels over all circuits of one
// structure at once (jit.h, batched mode); these three kernels do the rest of one
// evaluation for such a group of ncirc circuits of n qubits (states of circuit c at
// psi + c 2^n, lambda at lam + c 2^n).
// ---------------------------------------------------------------------------

// lambda_x = h(x) psi_x and the partial sums of E = sum_x h(x) |psi_x|^2, with
// h(x) = sum_t coeff_t (-1)^{|x & zmask_t|} (circuit c's terms obs[obs_off[c] ..
// obs_off[c + 1])); block (b, c) covers amplitudes [b chunk, (b + 1) chunk) and writes
// epart[c * gridDim.x + b] (FP32 per thread over its amplitudes, FP64 above).
__global__ void __launch_bounds__(256) k_bgs_obs(const float2* __restrict__ psi, float2* __restrict__ lam, int n,
                                                 const ObsTerm* __restrict__ obs, const uint32_t* __restrict__ obs_off,
                                                 double* __restrict__ epart) {
    __shared__ double red[8];
    const uint32_t c = blockIdx.y, tid = threadIdx.x;
    const uint64_t amps = 1ull << n;
    const uint64_t chunk = amps / gridDim.x;
    const uint64_t x0 = (uint64_t)blockIdx.x * chunk;
    const float2* ps = psi + ((uint64_t)c << n);
    float2* ls = lam + ((uint64_t)c << n);
    const uint32_t t0 = obs_off[c], t1 = obs_off[c + 1];
    float e = 0.f;
    for (uint64_t x = x0 + tid; x < x0 + chunk; x += blockDim.x) {
        float h = 0.f;
        for (uint32_t t = t0; t < t1; ++t) {
            const float cf = (float)obs[t].coeff;
            h += (__popcll(x & obs[t].zmask) & 1) ? -cf : cf;
        }
        const float2 v = ps[x];
        ls[x] = make_float2(h * v.x, h * v.y);
        e = fmaf(h, fmaf(v.x, v.x, v.y * v.y), e);
    }
    double d = (double)e;
    for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
    if ((tid & 31) == 0) red[tid >> 5] = d;
    __syncthreads();
    if (tid == 0) {
        double sum = 0.0;
        for (uint32_t w = 0; w < (blockDim.x + 31) / 32; ++w) sum += red[w];
        epart[(uint64_t)c * gridDim.x + blockIdx.x] = sum;
    }
}

// slotsum[c * nst + slot_off + s] = sum over tiles t of partial[(c * ntiles + t) * nsl + s]
// (one block per circuit, one thread per slot, tiles in order)
__global__ void k_bgs_slotsum(const double* __restrict__ partial, uint32_t ntiles, uint32_t nsl, uint32_t slot_off,
                              uint32_t nst, double* __restrict__ slotsum) {
    const uint32_t c = blockIdx.x;
    for (uint32_t sl = threadIdx.x; sl < nsl; sl += blockDim.x) {
        double x = 0.0;
        for (uint32_t t = 0; t < ntiles; ++t) x += partial[((uint64_t)c * ntiles + t) * nsl + sl];
        slotsum[(uint64_t)c * nst + slot_off + sl] = x;
    }
}

// E and the gradient of circuit c: expval[outidx[c]] = sum of its nblk E partials;
// grad[pofs[c] + p] = sum of its slot sums over the slots of parameter p
// (slots plist[pidx[p] .. pidx[p + 1]))
__global__ void k_bgs_finish(const double* __restrict__ epart, uint32_t nblk, const double* __restrict__ slotsum,
                             uint32_t nst, const uint32_t* __restrict__ pidx, const uint32_t* __restrict__ plist,
                             uint32_t np, const uint32_t* __restrict__ pofs, const uint32_t* __restrict__ outidx,
                             double* __restrict__ expval, double* __restrict__ grad) {
    const uint32_t c = blockIdx.x;
    if (threadIdx.x == 0) {
        double e = 0.0;
        for (uint32_t b = 0; b < nblk; ++b) e += epart[(uint64_t)c * nblk + b];
        expval[outidx[c]] = e;
    }
    for (uint32_t p = threadIdx.x; p < np; p += blockDim.x) {
        double g = 0.0;
        for (uint32_t k = pidx[p]; k < pidx[p + 1]; ++k) g += slotsum[(uint64_t)c * nst + plist[k]];
        grad[pofs[c] + p] = g;
    }
}

cudaError_t launch_bgs_obs(const void* psi, void* lam, int n, uint32_t ncirc, const ObsTerm* obs,
                           const uint32_t* obs_off, double* epart, uint32_t nblk, cudaStream_t s) {
    k_bgs_obs<<<dim3(nblk, ncirc), 256, 0, s>>>((const float2*)psi, (float2*)lam, n, obs, obs_off, epart);
    return cudaGetLastError();
}
cudaError_t launch_bgs_slotsum(const double* partial, uint32_t ncirc, uint32_t ntiles, uint32_t nsl, uint32_t slot_off,
                               uint32_t nst, double* slotsum, cudaStream_t s) {
    k_bgs_slotsum<<<ncirc, 64, 0, s>>>(partial, ntiles, nsl, slot_off, nst, slotsum);
    return cudaGetLastError();
}
cudaError_t launch_bgs_finish(const double* epart, uint32_t nblk, const double* slotsum, uint32_t nst,
                              const uint32_t* pidx, const uint32_t* plist, uint32_t np, const uint32_t* pofs,
                              const uint32_t* outidx, uint32_t ncirc, double* expval, double* grad, cudaStream_t s) {
    k_bgs_finish<<<ncirc, 128, 0, s>>>(epart, nblk, slotsum, nst, pidx, plist, np, pofs, outidx, expval, grad);
    return cudaGetLastError();
}

}  // namespace svk
