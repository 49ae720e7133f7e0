// aux_kernels.cu — bit-permutation sweep (the on-GPU form of the inter-partition
// exchange, Sec. 4.3 "Creating the Data Reshaping Operations"), Pauli-sum sweeps for
// expectation values and the adjoint seed lambda = O psi, FP64 reductions.
#include "kdev.cuh"
#include "kernels.h"

namespace svk {

// ---------------------------------------------------------------------------
// permutation: the tile contains the input's low bits and the input bits that land
// on the output's low bits (the host widens both runs to at least 512 bytes), so both
// the read and the write are contiguous runs.  Persistent CTAs, two tile buffers: the
// next tile's copy is in flight while the current one is written out.  Every chunk
// offset is XOR / OR-linear in the chunk index, so a thread forms its offsets once; a
// tile's global part is one OR-reduction over the warp (lane i holds global bit i).
// ---------------------------------------------------------------------------
constexpr int kPermThreads = 256;
constexpr int kPermChunks = 8;   // 16-byte chunks per thread and tile (tiles of 2^12 complex64 / 2^11 complex128)

__device__ __forceinline__ uint64_t warp_or64(uint64_t v) {
    const uint32_t lo = __reduce_or_sync(0xffffffffu, (uint32_t)v);
    const uint32_t hi = __reduce_or_sync(0xffffffffu, (uint32_t)(v >> 32));
    return ((uint64_t)hi << 32) | lo;
}

template <typename C>
__global__ void __launch_bounds__(kPermThreads, 3) k_permute(const C* __restrict__ in, C* __restrict__ out,
                                                          const __grid_constant__ PermDesc d, uint64_t ntiles) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int APC = 16 / (int)sizeof(C);   // elements per 16-byte chunk
    const uint32_t tid = threadIdx.x, lane = tid & 31u;
    const int T = (int)d.T;
    const uint32_t tsz = 1u << T, nch = tsz / APC;
    C* const buf0 = reinterpret_cast<C*>(smem_raw);
    C* const buf1 = buf0 + tsz;
    // this lane's global bit (input and output value), zero past the last one
    const uint64_t gin = lane < d.n_glob ? 1ull << d.glob_pos[lane] : 0ull;
    const uint64_t gou = lane < d.n_glob ? d.gout[lane] : 0ull;
    // per-chunk offsets: chunk c = tid + 256 j holds tile (or output-tile) elements c * APC
    uint64_t lin[kPermChunks], lout[kPermChunks];
    uint32_t sin[kPermChunks], sout[kPermChunks];
#pragma unroll
    for (int j = 0; j < kPermChunks; ++j) {
        const uint32_t e = (tid + (uint32_t)j * kPermThreads) * APC;
        uint64_t pi = 0, po = 0;
        uint32_t si = 0, so = 0;
        for (int b = 0; b < T; ++b)
            if ((e >> b) & 1u) {
                pi |= d.ptile[b];
                si ^= d.swbit[b];
                po |= d.pout[b];
                so ^= d.sig[b];
            }
        lin[j] = pi;
        sin[j] = si;
        lout[j] = po;
        sout[j] = so;
    }
    auto issue = [&](uint64_t t, C* buf) {
        const uint64_t base = warp_or64(((t >> lane) & 1ull) ? gin : 0ull);
#pragma unroll
        for (int j = 0; j < kPermChunks; ++j)
            if (tid + (uint32_t)j * kPermThreads < nch) cp_async16(buf + sin[j], in + (base | lin[j]));
        cp_async_commit();
    };
    uint64_t t = blockIdx.x;
    if (t >= ntiles) return;
    issue(t, buf0);
#pragma unroll 1
    for (uint32_t it = 0; t < ntiles; t += gridDim.x, ++it) {
        const uint64_t tn = t + gridDim.x;
        C* const cur = (it & 1u) ? buf1 : buf0;
        if (tn < ntiles) {
            issue(tn, (it & 1u) ? buf0 : buf1);
            cp_async_wait1();
        } else {
            cp_async_wait0();
        }
        __syncthreads();   // every thread's copies of tile t have landed
        const uint64_t obase = warp_or64(((t >> lane) & 1ull) ? gou : 0ull);
#pragma unroll
        for (int j = 0; j < kPermChunks; ++j) {
            if (tid + (uint32_t)j * kPermThreads >= nch) continue;
            C* const dst = out + (obase | lout[j]);
            if constexpr (APC == 2) {
                const C v0 = cur[sout[j]], v1 = cur[sout[j] ^ d.sig[0]];
                *reinterpret_cast<float4*>(dst) = make_float4(v0.x, v0.y, v1.x, v1.y);
            } else {
                *dst = cur[sout[j]];
            }
        }
        __syncthreads();   // this buffer is free for the copy of tile t + 2 gridDim
    }
}

cudaError_t launch_permute(int elem_bytes, const void* in, void* out, const PermDesc& d, uint64_t ntiles,
                           cudaStream_t s) {
    const size_t smem = 2 * ((size_t)elem_bytes << d.T);
    // one lane per global bit in the warp OR-reduction (tiles of 11 or 12 bits and at most
    // 40 qubits leave at most 29), and a tile of at most kPermChunks 16-byte chunks per thread
    if (d.n_glob > 32 || ((size_t)elem_bytes << d.T) > (size_t)16 * kPermThreads * kPermChunks) return cudaErrorInvalidValue;
    static int nsm[64] = {0}, per_sm[64][2] = {{0}};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const int w = elem_bytes == 8 ? 0 : 1;
    if (!per_sm[dev][w]) {
        if (!nsm[dev]) {
            e = cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return e;
        }
        const void* fn = w == 0 ? (const void*)k_permute<float2> : (const void*)k_permute<double2>;
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * (16 << 11));
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kPermThreads, 2 * (16 << 11));
        if (e != cudaSuccess) return e;
        per_sm[dev][w] = nb > 0 ? nb : 1;
    }
    const uint64_t g = (uint64_t)nsm[dev] * (uint64_t)per_sm[dev][w];
    const unsigned grid = (unsigned)(ntiles < g ? ntiles : g);
    if (w == 0)
        k_permute<float2><<<grid, kPermThreads, smem, s>>>((const float2*)in, (float2*)out, d, ntiles);
    else
        k_permute<double2><<<grid, kPermThreads, smem, s>>>((const double2*)in, (double2*)out, d, ntiles);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Pauli sweep, (P psi)_x = f (-1)^{parity(x & zmask)} psi_{x ^ xmask} with f carrying
// the coefficient, i^{#Y} and (-1)^{parity(xmask & zmask)}.  Persistent CTAs stage
// their tiles in shared memory two at a time (the next tile's copy is in flight while
// the current one is evaluated); a thread's 2^R register elements sit on the tile bits
// the host chose for the sweep's X / Y qubits, so most partners are in registers, the
// others are read from the staged tile.  lambda is written from registers: for each
// element index the lanes of a warp cover 2^L-amplitude runs.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float fmaf_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaf_t(double a, double b, double c) { return fma(a, b, c); }

// one term, read as three 16-byte words
// (complex64 sweeps read the FP32 copy of the coefficient: no FP64 conversion per term)
template <typename Real>
struct PTermR {
    uint64_t zmask;
    uint32_t xtile, flags, xreg, zreg, smask;
    Real fre, fim;
};
template <typename Real>
__device__ __forceinline__ PTermR<Real> load_term(const PauliTerm* __restrict__ t) {
    const uint4* q = reinterpret_cast<const uint4*>(t);
    const uint4 q0 = __ldg(q), q1 = __ldg(q + 1);
    PTermR<Real> r;
    r.zmask = (uint64_t)q0.x | ((uint64_t)q0.y << 32);
    r.xtile = q0.z;
    r.flags = q0.w;
    r.xreg = q1.x & 0xFFFFu;
    r.zreg = q1.x >> 16;
    r.smask = q1.y;
    if constexpr (sizeof(Real) == 4) {
        r.fre = __uint_as_float(q1.z);
        r.fim = __uint_as_float(q1.w);
    } else {
        const uint4 q2 = __ldg(q + 2);
        r.fre = __hiloint2double((int)q2.y, (int)q2.x);
        r.fim = __hiloint2double((int)q2.w, (int)q2.z);
    }
    return r;
}

// o[k] += f_k * p_k with f_k = +-(fr + i fi), the sign of element k from bit k of smask
template <typename C, typename Real, bool REAL, bool SGN>
__device__ __forceinline__ void pauli_acc(C& o, const C p, Real fr, Real fi, uint32_t smask, int k) {
    const bool nk = SGN && ((smask >> k) & 1u);
    const Real gr = nk ? -fr : fr;
    if (REAL) {
        o.x = fmaf_t(gr, p.x, o.x);
        o.y = fmaf_t(gr, p.y, o.y);
    } else {
        const Real gi = nk ? -fi : fi;
        o.x = fmaf_t(gr, p.x, fmaf_t(-gi, p.y, o.x));
        o.y = fmaf_t(gr, p.y, fmaf_t(gi, p.x, o.y));
    }
}

template <typename Real, int R, int XR, bool REAL, bool SGN>
__device__ __forceinline__ void pauli_reg_v(const typename CT<Real>::C (&a)[1 << R], typename CT<Real>::C (&o)[1 << R],
                                            Real fr, Real fi, uint32_t smask) {
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) pauli_acc<typename CT<Real>::C, Real, REAL, SGN>(o[k], a[k ^ XR], fr, fi, smask, k);
}
template <typename Real, int R, int XR>
__device__ __forceinline__ void pauli_reg(const typename CT<Real>::C (&a)[1 << R], typename CT<Real>::C (&o)[1 << R],
                                          Real fr, Real fi, uint32_t smask, bool real, bool sgn) {
    if (real) {
        if (sgn) pauli_reg_v<Real, R, XR, true, true>(a, o, fr, fi, smask);
        else pauli_reg_v<Real, R, XR, true, false>(a, o, fr, fi, smask);
    } else {
        if (sgn) pauli_reg_v<Real, R, XR, false, true>(a, o, fr, fi, smask);
        else pauli_reg_v<Real, R, XR, false, false>(a, o, fr, fi, smask);
    }
}
// partner of element k at tile index xi ^ (k << L); with no X / Y on the register bits
// (XR0) the partners sit at compile-time offsets from tb + xi
template <typename Real, int R, bool REAL, bool SGN, bool XR0>
__device__ __forceinline__ void pauli_smem_v(const typename CT<Real>::C* tb, uint32_t xi, int L,
                                             typename CT<Real>::C (&o)[1 << R], Real fr, Real fi, uint32_t smask) {
    const typename CT<Real>::C* pb = tb + xi;
#pragma unroll
    for (int k = 0; k < (1 << R); ++k)
        pauli_acc<typename CT<Real>::C, Real, REAL, SGN>(o[k], XR0 ? pb[(uint32_t)k << L] : tb[xi ^ ((uint32_t)k << L)],
                                                          fr, fi, smask, k);
}

// Diagonal run [t0, t1): real weights summed per run of equal zreg; a run on register
// bits is applied to the elements by its sign pattern (o[k] += +-w a[k]), the others
// add to the element-independent weight wconst.
template <typename Real, int R, bool TO_O>
__device__ __forceinline__ void pauli_diag(const PauliTerm* __restrict__ tl, uint32_t t0, uint32_t t1, uint64_t fix,
                                           typename CT<Real>::C (&o)[1 << R], const typename CT<Real>::C (&a)[1 << R],
                                           Real (&w)[1 << R], Real& wconst) {
    Real cacc = 0;
    for (uint32_t ti = t0; ti < t1; ++ti) {
        const PTermR<Real> pt = load_term<Real>(tl + ti);
        cacc += (__popcll(fix & pt.zmask) & 1) ? -pt.fre : pt.fre;
        if (pt.flags & PT_FLUSH) {
            if (pt.zreg == 0) {
                wconst += cacc;
            } else {
#pragma unroll
                for (int k = 0; k < (1 << R); ++k) {
                    const Real c = ((pt.smask >> k) & 1u) ? -cacc : cacc;
                    if (TO_O) {
                        o[k].x = fmaf_t(c, a[k].x, o[k].x);
                        o[k].y = fmaf_t(c, a[k].y, o[k].y);
                    } else {
                        w[k] += c;
                    }
                }
            }
            cacc = 0;
        }
    }
}

// L4: the tile's low part is 4 bits (every state of 5 or more qubits); otherwise L is
// read from the sweep (tiny states, one register bit)
// NT: threads per CTA at most (256: two CTAs per SM; 512: one, for complex128 and for
// complex64 tiles of 13 qubits)
template <typename Real, int R, bool L4, int NT>
__global__ void __launch_bounds__(NT, NT == 256 ? 2 : 1) k_pauli(
    const typename CT<Real>::C* __restrict__ psi, typename CT<Real>::C* __restrict__ lam, int accumulate,
    const PauliSweep* __restrict__ sp, const PauliTerm* __restrict__ terms, double* __restrict__ partial,
    uint64_t ntiles) {
    using C = typename CT<Real>::C;
    constexpr int K = 1 << R;
    constexpr int EPC = 16 / (int)sizeof(C);   // elements per 16-byte copy
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ PauliSweep s_sw;
    __shared__ uint64_t s_jp[16];   // physical offset of the CTA's j-th copy round
    __shared__ double s_wsum[16];
    __shared__ Real s_gc[2];        // global-bit diagonal constant of the current / next tile
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
    for (uint32_t i = tid; i < sizeof(PauliSweep) / 4; i += nthr)
        reinterpret_cast<uint32_t*>(&s_sw)[i] = reinterpret_cast<const uint32_t*>(sp)[i];
    __syncthreads();
    const PauliSweep& sw = s_sw;
    const int T = (int)sw.T, L = L4 ? 4 : (int)sw.L;
    const uint32_t telems = 1u << T;
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + telems;
    // static diagonal, [k][thread] with a fixed row stride (the widest CTA)
    constexpr uint32_t WS = NT;
    Real* wtab = reinterpret_cast<Real*>(buf1 + telems);
    auto phys = [&](uint32_t e) -> uint64_t {
        uint64_t p = 0;
        for (int b = 0; e; ++b, e >>= 1)
            if (e & 1) p |= sw.ptile[b];
        return p;
    };
    // copy rounds: chunk c = tid + j * nthr holds tile elements EPC c .. EPC c + EPC - 1
    const uint32_t rounds = (telems / EPC) / nthr;
    for (uint32_t j = tid; j < rounds; j += nthr) s_jp[j] = phys(j * nthr * EPC);
    const uint64_t ld_tid = phys(tid * EPC);
    // the thread's tile index (register bits zero) and its physical bits
    const uint32_t te = (tid & ((1u << L) - 1u)) | ((tid >> L) << (L + R));
    const uint64_t tphys = phys(te);
    const PauliTerm* __restrict__ tl = terms + sw.term_off;
    const uint32_t nterms = sw.n_terms, d0 = sw.n_dstat, d1 = d0 + sw.n_dglob, d2 = d1 + sw.n_dmix;
    {   // diagonal terms on tile bits only: the same for every tile
        Real w[K], wc = 0;
        C dummy[K];
#pragma unroll
        for (int k = 0; k < K; ++k) w[k] = 0;
        pauli_diag<Real, R, false>(tl, 0, d0, tphys, dummy, dummy, w, wc);
#pragma unroll
        for (int k = 0; k < K; ++k) wtab[k * WS + tid] = w[k] + wc;
    }
    // tile bases: the tile index's bits deposited on the global bits; the next tile of
    // this CTA by a masked add (carries run through the non-global bits set to one)
    uint64_t gmask = 0, pstep = 0, bcur = 0;
    for (uint32_t i = 0; i < sw.n_glob; ++i) {
        const uint64_t b = 1ull << sw.glob_pos[i];
        gmask |= b;
        if ((gridDim.x >> i) & 1) pstep |= b;
        if ((blockIdx.x >> i) & 1) bcur |= b;
    }
    auto next_base = [&](uint64_t b) -> uint64_t { return ((b | ~gmask) + pstep) & gmask; };
    // diagonal terms on global bits only: one constant per tile, summed by warp 0 in a
    // fixed order (lane-strided partial sums, then a shuffle tree read from lane 0)
    auto gconst = [&](uint64_t base) -> Real {
        Real v = 0;
        for (uint32_t ti = d0 + (tid & 31); ti < d1; ti += 32) {
            const PTermR<Real> pt = load_term<Real>(tl + ti);
            const Real c = pt.fre;
            v += (__popcll(base & pt.zmask) & 1) ? -c : c;
        }
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        return v;
    };
    auto issue = [&](uint64_t b, C* buf) {
        b |= ld_tid;
        for (uint32_t j = 0; j < rounds; ++j) cp_async16(buf + (tid + j * nthr) * EPC, psi + (b | s_jp[j]));
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    const bool has_gc = d1 > d0 && nthr >= 32;
    // expectation partial over the CTA's tiles: complex64 sweeps sum per tile in FP32
    // and across tiles with compensated (Kahan) FP32 sums, keeping the slow FP64
    // pipe out of the tile loop; complex128 sweeps sum in FP64
    Real esum = 0, ecomp = 0;
    uint64_t tile = blockIdx.x;
    uint64_t bnext = next_base(bcur);
    if (has_gc && tid < 32) {
        const Real v = gconst(bcur);
        if (tid == 0) s_gc[0] = v;
    }
    if (tile < ntiles) issue(bcur, buf0);
    for (uint32_t cur = 0; tile < ntiles; tile += gridDim.x, cur ^= 1u) {
        const bool more = tile + gridDim.x < ntiles;
        if (more) {
            issue(bnext, cur ? buf0 : buf1);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncthreads();
        const C* tb = cur ? buf1 : buf0;
        const uint64_t fix = bcur | tphys;
        C a[K], o[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            a[k] = tb[te | ((uint32_t)k << L)];
            o[k].x = o[k].y = 0;
        }
        Real wconst = 0;
        if (d1 > d0) {
            if (has_gc) {
                wconst = s_gc[cur];
            } else {   // fewer than 32 threads: every thread sums them
                for (uint32_t ti = d0; ti < d1; ++ti) {
                    const PTermR<Real> pt = load_term<Real>(tl + ti);
                    wconst += (__popcll(bcur & pt.zmask) & 1) ? -pt.fre : pt.fre;
                }
            }
        }
        {
            Real wnone[K];
            pauli_diag<Real, R, true>(tl, d1, d2, fix, o, a, wnone, wconst);
        }
        for (uint32_t ti = d2; ti < nterms; ++ti) {
            const PTermR<Real> pt = load_term<Real>(tl + ti);
            const bool neg = !(pt.flags & PT_NOZ) && (__popcll(fix & pt.zmask) & 1);
            const Real fr = neg ? -pt.fre : pt.fre, fi = neg ? -pt.fim : pt.fim;
            const bool real = (pt.flags & PT_REAL) != 0, sgn = pt.zreg != 0;
            if (pt.flags & PT_SMEM) {
                const uint32_t xi = te ^ pt.xtile;
                if (pt.xreg == 0) {
                    if (real) {
                        if (sgn) pauli_smem_v<Real, R, true, true, true>(tb, xi, L, o, fr, fi, pt.smask);
                        else pauli_smem_v<Real, R, true, false, true>(tb, xi, L, o, fr, fi, pt.smask);
                    } else {
                        if (sgn) pauli_smem_v<Real, R, false, true, true>(tb, xi, L, o, fr, fi, pt.smask);
                        else pauli_smem_v<Real, R, false, false, true>(tb, xi, L, o, fr, fi, pt.smask);
                    }
                } else {
                    if (real) pauli_smem_v<Real, R, true, true, false>(tb, xi, L, o, fr, fi, sgn ? pt.smask : 0u);
                    else pauli_smem_v<Real, R, false, true, false>(tb, xi, L, o, fr, fi, sgn ? pt.smask : 0u);
                }
                continue;
            }
            switch (pt.xreg) {
#define SVK_PAULI_XR(X) \
    case X:             \
        if constexpr ((X) < K) pauli_reg<Real, R, ((X) < K ? (X) : 0)>(a, o, fr, fi, pt.smask, real, sgn); \
        break;
                SVK_PAULI_XR(1) SVK_PAULI_XR(2) SVK_PAULI_XR(3) SVK_PAULI_XR(4) SVK_PAULI_XR(5)
                SVK_PAULI_XR(6) SVK_PAULI_XR(7) SVK_PAULI_XR(8) SVK_PAULI_XR(9) SVK_PAULI_XR(10)
                SVK_PAULI_XR(11) SVK_PAULI_XR(12) SVK_PAULI_XR(13) SVK_PAULI_XR(14) SVK_PAULI_XR(15)
#undef SVK_PAULI_XR
                default: break;
            }
        }
        Real e = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const Real w = wconst + wtab[k * WS + tid];
            o[k].x = fmaf_t(w, a[k].x, o[k].x);
            o[k].y = fmaf_t(w, a[k].y, o[k].y);
            e = fmaf_t(a[k].x, o[k].x, fmaf_t(a[k].y, o[k].y, e));
        }
        {
            const Real y = e - ecomp, t = esum + y;
            ecomp = (t - esum) - y;
            esum = t;
        }
        if (lam != nullptr) {
            uint64_t preg[R];
#pragma unroll
            for (int j = 0; j < R; ++j) preg[j] = sw.ptile[L + j];
            auto addr = [&](int k) -> uint64_t {
                uint64_t p = fix;
#pragma unroll
                for (int j = 0; j < R; ++j)
                    if ((k >> j) & 1) p |= preg[j];
                return p;
            };
            if (accumulate) {
                C g[K];
#pragma unroll
                for (int k = 0; k < K; ++k) g[k] = lam[addr(k)];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    o[k].x += g[k].x;
                    o[k].y += g[k].y;
                }
            }
#pragma unroll
            for (int k = 0; k < K; ++k) lam[addr(k)] = o[k];
        }
        if (has_gc && more && tid < 32) {   // the next tile's constant, published by the barrier below
            const Real v = gconst(bnext);
            if (tid == 0) s_gc[cur ^ 1u] = v;
        }
        __syncthreads();   // the buffer is refilled two tiles on
        bcur = bnext;
        bnext = next_base(bnext);
    }
    // CTA partial: thread sums in FP64, fixed-order warp and CTA reductions
    double eacc = (double)esum - (double)ecomp;
    for (int off = 16; off > 0; off >>= 1)
        if ((uint32_t)off < nthr) eacc += __shfl_xor_sync(nthr >= 32 ? 0xffffffffu : ((1u << nthr) - 1u), eacc, off);
    if ((tid & 31) == 0) s_wsum[tid >> 5] = eacc;
    __syncthreads();
    if (tid == 0) {
        double s = 0;
        for (uint32_t w = 0; w < (nthr + 31) / 32; ++w) s += s_wsum[w];
        partial[blockIdx.x] = s;
    }
}

template <typename Real, int R, bool L4, int NT>
struct PauliCfg {
    // two tile buffers and the static-diagonal table
    static size_t smem(int T) {
        return ((size_t)sizeof(typename CT<Real>::C) << (T + 1)) + (size_t)sizeof(Real) * (1u << R) * NT;
    }
    static uint32_t grid(int T, uint64_t ntiles) {
        static int per_sm[14] = {0};
        static int nsm = 0;
        if (!nsm) {
            int dev = 0, m = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev);
            // the widest tile's two buffers (the kernel's static shared memory comes on top)
            if (cudaFuncSetAttribute(k_pauli<Real, R, L4, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem(NT == 512 && sizeof(Real) == 4 ? 13 : 12)) !=
                cudaSuccess)
                return 0;
            nsm = m;
        }
        if (!per_sm[T]) {
            int nb = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pauli<Real, R, L4, NT>, 1 << (T - R), smem(T));
            per_sm[T] = nb > 0 ? nb : 1;
        }
        const uint64_t g = (uint64_t)nsm * (uint64_t)per_sm[T];
        return (uint32_t)(ntiles < g ? ntiles : g);
    }
    static cudaError_t launch(const void* psi, void* lam, bool acc, const PauliSweep& hsw, const PauliSweep* d_sweep,
                              const PauliTerm* d_terms, double* partial, uint64_t ntiles, uint32_t* grid_out,
                              cudaStream_t s) {
        using C = typename CT<Real>::C;
        const int T = (int)hsw.T;
        const uint32_t g = grid(T, ntiles);
        *grid_out = g;
        if (g == 0) return ntiles ? cudaGetLastError() : cudaSuccess;
        k_pauli<Real, R, L4, NT><<<g, 1u << (T - R), smem(T), s>>>((const C*)psi, (C*)lam, acc ? 1 : 0, d_sweep, d_terms,
                                                                partial, ntiles);
        return cudaGetLastError();
    }
};

// the kernel instance of a sweep: (R, L == 4) with R <= 4 (complex64) or 3 (complex128);
// L < 4 only with one register bit
template <typename Real, typename F>
static auto pauli_dispatch(const PauliSweep& sw, F&& f) {
    constexpr int NT = sizeof(Real) == 4 ? 256 : 512;
    if (sw.L != 4) return f(PauliCfg<Real, 1, false, NT>{});
    switch (sw.R) {
        case 1: return f(PauliCfg<Real, 1, true, NT>{});
        case 2: return f(PauliCfg<Real, 2, true, NT>{});
        default: return f(PauliCfg<Real, 3, true, NT>{});
        case 4:
            if constexpr (sizeof(Real) == 4) {
                if (sw.T == 13) return f(PauliCfg<Real, 4, true, 512>{});
                return f(PauliCfg<Real, 4, true, 256>{});
            } else {
                return f(PauliCfg<Real, 3, true, NT>{});
            }
    }
}

static bool pauli_shape_ok(int elem_bytes, const PauliSweep& sw) {
    const uint32_t rmax = elem_bytes == 8 ? 4u : 3u;
    if (sw.R < 1 || sw.R > rmax || sw.T > (elem_bytes == 8 ? 13u : 12u) || sw.L + sw.R > sw.T) return false;
    if (sw.T - sw.R > 9u) return false;
    if (elem_bytes == 8 && sw.T == 13 && sw.R != 4) return false;
    if (elem_bytes == 8 && sw.T < 13 && sw.T - sw.R > 8u) return false;
    return sw.L == 4 || sw.R == 1;
}

uint32_t pauli_grid(int elem_bytes, const PauliSweep& sw, uint64_t ntiles) {
    if (!pauli_shape_ok(elem_bytes, sw)) return 0;
    auto f = [&](auto cfg) { return decltype(cfg)::grid((int)sw.T, ntiles); };
    return elem_bytes == 8 ? pauli_dispatch<float>(sw, f) : pauli_dispatch<double>(sw, f);
}

cudaError_t launch_pauli(int elem_bytes, const void* psi, void* lam, bool accumulate, const PauliSweep& hsw,
                         const PauliSweep* d_sweep, const PauliTerm* d_terms, double* partial,
                         uint64_t ntiles, uint32_t* grid_out, cudaStream_t s) {
    if (!pauli_shape_ok(elem_bytes, hsw)) return cudaErrorInvalidValue;
    auto f = [&](auto cfg) {
        return decltype(cfg)::launch(psi, lam, accumulate, hsw, d_sweep, d_terms, partial, ntiles, grid_out, s);
    };
    return elem_bytes == 8 ? pauli_dispatch<float>(hsw, f) : pauli_dispatch<double>(hsw, f);
}

// ---------------------------------------------------------------------------
// norm: FP32 partial sums over 16 complex64 amplitudes, FP64 above that
// ---------------------------------------------------------------------------
template <typename C>
__global__ void __launch_bounds__(256) k_norm(const C* __restrict__ psi, uint64_t n_amp,
                                              double* __restrict__ partial) {
    __shared__ double ws[8];
    double acc = 0.0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    if (sizeof(C) == 8) {
        const float4* p = reinterpret_cast<const float4*>(psi);
        const uint64_t n4 = n_amp / 2;   // float4 = two amplitudes
        uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
        for (; i + 7 * stride < n4; i += 8 * stride) {
            float s = 0.f;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float4 v = p[i + u * stride];
                s += v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
            }
            acc += (double)s;
        }
        for (; i < n4; i += stride) {
            const float4 v = p[i];
            acc += (double)(v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w);
        }
        if (n_amp & 1) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                const float2 v = reinterpret_cast<const float2*>(psi)[n_amp - 1];
                acc += (double)(v.x * v.x + v.y * v.y);
            }
        }
    } else {
        const double2* p = reinterpret_cast<const double2*>(psi);
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_amp; i += stride) {
            const double2 v = p[i];
            acc += v.x * v.x + v.y * v.y;
        }
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < 8; ++w) s += ws[w];
        partial[blockIdx.x] = s;
    }
}

cudaError_t launch_norm(int elem_bytes, const void* psi, uint64_t n_amp, double* partial,
                        uint32_t* nblocks, cudaStream_t s) {
    uint64_t want = (n_amp + 4095) / 4096;
    uint32_t nb = (uint32_t)(want < 152ull * 16 ? (want ? want : 1) : 152ull * 16);
    *nblocks = nb;
    if (elem_bytes == 8) k_norm<float2><<<nb, 256, 0, s>>>((const float2*)psi, n_amp, partial);
    else k_norm<double2><<<nb, 256, 0, s>>>((const double2*)psi, n_amp, partial);
    return cudaGetLastError();
}

// psi *= sqrt(norm_before / norm_after): the norm restoration after tensor-core stages
template <typename C>
__global__ void __launch_bounds__(256) k_scale_to_norm(C* __restrict__ psi, uint64_t n_amp,
                                                       const double* __restrict__ nb, const double* __restrict__ na) {
    const double b = *nb, a = *na;
    if (!(b > 0.0) || !(a > 0.0)) return;
    const double f = sqrt(b / a);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    if (sizeof(C) == 8) {
        const float ff = (float)f;
        float4* p = reinterpret_cast<float4*>(psi);
        const uint64_t n4 = n_amp / 2;
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            float4 v = p[i];
            v.x *= ff;
            v.y *= ff;
            v.z *= ff;
            v.w *= ff;
            p[i] = v;
        }
        if ((n_amp & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
            float2* q = reinterpret_cast<float2*>(psi) + (n_amp - 1);
            q->x *= ff;
            q->y *= ff;
        }
    } else {
        double2* p = reinterpret_cast<double2*>(psi);
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_amp; i += stride) {
            double2 v = p[i];
            v.x *= f;
            v.y *= f;
            p[i] = v;
        }
    }
}

cudaError_t launch_scale_to_norm(int elem_bytes, void* psi, uint64_t n_amp, const double* norm_before,
                                 const double* norm_after, cudaStream_t s) {
    const uint64_t want = (n_amp + 2047) / 2048;
    const uint32_t nb = (uint32_t)(want < 152ull * 16 ? (want ? want : 1) : 152ull * 16);
    if (elem_bytes == 8) k_scale_to_norm<float2><<<nb, 256, 0, s>>>((float2*)psi, n_amp, norm_before, norm_after);
    else k_scale_to_norm<double2><<<nb, 256, 0, s>>>((double2*)psi, n_amp, norm_before, norm_after);
    return cudaGetLastError();
}

// out[r] = sum_i in[i * rows + r], one block per row, strided fixed-order sums and a
// fixed tree: the result does not depend on timing.
__global__ void __launch_bounds__(256) k_reduce_rows(const double* __restrict__ in, uint64_t n,
                                                     uint32_t rows, double* __restrict__ out) {
    __shared__ double sm[256];
    const uint32_t r = blockIdx.x;
    double acc = 0.0;
    for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) acc += in[i * rows + r];
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[r] = sm[0];
}

cudaError_t launch_reduce_rows(const double* in, uint64_t n, uint32_t rows, double* out,
                               cudaStream_t s) {
    if (rows == 0) return cudaSuccess;
    k_reduce_rows<<<rows, 256, 0, s>>>(in, n, rows, out);
    return cudaGetLastError();
}

template <typename C>
__global__ void k_zero_state(C* __restrict__ psi, uint64_t n_amp) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_amp; i += stride) {
        C v;
        v.x = (i == 0) ? 1 : 0;
        v.y = 0;
        psi[i] = v;
    }
}

cudaError_t launch_zero_state(int elem_bytes, void* psi, uint64_t n_amp, cudaStream_t s) {
    uint64_t want = (n_amp + 255) / 256;
    unsigned nb = (unsigned)(want < 152ull * 32 ? (want ? want : 1) : 152ull * 32);
    if (elem_bytes == 8) k_zero_state<float2><<<nb, 256, 0, s>>>((float2*)psi, n_amp);
    else k_zero_state<double2><<<nb, 256, 0, s>>>((double2*)psi, n_amp);
    return cudaGetLastError();
}

}  // namespace svk
