// aux_kernels.cu — bit-permutation sweep (the on-GPU form of the inter-partition
// exchange, Sec. 4.3 "Creating the Data Reshaping Operations"), Pauli-sum sweeps for
// expectation values and the adjoint seed lambda = O psi, FP64 reductions.
#include "kdev.cuh"
#include "kernels.h"

namespace svk {

// ---------------------------------------------------------------------------
// permutation: the tile contains the input's low bits and the input bits that land
// on the output's low bits, so both the read and the write are contiguous runs.
// ---------------------------------------------------------------------------
template <typename C>
__global__ void __launch_bounds__(256) k_permute(const C* __restrict__ in, C* __restrict__ out,
                                                 const PermDesc* __restrict__ dp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tile = reinterpret_cast<C*>(smem_raw);
    const PermDesc& d = *dp;
    const int T = (int)d.T;
    constexpr int APC = 16 / (int)sizeof(C);
    const uint32_t nch = (1u << T) / APC;
    uint64_t base = 0, obase = 0;
    {
        uint64_t t = blockIdx.x;
        for (int i = 0; t; ++i, t >>= 1)
            if (t & 1) {
                base |= 1ull << d.glob_pos[i];
                obase |= d.gout[i];
            }
    }
    for (uint32_t c = threadIdx.x; c < nch; c += blockDim.x) {
        const uint32_t t = c * APC;
        uint64_t p = base;
        uint32_t sa = 0;
        for (int b = 0; b < T; ++b)
            if ((t >> b) & 1) {
                p |= d.ptile[b];
                sa ^= d.swbit[b];
            }
        cp_async16(tile + sa, in + p);
    }
    cp_async_commit_wait_all();
    __syncthreads();
    for (uint32_t c = threadIdx.x; c < nch; c += blockDim.x) {
        const uint32_t u = c * APC;
        uint64_t p = obase;
        uint32_t sa = 0;
        for (int b = 0; b < T; ++b)
            if ((u >> b) & 1) {
                p |= d.pout[b];
                sa ^= d.sig[b];
            }
        if (APC == 2) {
            const C v0 = tile[sa], v1 = tile[sa ^ d.sig[0]];
            float4 v;
            v.x = (float)v0.x; v.y = (float)v0.y; v.z = (float)v1.x; v.w = (float)v1.y;
            *reinterpret_cast<float4*>(out + p) = v;
        } else {
            out[p] = tile[sa];
        }
    }
}

cudaError_t launch_permute(int elem_bytes, const void* in, void* out, const PermDesc* d, int T,
                           uint64_t ntiles, cudaStream_t s) {
    const size_t smem = (size_t)elem_bytes << T;
    if (elem_bytes == 8) {
        static bool cfg = false;
        if (!cfg) { cudaFuncSetAttribute(k_permute<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024); cfg = true; }
        k_permute<float2><<<(unsigned)ntiles, 256, smem, s>>>((const float2*)in, (float2*)out, d);
    } else {
        static bool cfg = false;
        if (!cfg) { cudaFuncSetAttribute(k_permute<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024); cfg = true; }
        k_permute<double2><<<(unsigned)ntiles, 256, smem, s>>>((const double2*)in, (double2*)out, d);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Pauli sweep.  Thread holds 2^R consecutive tile elements (register bits = tile bits
// 0..R-1); (P psi)_x = f * (-1)^{parity((x ^ xmask) & zmask)} psi_{x ^ xmask}.
// ---------------------------------------------------------------------------
template <typename C, typename Real, int R, int XT>
__device__ __forceinline__ void pauli_reg_partner(const C (&a)[1 << R], C (&o)[1 << R], C f, int par0,
                                                  uint32_t zr) {
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) {
        C v = cmul(a[k ^ XT], f);
        if ((par0 ^ __popc(k & zr)) & 1) { v.x = -v.x; v.y = -v.y; }
        o[k].x += v.x;
        o[k].y += v.y;
    }
}

template <typename Real, int R>
__global__ void __launch_bounds__(512) k_pauli(const typename CT<Real>::C* __restrict__ psi,
                                               typename CT<Real>::C* __restrict__ lam, int accumulate,
                                               const PauliSweep* __restrict__ sp,
                                               const PauliTerm* __restrict__ terms,
                                               double* __restrict__ partial) {
    using C = typename CT<Real>::C;
    constexpr int K = 1 << R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const PauliSweep& sw = *sp;
    const int T = (int)sw.T;
    const int TR = T - R;
    C* tile = reinterpret_cast<C*>(smem_raw);
    C* tout = tile + (1u << T);
    double* wsum = reinterpret_cast<double*>(tout + (1u << T));
    const uint32_t tid = threadIdx.x;
    const uint64_t base = tile_base(blockIdx.x, sw.glob_pos);
    tile_load<C, R>(tile, psi, base, sw.ptile, sw.swbit, TR, tid);
    cp_async_commit_wait_all();
    __syncthreads();

    uint64_t fix = base;
    uint32_t soff = 0;
    for (int i = 0; i < TR; ++i)
        if ((tid >> i) & 1) {
            fix |= sw.ptile[R + i];
            soff ^= sw.swbit[R + i];
        }
    uint32_t sr[R];
#pragma unroll
    for (int j = 0; j < R; ++j) sr[j] = sw.swbit[j];
    const bool pairs = sizeof(C) == 8;   // tile bit 0 is register bit 0
    C a[K], o[K];
    load_regs<C, C, R>(a, tile, soff, sr, pairs);
#pragma unroll
    for (int k = 0; k < K; ++k) o[k].x = o[k].y = 0;
    Real wd[K];
#pragma unroll
    for (int k = 0; k < K; ++k) wd[k] = 0;
    Real wconst = 0;
    for (uint32_t ti = 0; ti < sw.n_terms; ++ti) {
        const PauliTerm& pt = terms[sw.term_off + ti];
        const int par0 = (__popcll(fix & pt.zmask) ^ __popcll(pt.xmask & pt.zmask)) & 1;
        const uint32_t zr = pt.zreg;
        if (pt.xmask == 0) {   // diagonal: a real weight per element
            const Real c = par0 ? -(Real)pt.fre : (Real)pt.fre;
            if (zr == 0) {
                wconst += c;
            } else {
#pragma unroll
                for (int k = 0; k < K; ++k) wd[k] += (__popc(k & zr) & 1) ? -c : c;
            }
            continue;
        }
        const uint32_t xt = pt.xtile;
        C f;
        f.x = (Real)pt.fre;
        f.y = (Real)pt.fim;
        if (xt == 1) {
            pauli_reg_partner<C, Real, R, 1>(a, o, f, par0, zr);
        } else if (R > 1 && xt == 2) {
            pauli_reg_partner<C, Real, R, (R > 1 ? 2 : 0)>(a, o, f, par0, zr);
        } else if (R > 2 && xt == 4) {
            pauli_reg_partner<C, Real, R, (R > 2 ? 4 : 0)>(a, o, f, par0, zr);
        } else if (R > 3 && xt == 8) {
            pauli_reg_partner<C, Real, R, (R > 3 ? 8 : 0)>(a, o, f, par0, zr);
        } else {
            uint32_t sx = 0;
            for (int b = 0; b < T; ++b)
                if ((xt >> b) & 1) sx ^= sw.swbit[b];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                C v = cmul(tile[reg_addr<C, R>(k, soff, sr) ^ sx], f);
                if ((par0 ^ __popc(k & zr)) & 1) { v.x = -v.x; v.y = -v.y; }
                o[k].x += v.x;
                o[k].y += v.y;
            }
        }
    }
    Real e = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const Real w = wd[k] + wconst;
        o[k].x += w * a[k].x;
        o[k].y += w * a[k].y;
        e += a[k].x * o[k].x + a[k].y * o[k].y;
    }
    // expectation partial: FP32 over the thread's 2^R elements, FP64 above, fixed order
    double ev = (double)e;
    const uint32_t wmask = blockDim.x >= 32 ? 0xffffffffu : ((1u << blockDim.x) - 1u);
    for (int off = 16; off > 0; off >>= 1)
        if ((uint32_t)off < blockDim.x) ev += __shfl_xor_sync(wmask, ev, off);
    if (lam != nullptr) store_regs<C, C, R>(o, tout, soff, sr, pairs);
    if ((tid & 31) == 0) wsum[tid >> 5] = ev;
    __syncthreads();
    if (tid == 0) {
        double s = 0;
        for (uint32_t w = 0; w < (blockDim.x + 31) / 32; ++w) s += wsum[w];
        partial[blockIdx.x] = s;
    }
    if (lam != nullptr) {
        constexpr int APC = 16 / (int)sizeof(C);
        constexpr int LA = APC == 2 ? 1 : 0;
        constexpr int NCH = K / APC;
        uint64_t ptid = 0;
        uint32_t stid = 0;
        for (int b = 0; b < TR; ++b)
            if ((tid >> b) & 1) {
                ptid ^= sw.ptile[b + LA];
                stid ^= sw.swbit[b + LA];
            }
#pragma unroll
        for (int i = 0; i < NCH; ++i) {
            uint64_t pi = 0;
            uint32_t si = 0;
#pragma unroll
            for (int b = 0; (1 << b) < NCH; ++b)
                if ((i >> b) & 1) {
                    pi ^= sw.ptile[TR + LA + b];
                    si ^= sw.swbit[TR + LA + b];
                }
            float4 v = *reinterpret_cast<const float4*>(tout + (stid ^ si));
            float4* gp = reinterpret_cast<float4*>(lam + (base | (ptid ^ pi)));
            if (accumulate) {
                if (sizeof(C) == 8) {
                    const float4 g = *gp;
                    v.x += g.x; v.y += g.y; v.z += g.z; v.w += g.w;
                } else {
                    double2 vd = *reinterpret_cast<double2*>(&v);
                    const double2 g = *reinterpret_cast<const double2*>(gp);
                    vd.x += g.x; vd.y += g.y;
                    v = *reinterpret_cast<float4*>(&vd);
                }
            }
            *gp = v;
        }
    }
}

template <typename Real, int R>
static cudaError_t launch_pauli_R(const void* psi, void* lam, bool acc, const PauliSweep* d_sweep,
                                  const PauliTerm* d_terms, double* partial, int T, uint64_t ntiles,
                                  cudaStream_t s) {
    using C = typename CT<Real>::C;
    const uint32_t nthr = 1u << (T - R);
    const size_t smem = ((size_t)sizeof(C) << (T + 1)) + ((nthr + 31) / 32) * sizeof(double);
    static bool cfg = false;
    if (!cfg) {
        cudaError_t e = cudaFuncSetAttribute(k_pauli<Real, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        cfg = true;
    }
    k_pauli<Real, R><<<(unsigned)ntiles, nthr, smem, s>>>((const C*)psi, (C*)lam, acc ? 1 : 0, d_sweep,
                                                          d_terms, partial);
    return cudaGetLastError();
}

cudaError_t launch_pauli(int elem_bytes, int R, const void* psi, void* lam, bool accumulate,
                         const PauliSweep* d_sweep, const PauliTerm* d_terms, double* partial, int T,
                         uint64_t ntiles, cudaStream_t s) {
    if (elem_bytes == 8) {
        switch (R) {
            case 1: return launch_pauli_R<float, 1>(psi, lam, accumulate, d_sweep, d_terms, partial, T, ntiles, s);
            case 2: return launch_pauli_R<float, 2>(psi, lam, accumulate, d_sweep, d_terms, partial, T, ntiles, s);
            case 3: return launch_pauli_R<float, 3>(psi, lam, accumulate, d_sweep, d_terms, partial, T, ntiles, s);
            case 4: return launch_pauli_R<float, 4>(psi, lam, accumulate, d_sweep, d_terms, partial, T, ntiles, s);
        }
    } else {
        switch (R) {
            case 1: return launch_pauli_R<double, 1>(psi, lam, accumulate, d_sweep, d_terms, partial, T, ntiles, s);
            case 2: return launch_pauli_R<double, 2>(psi, lam, accumulate, d_sweep, d_terms, partial, T, ntiles, s);
            case 3: return launch_pauli_R<double, 3>(psi, lam, accumulate, d_sweep, d_terms, partial, T, ntiles, s);
            case 4: return launch_pauli_R<double, 4>(psi, lam, accumulate, d_sweep, d_terms, partial, T, ntiles, s);
        }
    }
    return cudaErrorInvalidValue;
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
