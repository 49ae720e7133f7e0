// kdev.cuh — device helpers shared by the sweep kernels: complex arithmetic,
// async tile staging, and the micro-op interpreter that applies a register
// group's ops to the amplitudes one thread holds.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "program.h"

namespace svk {

template <typename Real> struct CT;
template <> struct CT<float> { using C = float2; };
template <> struct CT<double> { using C = double2; };

template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) {
    C r;
    r.x = a.x * s;
    r.y = a.y * s;
    return r;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// e^{i a} with a reduced to [-pi, pi]; float uses the hardware approximation.
__device__ __forceinline__ float2 expi(float a) {
    const float inv2pi = 0.15915494309189535f, twopi = 6.283185307179586f;
    a = fmaf(-twopi, rintf(a * inv2pi), a);
    float s, c;
    __sincosf(a, &s, &c);
    return make_float2(c, s);
}
__device__ __forceinline__ double2 expi(double a) {
    double s, c;
    sincos(a, &s, &c);
    return make_double2(c, s);
}

template <typename Real>
__device__ __forceinline__ Real term_angle(const Term* __restrict__ terms, uint32_t off, uint32_t n,
                                           uint64_t fix) {
    Real ang = 0;
    for (uint32_t i = 0; i < n; ++i) {
        const uint64_t m = terms[off + i].mask;
        if ((fix & m) == m) ang += (Real)terms[off + i].angle;
    }
    return ang;
}

// tile base: global bits of the tile index deposited at their physical positions
__device__ __forceinline__ uint64_t tile_base(uint64_t tile, const uint8_t* __restrict__ glob_pos) {
    uint64_t base = 0;
    for (int i = 0; tile; ++i, tile >>= 1)
        if (tile & 1) base |= 1ull << glob_pos[i];
    return base;
}

// ---------------------------------------------------------------------------
// register-resident op application
// ---------------------------------------------------------------------------
template <int R, int J, typename C, typename Real>
__device__ __forceinline__ void dense_u(C (&a)[1 << R], const Real (&m)[8], uint32_t creg) {
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) {
        if (k & (1 << J)) continue;
        if ((k & creg) != creg) continue;
        const C x0 = a[k], x1 = a[k | (1 << J)];
        C y0, y1;
        y0.x = m[0] * x0.x - m[1] * x0.y + m[2] * x1.x - m[3] * x1.y;
        y0.y = m[0] * x0.y + m[1] * x0.x + m[2] * x1.y + m[3] * x1.x;
        y1.x = m[4] * x0.x - m[5] * x0.y + m[6] * x1.x - m[7] * x1.y;
        y1.y = m[4] * x0.y + m[5] * x0.x + m[6] * x1.y + m[7] * x1.x;
        a[k] = y0;
        a[k | (1 << J)] = y1;
    }
}
template <int R, int J, typename C, typename Real>
__device__ __forceinline__ void dense_ur(C (&a)[1 << R], const Real (&m)[8], uint32_t creg) {
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) {
        if (k & (1 << J)) continue;
        if ((k & creg) != creg) continue;
        const C x0 = a[k], x1 = a[k | (1 << J)];
        C y0, y1;
        y0.x = m[0] * x0.x + m[2] * x1.x;
        y0.y = m[0] * x0.y + m[2] * x1.y;
        y1.x = m[4] * x0.x + m[6] * x1.x;
        y1.y = m[4] * x0.y + m[6] * x1.y;
        a[k] = y0;
        a[k | (1 << J)] = y1;
    }
}
template <int R, int J, typename C>
__device__ __forceinline__ void dense_x(C (&a)[1 << R], uint32_t creg) {
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) {
        if (k & (1 << J)) continue;
        if ((k & creg) != creg) continue;
        const C t = a[k];
        a[k] = a[k | (1 << J)];
        a[k | (1 << J)] = t;
    }
}
template <int R, int J, typename C>
__device__ __forceinline__ void phase_bit(C (&a)[1 << R], C w) {
#pragma unroll
    for (int k = 0; k < (1 << R); ++k)
        if (k & (1 << J)) a[k] = cmul(a[k], w);
}

#define SVK_SWITCH_J(j, R, CALL)                          \
    switch (j) {                                          \
        case 0: { constexpr int J_ = 0; CALL; } break;     \
        case 1: if constexpr (R > 1) { constexpr int J_ = 1; CALL; } break; \
        case 2: if constexpr (R > 2) { constexpr int J_ = 2; CALL; } break; \
        case 3: if constexpr (R > 3) { constexpr int J_ = 3; CALL; } break; \
        case 4: if constexpr (R > 4) { constexpr int J_ = 4; CALL; } break; \
        default: break;                                   \
    }

// Apply one (non-gradient) op to a register array.
template <typename Real, int R>
__device__ __forceinline__ void apply_op(typename CT<Real>::C (&a)[1 << R], const Op& o, uint64_t fix,
                                         const Term* __restrict__ terms) {
    using C = typename CT<Real>::C;
    const uint8_t type = o.type;
    if (type <= OP_X) {
        if ((fix & o.ctrl_fix) != o.ctrl_fix) return;   // control on a thread / global bit
        const uint32_t creg = o.ctrl_reg;
        if (type == OP_X) {
            SVK_SWITCH_J(o.j, R, (dense_x<R, J_, C>(a, creg)));
        } else {
            Real m[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) m[i] = (Real)o.m[i];
            if (type == OP_UR) {
                SVK_SWITCH_J(o.j, R, (dense_ur<R, J_, C, Real>(a, m, creg)));
            } else {
                SVK_SWITCH_J(o.j, R, (dense_u<R, J_, C, Real>(a, m, creg)));
            }
        }
    } else if (type == OP_PHASE1) {
        C w;
        w.x = (Real)o.m[0];
        w.y = (Real)o.m[1];
        if (o.n_terms) w = cmul(w, expi(term_angle<Real>(terms, o.term_off, o.n_terms, fix)));
        SVK_SWITCH_J(o.j, R, (phase_bit<R, J_, C>(a, w)));
    } else if (type == OP_PHASE2) {
        C w;
        w.x = (Real)o.m[0];
        w.y = (Real)o.m[1];
        const uint32_t mk = (1u << o.j) | (1u << o.u);
#pragma unroll
        for (int k = 0; k < (1 << R); ++k)
            if ((k & mk) == mk) a[k] = cmul(a[k], w);
    } else if (type == OP_PHASE0) {
        C w;
        w.x = (Real)o.m[0];
        w.y = (Real)o.m[1];
        if (o.n_terms) w = cmul(w, expi(term_angle<Real>(terms, o.term_off, o.n_terms, fix)));
#pragma unroll
        for (int k = 0; k < (1 << R); ++k) a[k] = cmul(a[k], w);
    }
}

// Register <-> shared-memory transfer for a group mapping.  Element k of the thread
// lives at swizzled index soff ^ XOR_{j in k} sreg[j].
template <typename C, int R>
__device__ __forceinline__ uint32_t reg_addr(int k, uint32_t soff, const uint32_t (&sr)[R]) {
    uint32_t a = soff;
#pragma unroll
    for (int j = 0; j < R; ++j)
        if (k & (1 << j)) a ^= sr[j];
    return a;
}

template <typename C, int R>
__device__ __forceinline__ void load_regs(C (&a)[1 << R], const C* tile, uint32_t soff,
                                          const uint32_t (&sr)[R], bool pairs) {
    if (sizeof(C) == 8 && pairs) {
#pragma unroll
        for (int k = 0; k < (1 << R); k += 2) {
            const float4 v = *reinterpret_cast<const float4*>(tile + reg_addr<C, R>(k, soff, sr));
            a[k].x = v.x; a[k].y = v.y; a[k + 1].x = v.z; a[k + 1].y = v.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < (1 << R); ++k) a[k] = tile[reg_addr<C, R>(k, soff, sr)];
    }
}
template <typename C, int R>
__device__ __forceinline__ void store_regs(const C (&a)[1 << R], C* tile, uint32_t soff,
                                           const uint32_t (&sr)[R], bool pairs) {
    if (sizeof(C) == 8 && pairs) {
#pragma unroll
        for (int k = 0; k < (1 << R); k += 2) {
            float4 v;
            v.x = a[k].x; v.y = a[k].y; v.z = a[k + 1].x; v.w = a[k + 1].y;
            *reinterpret_cast<float4*>(tile + reg_addr<C, R>(k, soff, sr)) = v;
        }
    } else {
#pragma unroll
        for (int k = 0; k < (1 << R); ++k) tile[reg_addr<C, R>(k, soff, sr)] = a[k];
    }
}

// Stage a tile HBM -> shared memory (16-byte cp.async chunks, swizzled) and back.
// Chunk c = tid + i * 2^(T-R); element t = c * APC; element bit (b + log2 APC) is
// chunk bit b, so thread bits and loop bits deposit independently (XOR-linear).
template <typename C, int R>
__device__ __forceinline__ void tile_load(C* tile, const C* __restrict__ g, uint64_t base,
                                          const uint64_t* __restrict__ ptile,
                                          const uint32_t* __restrict__ swbit, int TR, uint32_t tid) {
    constexpr int APC = 16 / (int)sizeof(C);
    constexpr int LA = APC == 2 ? 1 : 0;
    constexpr int NCH = (1 << R) / APC;
    uint64_t ptid = 0;
    uint32_t stid = 0;
    for (int b = 0; b < TR; ++b)
        if ((tid >> b) & 1) {
            ptid ^= ptile[b + LA];
            stid ^= swbit[b + LA];
        }
#pragma unroll
    for (int i = 0; i < NCH; ++i) {
        uint64_t pi = 0;
        uint32_t si = 0;
#pragma unroll
        for (int b = 0; (1 << b) < NCH; ++b)
            if ((i >> b) & 1) {
                pi ^= ptile[TR + LA + b];
                si ^= swbit[TR + LA + b];
            }
        cp_async16(tile + (stid ^ si), g + (base | (ptid ^ pi)));
    }
}
template <typename C, int R>
__device__ __forceinline__ void tile_store(const C* tile, C* __restrict__ g, uint64_t base,
                                           const uint64_t* __restrict__ ptile,
                                           const uint32_t* __restrict__ swbit, int TR, uint32_t tid) {
    constexpr int APC = 16 / (int)sizeof(C);
    constexpr int LA = APC == 2 ? 1 : 0;
    constexpr int NCH = (1 << R) / APC;
    uint64_t ptid = 0;
    uint32_t stid = 0;
    for (int b = 0; b < TR; ++b)
        if ((tid >> b) & 1) {
            ptid ^= ptile[b + LA];
            stid ^= swbit[b + LA];
        }
#pragma unroll
    for (int i = 0; i < NCH; ++i) {
        uint64_t pi = 0;
        uint32_t si = 0;
#pragma unroll
        for (int b = 0; (1 << b) < NCH; ++b)
            if ((i >> b) & 1) {
                pi ^= ptile[TR + LA + b];
                si ^= swbit[TR + LA + b];
            }
        const float4 v = *reinterpret_cast<const float4*>(tile + (stid ^ si));
        *reinterpret_cast<float4*>(g + (base | (ptid ^ pi))) = v;
    }
}

}  // namespace svk
