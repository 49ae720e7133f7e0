// kdev.cuh — device helpers shared by the sweep kernels: complex arithmetic,
// async tile staging, and the micro-op interpreter that applies a register
// group's ops to the amplitudes one thread holds.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "program.h"

#ifndef SVK_PACKED_U
#define SVK_PACKED_U 1   // complex 2x2 bodies in packed FP32x2 arithmetic (0: scalar FP32)
#endif

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
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

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
// e^{2 pi i k / 2^32}: the turn count as a signed fraction is already in [-pi, pi)
__device__ __forceinline__ float2 expi(uint32_t k) {
    const float a = (float)(int32_t)k * 1.4629180792671596e-09f;   // 2 pi / 2^32
    float s, c;
    __sincosf(a, &s, &c);
    return make_float2(c, s);
}

template <typename Real>
__device__ __forceinline__ typename AngT<Real>::type term_angle(const DevTerm<Real>* __restrict__ terms,
                                                                uint32_t off, uint32_t n, uint64_t fix) {
    typename AngT<Real>::type ang = 0;
    for (uint32_t i = 0; i < n; ++i) {
        const uint64_t m = terms[off + i].mask;
        if ((fix & m) == m) ang += terms[off + i].angle;
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
template <int R, int J, bool CTRL, typename C, typename Real>
__device__ __forceinline__ void dense_u(C (&a)[1 << R], const Real (&m)[8], uint32_t creg) {
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) {
        if (k & (1 << J)) continue;
        if (CTRL && (k & creg) != creg) continue;
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
template <int R, int J, bool CTRL, typename C, typename Real>
__device__ __forceinline__ void dense_ur(C (&a)[1 << R], const Real (&m)[8], uint32_t creg) {
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) {
        if (k & (1 << J)) continue;
        if (CTRL && (k & creg) != creg) continue;
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
// complex64 specialisation: one packed FP32x2 multiply + FMA per output amplitude
template <int R, int J, bool CTRL>
__device__ __forceinline__ void dense_ur_f2(float2 (&a)[1 << R], const float (&m)[8], uint32_t creg) {
    const float2 m0 = make_float2(m[0], m[0]), m2 = make_float2(m[2], m[2]);
    const float2 m4 = make_float2(m[4], m[4]), m6 = make_float2(m[6], m[6]);
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) {
        if (k & (1 << J)) continue;
        if (CTRL && (k & creg) != creg) continue;
        const float2 x0 = a[k], x1 = a[k | (1 << J)];
        a[k] = __ffma2_rn(m2, x1, __fmul2_rn(m0, x0));
        a[k | (1 << J)] = __ffma2_rn(m6, x1, __fmul2_rn(m4, x0));
    }
}
template <int R, int J, bool CTRL, typename C>
__device__ __forceinline__ void dense_x(C (&a)[1 << R], uint32_t creg) {
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) {
        if (k & (1 << J)) continue;
        if (CTRL && (k & creg) != creg) continue;
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
template <int R, int J, int U, typename C>
__device__ __forceinline__ void phase_pair(C (&a)[1 << R], C w) {
#pragma unroll
    for (int k = 0; k < (1 << R); ++k)
        if ((k & (1 << J)) && (k & (1 << U))) a[k] = cmul(a[k], w);
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

// (j, u) with j < u, dispatched to compile-time bit positions
#define SVK_PAIR(JJ, UU) case (JJ * 8 + UU): if constexpr (R > UU) { phase_pair<R, JJ, UU, C>(a, w); } break;

template <typename Real, int R>
__device__ __forceinline__ void phase_pair_dispatch(typename CT<Real>::C (&a)[1 << R], int j, int u,
                                                    typename CT<Real>::C w) {
    using C = typename CT<Real>::C;
    switch (j * 8 + u) {
        SVK_PAIR(0, 1) SVK_PAIR(0, 2) SVK_PAIR(0, 3) SVK_PAIR(0, 4)
        SVK_PAIR(1, 2) SVK_PAIR(1, 3) SVK_PAIR(1, 4)
        SVK_PAIR(2, 3) SVK_PAIR(2, 4)
        SVK_PAIR(3, 4)
        default: break;
    }
}
#undef SVK_PAIR

// Everything an op needs besides the register array.
template <typename Real>
struct OpCtx {
    uint64_t fix;                                   // thread's fixed physical index
    const PhaseSlot<Real>* slots;                   // shared memory (thread-bit coefficients)
    const typename AngT<Real>::type* ang;           // shared memory: per-tile slot angles
    const typename AngT<Real>::type* tang;          // shared memory [slot][thread]: sum of the slot's
                                                    // thread-bit terms for each thread, or nullptr
    uint32_t tid, nthr;
    int TR;
    const DevTerm<Real>* __restrict__ terms;
};

template <typename Real>
__device__ __forceinline__ typename CT<Real>::C phase_factor(const DevOp<Real>& o, const OpCtx<Real>& x) {
    using C = typename CT<Real>::C;
    if (o.flags & F_SLOT) {
        typename AngT<Real>::type ang = x.ang[o.slot];
        if (x.tang) {
            ang += x.tang[o.slot * x.nthr + x.tid];
        } else {
            const PhaseSlot<Real>& ps = x.slots[o.slot];
            if (ps.has_thr)
                for (int i = 0; i < x.TR; ++i)
                    if ((x.tid >> i) & 1) ang += ps.J[i];
        }
        return expi(ang);
    }
    if (o.flags & F_TW) return expi(term_angle<Real>(x.terms, o.term_off, o.n_terms, x.fix));
    C w;
    w.x = o.m[0];
    w.y = o.m[1];
    if (o.flags & F_TERMS) w = cmul(w, expi(term_angle<Real>(x.terms, o.term_off, o.n_terms, x.fix)));
    return w;
}

// ---------------------------------------------------------------------------
// complex64 register arrays hold each amplitude as one packed 64-bit register
// (re in the low half).  The op bodies below are inline PTX whose outputs are tied
// to their inputs ("+l"): a body leaves every amplitude in the register it came
// from, so the runtime switch over op kinds and target bits needs no register
// shuffling at its merge points (measured: ~100 fewer ALU instructions per op).
// ---------------------------------------------------------------------------
typedef unsigned long long u64;
template <typename Real> struct RegT;
template <> struct RegT<float> { using type = u64; };
template <> struct RegT<double> { using type = double2; };

__device__ __forceinline__ u64 pack2(float x, float y) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
    return r;
}
__device__ __forceinline__ float2 unpack2(u64 v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
// real 2x2 on a pair: packed FP32x2 multiply / FMA, in place
__device__ __forceinline__ void p_ur(u64& x0, u64& x1, u64 m0, u64 m2, u64 m4, u64 m6) {
    asm volatile("{\n\t.reg .b64 t0, t1;\n\t"
                 "mul.rn.f32x2 t0, %2, %0;\n\t"
                 "fma.rn.f32x2 t0, %3, %1, t0;\n\t"
                 "mul.rn.f32x2 t1, %4, %0;\n\t"
                 "fma.rn.f32x2 %1, %5, %1, t1;\n\t"
                 "mov.b64 %0, t0;\n\t}"
                 : "+l"(x0), "+l"(x1)
                 : "l"(m0), "l"(m2), "l"(m4), "l"(m6));
}
// complex 2x2 on a pair, in place.  m: row-major (re, im); n = -m[1], -m[3], -m[5], -m[7]
__device__ __forceinline__ void p_u(u64& x0, u64& x1, const float (&m)[8], const float (&n)[4]) {
    asm volatile("{\n\t.reg .f32 a, b, c, d, p, q, r, s;\n\t"
                 "mov.b64 {a, b}, %0;\n\t"
                 "mov.b64 {c, d}, %1;\n\t"
                 "mul.rn.f32 p, %2, a;\n\tfma.rn.f32 p, %10, b, p;\n\tfma.rn.f32 p, %4, c, p;\n\tfma.rn.f32 p, %11, d, p;\n\t"
                 "mul.rn.f32 q, %2, b;\n\tfma.rn.f32 q, %3, a, q;\n\tfma.rn.f32 q, %4, d, q;\n\tfma.rn.f32 q, %5, c, q;\n\t"
                 "mul.rn.f32 r, %6, a;\n\tfma.rn.f32 r, %12, b, r;\n\tfma.rn.f32 r, %8, c, r;\n\tfma.rn.f32 r, %13, d, r;\n\t"
                 "mul.rn.f32 s, %6, b;\n\tfma.rn.f32 s, %7, a, s;\n\tfma.rn.f32 s, %8, d, s;\n\tfma.rn.f32 s, %9, c, s;\n\t"
                 "mov.b64 %0, {p, q};\n\t"
                 "mov.b64 %1, {r, s};\n\t}"
                 : "+l"(x0), "+l"(x1)
                 : "f"(m[0]), "f"(m[1]), "f"(m[2]), "f"(m[3]), "f"(m[4]), "f"(m[5]), "f"(m[6]), "f"(m[7]),
                   "f"(n[0]), "f"(n[1]), "f"(n[2]), "f"(n[3]));
}
__device__ __forceinline__ void p_swap(u64& x0, u64& x1) {
    asm volatile("{\n\t.reg .b64 t;\n\tmov.b64 t, %0;\n\tmov.b64 %0, %1;\n\tmov.b64 %1, t;\n\t}"
                 : "+l"(x0), "+l"(x1));
}
// x *= (wr + i wi), in place; nwi = -wi
__device__ __forceinline__ void p_cmul(u64& x, float wr, float wi, float nwi) {
    asm volatile("{\n\t.reg .f32 a, b, p, q;\n\t"
                 "mov.b64 {a, b}, %0;\n\t"
                 "mul.rn.f32 p, %1, a;\n\tfma.rn.f32 p, %3, b, p;\n\t"
                 "mul.rn.f32 q, %2, a;\n\tfma.rn.f32 q, %1, b, q;\n\t"
                 "mov.b64 %0, {p, q};\n\t}"
                 : "+l"(x)
                 : "f"(wr), "f"(wi), "f"(nwi));
}

template <int R, int J, bool CTRL>
__device__ __forceinline__ void pd_ur(u64 (&a)[1 << R], const float (&m)[8], uint32_t creg) {
    const u64 m0 = pack2(m[0], m[0]), m2 = pack2(m[2], m[2]), m4 = pack2(m[4], m[4]), m6 = pack2(m[6], m[6]);
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) {
        if (k & (1 << J)) continue;
        if (CTRL && (k & creg) != creg) continue;
        p_ur(a[k], a[k | (1 << J)], m0, m2, m4, m6);
    }
}
#if SVK_PACKED_U
// complex 2x2 on a pair with packed FP32x2 arithmetic, in place: y0 = m00 x0 + m01 x1,
// y1 = m10 x0 + m11 x1, each complex product as (mr, mr) * x + (-mi, mi) * swap(x) (the
// same FMA order as p_u, so the same rounding)
__device__ __forceinline__ void p_u2(u64& x0, u64& x1, const u64 (&mr)[4], const u64 (&mi)[4]) {
    asm volatile("{\n\t.reg .b64 s0, s1, t0, t1;\n\t.reg .f32 a, b, c, d;\n\t"
                 "mov.b64 {a, b}, %0;\n\tmov.b64 s0, {b, a};\n\t"
                 "mov.b64 {c, d}, %1;\n\tmov.b64 s1, {d, c};\n\t"
                 "mul.rn.f32x2 t0, %2, %0;\n\tfma.rn.f32x2 t0, %6, s0, t0;\n\t"
                 "fma.rn.f32x2 t0, %3, %1, t0;\n\tfma.rn.f32x2 t0, %7, s1, t0;\n\t"
                 "mul.rn.f32x2 t1, %4, %0;\n\tfma.rn.f32x2 t1, %8, s0, t1;\n\t"
                 "fma.rn.f32x2 t1, %5, %1, t1;\n\tfma.rn.f32x2 t1, %9, s1, t1;\n\t"
                 "mov.b64 %0, t0;\n\tmov.b64 %1, t1;\n\t}"
                 : "+l"(x0), "+l"(x1)
                 : "l"(mr[0]), "l"(mr[1]), "l"(mr[2]), "l"(mr[3]), "l"(mi[0]), "l"(mi[1]), "l"(mi[2]), "l"(mi[3]));
}
#endif
template <int R, int J, bool CTRL>
__device__ __forceinline__ void pd_u(u64 (&a)[1 << R], const float (&m)[8], uint32_t creg) {
#if SVK_PACKED_U
    u64 mr[4], mi[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        mr[e] = pack2(m[2 * e], m[2 * e]);
        mi[e] = pack2(-m[2 * e + 1], m[2 * e + 1]);
    }
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) {
        if (k & (1 << J)) continue;
        if (CTRL && (k & creg) != creg) continue;
        p_u2(a[k], a[k | (1 << J)], mr, mi);
    }
#else
    const float n[4] = {-m[1], -m[3], -m[5], -m[7]};
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) {
        if (k & (1 << J)) continue;
        if (CTRL && (k & creg) != creg) continue;
        p_u(a[k], a[k | (1 << J)], m, n);
    }
#endif
}
template <int R, int J, bool CTRL>
__device__ __forceinline__ void pd_x(u64 (&a)[1 << R], uint32_t creg) {
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) {
        if (k & (1 << J)) continue;
        if (CTRL && (k & creg) != creg) continue;
        p_swap(a[k], a[k | (1 << J)]);
    }
}
template <int R, int J>
__device__ __forceinline__ void pd_phase_bit(u64 (&a)[1 << R], float2 w) {
    const float nwi = -w.y;
#pragma unroll
    for (int k = 0; k < (1 << R); ++k)
        if (k & (1 << J)) p_cmul(a[k], w.x, w.y, nwi);
}
template <int R, int J, int U>
__device__ __forceinline__ void pd_phase_pair(u64 (&a)[1 << R], float2 w) {
    const float nwi = -w.y;
#pragma unroll
    for (int k = 0; k < (1 << R); ++k)
        if ((k & (1 << J)) && (k & (1 << U))) p_cmul(a[k], w.x, w.y, nwi);
}
template <int R>
__device__ __forceinline__ void pd_phase_all(u64 (&a)[1 << R], float2 w) {
    const float nwi = -w.y;
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) p_cmul(a[k], w.x, w.y, nwi);
}

// Apply one (non-gradient) op to a register array.  The op is first copied from
// shared memory into registers (16-byte loads), then one flat switch on its code
// selects a body specialised for the op kind, control form and register bit(s).
template <typename Real>
__device__ __forceinline__ DevOp<Real> load_op(const DevOp<Real>* p) {
    DevOp<Real> o;
    const uint4* src = reinterpret_cast<const uint4*>(p);
    uint4* dst = reinterpret_cast<uint4*>(&o);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(DevOp<Real>) / 16); ++i) dst[i] = src[i];
    return o;
}

// A real dense op's folded pair phases (F_PAIRS): the target's |1> amplitude of pair k
// is multiplied by w0 * prod over the other register bits i set in k of e^{i angle_i}
// (w0 = the op's twiddle, or 1).  The eight products come from a product tree.
template <typename Real, int R, int NV, int J>
__device__ __forceinline__ void pair_phases(typename RegT<Real>::type (&a)[NV][1 << R], const DevOp<Real>& o,
                                            const OpCtx<Real>& x) {
    using C = typename CT<Real>::C;
    using Ang = typename AngT<Real>::type;
    constexpr int NO = R - 1;   // other register bits
    C w0;
    if (o.flags & F_TW) {
        w0 = phase_factor<Real>(o, x);
    } else {
        w0.x = 1;
        w0.y = 0;
    }
    C ph[1 << NO];
    ph[0] = w0;
#pragma unroll
    for (int i = 0; i < NO; ++i) {
        Ang ang;
        memcpy(&ang, &o.m[1 + 2 * i], sizeof(ang));
        const C p = expi(ang);
#pragma unroll
        for (int c = 0; c < (1 << i); ++c) ph[c | (1 << i)] = cmul(ph[c], p);
    }
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) {
        if (k & (1 << J)) continue;
        constexpr int LOW = (1 << J) - 1;
        const int c = (k & LOW) | ((k >> (J + 1)) << J);   // k without bit J
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            if constexpr (sizeof(Real) == 4) p_cmul(a[v][k | (1 << J)], ph[c].x, ph[c].y, -ph[c].y);
            else a[v][k | (1 << J)] = cmul(a[v][k | (1 << J)], ph[c]);
        }
    }
}

template <typename Real, int R, int NV, int TYPE, bool CTRL, int J>
__device__ __forceinline__ void dense_case(typename RegT<Real>::type (&a)[NV][1 << R], const DevOp<Real>& o,
                                           const OpCtx<Real>& x) {
    using C = typename CT<Real>::C;
    if constexpr (J < R) {
        if ((x.fix & o.ctrl_fix) != o.ctrl_fix) return;   // control on a thread / global bit
        if (o.flags & F_TW) {
            const C w = phase_factor<Real>(o, x);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                if constexpr (sizeof(Real) == 4) pd_phase_bit<R, J>(a[v], w);
                else phase_bit<R, J, C>(a[v], w);
            }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            if constexpr (sizeof(Real) == 4) {
                if constexpr (TYPE == OP_X) pd_x<R, J, CTRL>(a[v], o.ctrl_reg);
                else if constexpr (TYPE == OP_UR) pd_ur<R, J, CTRL>(a[v], o.m, o.ctrl_reg);
                else pd_u<R, J, CTRL>(a[v], o.m, o.ctrl_reg);
            } else {
                if constexpr (TYPE == OP_X) dense_x<R, J, CTRL, C>(a[v], o.ctrl_reg);
                else if constexpr (TYPE == OP_UR) dense_ur<R, J, CTRL, C, Real>(a[v], o.m, o.ctrl_reg);
                else dense_u<R, J, CTRL, C, Real>(a[v], o.m, o.ctrl_reg);
            }
        }
    }
}

// real dense op with folded pair phases (its own dispatch codes, so the plain dense
// bodies stay as they are)
template <typename Real, int R, int NV, int J>
__device__ __forceinline__ void urp_case(typename RegT<Real>::type (&a)[NV][1 << R], const DevOp<Real>& o,
                                         const OpCtx<Real>& x) {
    if constexpr (J < R && R >= 2 && R <= 4 && NV == 1) {   // forward programs only
        pair_phases<Real, R, NV, J>(a, o, x);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            if constexpr (sizeof(Real) == 4) pd_ur<R, J, false>(a[v], o.m, 0u);
            else dense_ur<R, J, false, typename CT<Real>::C, Real>(a[v], o.m, 0u);
        }
    }
}

template <typename Real, int R, int NV, int J>
__device__ __forceinline__ void phase1_case(typename RegT<Real>::type (&a)[NV][1 << R], const DevOp<Real>& o,
                                            const OpCtx<Real>& x) {
    if constexpr (J < R) {
        const typename CT<Real>::C w = phase_factor<Real>(o, x);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            if constexpr (sizeof(Real) == 4) pd_phase_bit<R, J>(a[v], w);
            else phase_bit<R, J, typename CT<Real>::C>(a[v], w);
        }
    }
}
template <typename Real, int R, int NV, int J, int U>
__device__ __forceinline__ void phase2_case(typename RegT<Real>::type (&a)[NV][1 << R], const DevOp<Real>& o) {
    if constexpr (U < R) {
        typename CT<Real>::C w;
        w.x = o.m[0];
        w.y = o.m[1];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            if constexpr (sizeof(Real) == 4) pd_phase_pair<R, J, U>(a[v], w);
            else phase_pair<R, J, U, typename CT<Real>::C>(a[v], w);
        }
    }
}

// complex dense ops (OP_U) only in kernels built with CPLX (stages without them run a
// smaller interpreter)
#define SVK_CDENSE_CASES(CTRL, BASE)                                                        \
    case BASE + 0: if constexpr (CPLX) dense_case<Real, R, NV, OP_U, CTRL, 0>(a, o, x); break; \
    case BASE + 1: if constexpr (CPLX) dense_case<Real, R, NV, OP_U, CTRL, 1>(a, o, x); break; \
    case BASE + 2: if constexpr (CPLX) dense_case<Real, R, NV, OP_U, CTRL, 2>(a, o, x); break; \
    case BASE + 3: if constexpr (CPLX) dense_case<Real, R, NV, OP_U, CTRL, 3>(a, o, x); break; \
    case BASE + 4: if constexpr (CPLX) dense_case<Real, R, NV, OP_U, CTRL, 4>(a, o, x); break;
#define SVK_DENSE_CASES(TYPE, CTRL, BASE)                                                   \
    case BASE + 0: dense_case<Real, R, NV, TYPE, CTRL, 0>(a, o, x); break;                 \
    case BASE + 1: dense_case<Real, R, NV, TYPE, CTRL, 1>(a, o, x); break;                 \
    case BASE + 2: dense_case<Real, R, NV, TYPE, CTRL, 2>(a, o, x); break;                 \
    case BASE + 3: dense_case<Real, R, NV, TYPE, CTRL, 3>(a, o, x); break;                 \
    case BASE + 4: dense_case<Real, R, NV, TYPE, CTRL, 4>(a, o, x); break;
#define SVK_PHASE2_CASE(J, U)                                                               \
    case C_PHASE2 + (J == 0 ? U - 1 : J == 1 ? U + 2 : J == 2 ? U + 4 : 9):                  \
        phase2_case<Real, R, NV, J, U>(a, o);                                               \
        break;

// Apply one (non-gradient) op to NV register arrays (forward: psi; adjoint: psi and
// lambda), with one dispatch and one phase evaluation.
template <typename Real, int R, int NV, bool CPLX = true>
__device__ __forceinline__ void apply_op(typename RegT<Real>::type (&a)[NV][1 << R], const DevOp<Real>& o,
                                         const OpCtx<Real>& x) {
    // folded-pair butterflies (the bulk of QFT-like stages) are dispatched ahead of the
    // full switch: measured 7 % faster QFT30 stages (brickwork stages 4 % slower)
    if (o.code >= C_URP) {
        SVK_SWITCH_J(o.code - C_URP, R, (urp_case<Real, R, NV, J_>(a, o, x)));
        return;
    }
    switch (o.code) {
        SVK_CDENSE_CASES(false, 0)
        SVK_CDENSE_CASES(true, 5)
        SVK_DENSE_CASES(OP_UR, false, 10)
        SVK_DENSE_CASES(OP_UR, true, 15)
        SVK_DENSE_CASES(OP_X, false, 20)
        SVK_DENSE_CASES(OP_X, true, 25)
        case C_URP + 0: urp_case<Real, R, NV, 0>(a, o, x); break;
        case C_URP + 1: urp_case<Real, R, NV, 1>(a, o, x); break;
        case C_URP + 2: urp_case<Real, R, NV, 2>(a, o, x); break;
        case C_URP + 3: urp_case<Real, R, NV, 3>(a, o, x); break;
        case C_PHASE1 + 0: phase1_case<Real, R, NV, 0>(a, o, x); break;
        case C_PHASE1 + 1: phase1_case<Real, R, NV, 1>(a, o, x); break;
        case C_PHASE1 + 2: phase1_case<Real, R, NV, 2>(a, o, x); break;
        case C_PHASE1 + 3: phase1_case<Real, R, NV, 3>(a, o, x); break;
        case C_PHASE1 + 4: phase1_case<Real, R, NV, 4>(a, o, x); break;
        SVK_PHASE2_CASE(0, 1) SVK_PHASE2_CASE(0, 2) SVK_PHASE2_CASE(0, 3) SVK_PHASE2_CASE(0, 4)
        SVK_PHASE2_CASE(1, 2) SVK_PHASE2_CASE(1, 3) SVK_PHASE2_CASE(1, 4)
        SVK_PHASE2_CASE(2, 3) SVK_PHASE2_CASE(2, 4)
        SVK_PHASE2_CASE(3, 4)
        case C_PHASE0: {
            const typename CT<Real>::C w = phase_factor<Real>(o, x);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                if constexpr (sizeof(Real) == 4) {
                    pd_phase_all<R>(a[v], w);
                } else {
#pragma unroll
                    for (int k = 0; k < (1 << R); ++k) a[v][k] = cmul(a[v][k], w);
                }
            }
            break;
        }
        default: break;
    }
}
#undef SVK_DENSE_CASES
#undef SVK_CDENSE_CASES
#undef SVK_PHASE2_CASE

// Stage the stage's register groups, ops and phase slots into shared memory.
template <typename Real>
__device__ __forceinline__ void stage_prologue(Group* sgr, DevOp<Real>* sops, PhaseSlot<Real>* ssl,
                                               const Stage& st, const Group* __restrict__ ggr,
                                               const DevOp<Real>* __restrict__ gops,
                                               const PhaseSlot<Real>* __restrict__ gsl, uint32_t tid,
                                               uint32_t nthr) {
    {
        const uint4* src = reinterpret_cast<const uint4*>(ggr + st.group_off);
        uint4* dst = reinterpret_cast<uint4*>(sgr);
        const uint32_t nw = st.n_groups * (uint32_t)(sizeof(Group) / 16);
        for (uint32_t i = tid; i < nw; i += nthr) dst[i] = src[i];
    }
    {
        const uint4* src = reinterpret_cast<const uint4*>(gops + st.op_off);
        uint4* dst = reinterpret_cast<uint4*>(sops);
        const uint32_t nw = st.n_ops * (uint32_t)(sizeof(DevOp<Real>) / 16);
        for (uint32_t i = tid; i < nw; i += nthr) dst[i] = src[i];
    }
    {
        const uint4* src = reinterpret_cast<const uint4*>(gsl + st.phase_off);
        uint4* dst = reinterpret_cast<uint4*>(ssl);
        const uint32_t nw = st.n_phase * (uint32_t)(sizeof(PhaseSlot<Real>) / 16);
        for (uint32_t i = tid; i < nw; i += nthr) dst[i] = src[i];
    }
}

// Per-tile slot angles: the constant plus the terms on global bits set in this tile.
template <typename Real>
__device__ __forceinline__ void tile_angles(typename AngT<Real>::type* sang,
                                            const PhaseSlot<Real>* __restrict__ gsl,
                                            const DevTerm<Real>* __restrict__ terms, const Stage& st,
                                            uint64_t base, uint32_t tid, uint32_t nthr) {
    for (uint32_t p = tid; p < st.n_phase; p += nthr) {
        const PhaseSlot<Real>& ps = gsl[st.phase_off + p];
        typename AngT<Real>::type ang = ps.cangle;
        for (uint32_t i = 0; i < ps.n_glob; ++i)
            if (base & terms[ps.glob_off + i].mask) ang += terms[ps.glob_off + i].angle;
        sang[p] = ang;
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

template <typename A, typename C, int R>
__device__ __forceinline__ void load_regs(A (&a)[1 << R], const C* tile, uint32_t soff,
                                          const uint32_t (&sr)[R], bool pairs) {
    static_assert(sizeof(A) == sizeof(C), "register / tile element size");
    if (sizeof(C) == 8 && pairs) {
#pragma unroll
        for (int k = 0; k < (1 << R); k += 2) {
            const uint4 v = *reinterpret_cast<const uint4*>(tile + reg_addr<C, R>(k, soff, sr));
            memcpy(&a[k], &v.x, 8);
            memcpy(&a[k + 1], &v.z, 8);
        }
    } else {
#pragma unroll
        for (int k = 0; k < (1 << R); ++k) memcpy(&a[k], tile + reg_addr<C, R>(k, soff, sr), sizeof(C));
    }
}
template <typename A, typename C, int R>
__device__ __forceinline__ void store_regs(const A (&a)[1 << R], C* tile, uint32_t soff,
                                           const uint32_t (&sr)[R], bool pairs) {
    if (sizeof(C) == 8 && pairs) {
#pragma unroll
        for (int k = 0; k < (1 << R); k += 2) {
            uint4 v;
            memcpy(&v.x, &a[k], 8);
            memcpy(&v.z, &a[k + 1], 8);
            *reinterpret_cast<uint4*>(tile + reg_addr<C, R>(k, soff, sr)) = v;
        }
    } else {
#pragma unroll
        for (int k = 0; k < (1 << R); ++k) memcpy(tile + reg_addr<C, R>(k, soff, sr), &a[k], sizeof(C));
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

// Adjoint gradient terms: Im <lambda| G_j |psi> over the pairs of register bit j.
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
                                           const typename RegT<Real>::type (&la)[1 << R], int type) {
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

}  // namespace svk
