// jit_prelude.cuh — device helpers included by the per-stage kernels that jit.cpp
// generates and compiles at run time (NVRTC, sm_103a).  Self-contained: NVRTC gets
// this file as an in-memory header, with no CUDA headers on its include path.
//
// Complex64 amplitudes are float2 (re, im).  Phase angles are 32-bit fixed-point turns
// (angle = 2 pi k / 2^32), whose sums wrap exactly modulo 2 pi.
#pragma once

typedef unsigned int u32;
typedef unsigned long long u64;

#define SVJ_DI __device__ __forceinline__

// e^{2 pi i k / 2^32}: the turn count read as a signed fraction is already in [-pi, pi)
SVJ_DI float2 svj_expi(u32 k) {
    const float a = (float)(int)k * 1.4629180792671596e-09f;   // 2 pi / 2^32
    float s, c;
    __sincosf(a, &s, &c);
    return make_float2(c, s);
}

// a * w (complex)
SVJ_DI float2 svj_cmul(float2 a, float2 w) {
    return make_float2(fmaf(-a.y, w.y, a.x * w.x), fmaf(a.y, w.x, a.x * w.y));
}

// real 2x2 on a pair: y0 = m0 x0 + m2 x1, y1 = m4 x0 + m6 x1 (packed FP32x2)
SVJ_DI void svj_ur(float2& x0, float2& x1, float m0, float m2, float m4, float m6) {
    const float2 y0 = __ffma2_rn(make_float2(m2, m2), x1, __fmul2_rn(make_float2(m0, m0), x0));
    const float2 y1 = __ffma2_rn(make_float2(m6, m6), x1, __fmul2_rn(make_float2(m4, m4), x0));
    x0 = y0;
    x1 = y1;
}

// complex 2x2 on a pair; m = row-major (re, im) pairs
SVJ_DI void svj_u(float2& x0, float2& x1, float m0, float m1, float m2, float m3, float m4, float m5,
                  float m6, float m7) {
    float2 y0, y1;
    y0.x = fmaf(-m3, x1.y, fmaf(m2, x1.x, fmaf(-m1, x0.y, m0 * x0.x)));
    y0.y = fmaf(m3, x1.x, fmaf(m2, x1.y, fmaf(m1, x0.x, m0 * x0.y)));
    y1.x = fmaf(-m7, x1.y, fmaf(m6, x1.x, fmaf(-m5, x0.y, m4 * x0.x)));
    y1.y = fmaf(m7, x1.x, fmaf(m6, x1.y, fmaf(m5, x0.x, m4 * x0.y)));
    x0 = y0;
    x1 = y1;
}

// conditional swap (a control on a thread or global bit)
SVJ_DI void svj_cswap(bool p, float2& a, float2& b) {
    const float2 t = a;
    a = p ? b : a;
    b = p ? t : b;
}

// Im(conj(l) p), Re(conj(l) p)
SVJ_DI float svj_imc(float2 l, float2 p) { return fmaf(l.x, p.y, -l.y * p.x); }
SVJ_DI float svj_rec(float2 l, float2 p) { return fmaf(l.x, p.x, l.y * p.y); }

SVJ_DI void svj_cp_async16(void* smem, const void* gmem) {
    const u32 s = (u32)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
SVJ_DI void svj_cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
SVJ_DI void svj_cp_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
SVJ_DI void svj_cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
