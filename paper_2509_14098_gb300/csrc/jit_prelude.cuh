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

// Hadamard butterfly without its factor: (x0, x1) -> (x0 + x1, x0 - x1) (packed FP32x2)
SVJ_DI void svj_hb(float2& x0, float2& x1) {
    const float2 y0 = __ffma2_rn(make_float2(1.f, 1.f), x1, x0);
    const float2 y1 = __ffma2_rn(make_float2(-1.f, -1.f), x1, x0);
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

// acc + (l.x p.x, l.y p.y): Re(conj(l) p) summed in packed FP32x2 halves
SVJ_DI float2 svj_rec2(float2 acc, float2 l, float2 p) { return __ffma2_rn(l, p, acc); }

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

// ---------------------------------------------------------------------------
// Tensor-memory-access (TMA) tile staging.  A stage's tile is one 5-D box of the state
// viewed as a tensor whose dimensions are the runs of consecutive local / global
// physical bits (local runs are box extents, global runs have box extent 1); the
// innermost dimension is physical bits 0..3 (128 bytes), loaded with the 128-byte
// swizzle, so tile element e sits at e ^ (((e >> 4) & 7) << 1).
// ---------------------------------------------------------------------------
struct alignas(64) SvjTmap { u64 w[16]; };   // CUtensorMap, filled by the host

SVJ_DI u32 svj_saddr(const void* p) { return (u32)__cvta_generic_to_shared(p); }
SVJ_DI void svj_mbar_init(u64* bar, u32 count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(svj_saddr(bar)), "r"(count) : "memory");
}
// make the initialised barriers visible to the asynchronous (TMA) proxy
SVJ_DI void svj_fence_barrier_init() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
SVJ_DI void svj_mbar_expect_tx(u64* bar, u32 bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(svj_saddr(bar)), "r"(bytes) : "memory");
}
SVJ_DI bool svj_mbar_try_wait(u64* bar, u32 parity) {
    u32 ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
                 : "=r"(ok)
                 : "r"(svj_saddr(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
// bounded wait on a barrier phase: false (and *flag set) if it did not complete within
// 2^22 polls (a few seconds at most); the caller stops and the host reports SV_ERR_TIMEOUT
SVJ_DI bool svj_mbar_wait(u64* bar, u32 parity, int* flag) {
    for (u32 i = 0; i < (1u << 22); ++i)
        if (svj_mbar_try_wait(bar, parity)) return true;
    if (flag) atomicExch(flag, 1);
    return false;
}
SVJ_DI void svj_tma_load(void* dst, const SvjTmap* map, int c0, int c1, int c2, int c3, int c4, u64* bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], [%7];\n" ::"r"(
            svj_saddr(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(svj_saddr(bar))
        : "memory");
}
SVJ_DI void svj_tma_store(const SvjTmap* map, int c0, int c1, int c2, int c3, int c4, const void* src) {
    asm volatile("cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4, %5}], [%6];\n" ::"l"(map),
                 "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(svj_saddr(src))
                 : "memory");
}
SVJ_DI void svj_bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
SVJ_DI void svj_bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
SVJ_DI void svj_bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
// generic-proxy shared-memory writes become visible to a following TMA store
SVJ_DI void svj_fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
