// jit.cpp — generator, NVRTC compiler cache and launcher of the per-stage sweep
// kernels (complex64).  See jit.h.
//
// A generated kernel is the stage sweep of Sec. 4.3 with one partition compiled in:
// persistent CTAs walk the stage's tiles (2^T amplitudes whose local bits vary, the
// lowest physical bits always among them, so every HBM access is a run of >= 128 B),
// stage each tile into shared memory with 16-byte cp.async copies, run the register
// groups (the partitioner re-run with the register budget: each thread holds 2^R
// amplitudes in registers, applies the group's gates as straight-line code, and
// exchanges through the swizzled shared-memory tile between groups), and write the
// tile back in place.  The adjoint variant carries psi and lambda together and
// accumulates Im <lambda|G|psi> per parametric rotation: a warp's sum over one tile in
// FP32, added in FP64 to that warp's per-CTA slot sum across tiles.
#include "jit.h"

#include <cuda.h>   // tensor-map types (the encoder is looked up at run time)
#include <nvrtc.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "kernels.h"
#include "jit_prelude_inc.h"   // kJitPrelude: jit_prelude.cuh as a string (generated by the build)

namespace svj {

struct Kernel {
    std::vector<char> cubin;   // NVRTC output (sm_103a)
    std::string err;
    std::mutex mu;             // guards the lazy load below
    cudaLibrary_t lib = nullptr;
    cudaKernel_t fn = nullptr;
    int per_sm_dev = -1;       // occupancy, cached for the device it was computed on
    int dev = -1;
    uint32_t smem_set = 0;
};

namespace {

// argument block layout (generated struct Args): m0 @0, m1 @128 (CUtensorMap, 64-byte
// aligned), v0 @256, v1 @264, partial @272, flag @280, params @288, pofs @296,
// ncirc @304, q[] @312
constexpr size_t kArgV0 = 256, kArgV1 = 264, kArgPartial = 272, kArgFlag = 280, kArgParams = 288, kArgPofs = 296,
                 kArgNcirc = 304, kArgQ = 312;

std::mutex g_mu;
std::unordered_map<std::string, Kernel*> g_cache;   // source -> kernel (never freed: process lifetime)
std::atomic<uint64_t> g_compiles{0}, g_hits{0};
std::atomic<uint64_t> g_compile_us{0};

// Set while a stage of an already-generated structure is re-walked to fill only its
// argument block: the source text is not needed then, so formatting is skipped.
thread_local bool g_quiet = false;

std::string fmt(const char* f, ...) {
    if (g_quiet) return std::string();
    char buf[1024];
    va_list ap;
    va_start(ap, f);
    vsnprintf(buf, sizeof(buf), f, ap);
    va_end(ap);
    return buf;
}

uint64_t fnv1a(const std::string& s) {
    uint64_t h = 1469598103934665603ull;
    for (unsigned char c : s) {
        h ^= c;
        h *= 1099511628211ull;
    }
    return h;
}

// ---------------------------------------------------------------------------
// argument block: value arrays filled while generating, laid out after the pointers
// ---------------------------------------------------------------------------
struct ArgBuilder {
    std::vector<uint64_t> q;   // 8-byte values (masks, physical bit values)
    std::vector<uint32_t> u;   // 4-byte values (angles in turns, counts)
    std::vector<float> f;      // FP32 constants (matrices, phase factors)
    int Q(uint64_t v) { q.push_back(v); return (int)q.size() - 1; }
    int U(uint32_t v) { u.push_back(v); return (int)u.size() - 1; }
    int F(float v) { f.push_back(v); return (int)f.size() - 1; }
};

struct Run { int start, len; bool local; };

// TMA eligibility of a stage: the tile holds physical bits 0..3 and is at least 1 KiB
// (the 128-byte swizzle repeats every 1 KiB), and the runs of local / global physical bits
// (local runs cut into pieces of at most 8 bits, the first piece exactly bits 0..3, global
// runs of at most 32 bits) form at most 5 dimensions.  SVGB_JIT_TMA=0 disables it.
bool tma_runs(const svk::Stage& st, int n, int nv, std::vector<Run>* dims) {
    dims->clear();
    const int T = (int)st.T;
    uint64_t tmask = 0;
    for (int b = 0; b < T; ++b) tmask |= 1ull << st.tile_pos[b];
    bool ok = n > T && T >= 7 && (tmask & 15ull) == 15ull;
    for (int b = 0; ok && b < n;) {
        const bool loc = (tmask >> b) & 1;
        int e = b;
        while (e < n && (((tmask >> e) & 1) != 0) == loc) ++e;
        if (loc) {
            for (int x = b; x < e;) {
                const int len = (x == 0) ? 4 : std::min(8, e - x);
                dims->push_back({x, len, true});
                x += len;
            }
        } else {
            if (e - b > 32) ok = false;
            dims->push_back({b, e - b, false});
        }
        b = e;
    }
    if ((int)dims->size() > 5) ok = false;
    // measured: the second ring slot costs the forward sweep more resident CTAs than the
    // overlap gains (QFT30 26.5 -> 27.7 ms), while the adjoint gains about 4 %
    bool want = nv == 2;
    if (const char* e = getenv("SVGB_JIT_TMA")) want = atoi(e) != 0;
    return ok && want;
}

// An uncontrolled real 2x2 of the form c [[1, 1], [1, -1]] (the Hadamard): a forward
// stage applies it as the butterfly (x0 + x1, x0 - x1) and multiplies the product of
// the factors c into every amplitude once, at the end of the stage
bool h_like(const svk::DevOp<float>& o) {
    return o.type == svk::OP_UR && !(o.flags & svk::F_BIND) && o.ctrl_fix == 0 && o.ctrl_reg == 0 && o.m[0] != 0.f &&
           o.m[2] == o.m[0] && o.m[4] == o.m[0] && o.m[6] == -o.m[0];
}

class Gen {
  public:
    Gen(const StageView& v, Built* out) : V(v), st(*v.st), B(out) {}
    std::string run();

  private:
    const StageView& V;
    const svk::Stage& st;
    Built* B;
    ArgBuilder A;
    std::string s;            // kernel body
    int T = 0, R = 0, TR = 0, NT = 0, NV = 1, NB = 1, NPH = 0, NSL = 0, NW = 1;
    bool ttab = false;        // per-(slot, thread) thread-bit angle table in shared memory
    bool cbank = false;       // per-op constants read from the parameter bank (else shared memory)
    bool tma = false;         // tiles staged by TMA (128-byte swizzle) instead of cp.async (software swizzle)
    bool hdefer = false;      // Hadamard-like ops as butterflies, their factor applied once per stage
    double hscale = 1.0;      // product of the deferred factors
    int NS = 2;               // TMA ring slots (set in run())
    uint32_t swz(uint32_t e) const { return tma ? (e ^ (((e >> 4) & 7u) << 1)) : svk::swizzle8(e); }
    std::vector<std::vector<int>> tbo;   // per group: tile bit of each thread bit
    int BM = 0, ZI = 0;       // batched over circuits; first stage starts from |0...0>
    struct Bind { int fi, type, kind, param; };
    std::vector<Bind> binds;  // batched: bound ops whose constants the kernel forms per circuit
    std::vector<int> slot_thr;   // per phase slot: first u[] index of its J[i] (or -1)
    int perm[32];             // logical register index -> variable holding it
    std::string fixvar;       // name of the current group's fixed-index variable ("" = none)
    std::vector<std::pair<std::string, uint32_t>> pend;   // deferred gradient partials: variable, slot
    int ngvar = 0;            // deferred partials named so far (unique names)
    int zgen = -1;            // Im(conj(lambda_r) psi_r) per register r is held in zi<zgen>_<r> (-1: none valid)
    int nzgen = 0;
    int nred = 0;             // reductions emitted so far (unique names)
    std::string reduce_pending();

    void emit(const std::string& x) { s += x; }
    std::string amp(int v, int k) const { return fmt("%c%d", v ? 'l' : 'p', perm[k]); }
    std::string slot_angle(uint32_t slot);
    std::string term_angle(const svk::DevOp<float>& o);
    std::string phase_factor(const svk::DevOp<float>& o, int gi);
    std::string fix_pred(uint64_t mask, bool all);
    std::string op(const svk::DevOp<float>& o, int gi);
    std::string dense(const svk::DevOp<float>& o, int gi);
    std::string grad(const svk::DevOp<float>& o);
};

std::string Gen::slot_angle(uint32_t slot) {
    std::string a = fmt("sang[%u]", slot);
    if (slot_thr[slot] < 0) return a;
    if (ttab) return a + fmt(" + tang[%u * %d + tid]", slot, NT);
    std::string r = "(" + a;
    for (int i = 0; i < TR; ++i) r += fmt(" + ((tid >> %d) & 1u ? S.u[%d] : 0u)", i, slot_thr[slot] + i);
    return r + ")";
}

// sum of an op's terms (masks on the thread's fixed physical index) in turns
std::string Gen::term_angle(const svk::DevOp<float>& o) {
    std::string r = "0u";
    for (uint32_t i = 0; i < o.n_terms; ++i) {
        const svk::DevTerm<float>& t = V.terms[o.term_off + i];
        const int ia = A.U(t.angle);
        if (t.mask == 0) {
            r += fmt(" + S.u[%d]", ia);
        } else {
            const int im = A.Q(t.mask);
            r += fmt(" + ((%s & S.q[%d]) == S.q[%d] ? S.u[%d] : 0u)", fixvar.c_str(), im, im, ia);
        }
    }
    return r;
}

// expression of an op's phase factor (float2)
std::string Gen::phase_factor(const svk::DevOp<float>& o, int gi) {
    (void)gi;
    if (o.flags & svk::F_SLOT) return "svj_expi(" + slot_angle(o.slot) + ")";
    if (o.flags & svk::F_TW) return "svj_expi(" + term_angle(o) + ")";
    const int c = A.F(o.m[0]);
    A.F(o.m[1]);
    std::string w = fmt("make_float2(S.f[%d], S.f[%d])", c, c + 1);
    if (o.flags & svk::F_TERMS) w = "svj_cmul(" + w + ", svj_expi(" + term_angle(o) + "))";
    return w;
}

std::string Gen::fix_pred(uint64_t mask, bool all) {
    const int im = A.Q(mask);
    return all ? fmt("((%s & S.q[%d]) == S.q[%d])", fixvar.c_str(), im, im)
               : fmt("((%s & S.q[%d]) != 0ull)", fixvar.c_str(), im);
}

std::string Gen::dense(const svk::DevOp<float>& o, int gi) {
    const int j = o.j, bj = 1 << j, K = 1 << R;
    zgen = -1;   // psi and lambda change: the shared Z-gradient products are stale
    std::string r = "{\n";
    const bool pred = o.ctrl_fix != 0;
    if (pred) r += "if " + fix_pred(o.ctrl_fix, true) + " {\n";
    auto selected = [&](int k) { return !(k & bj) && ((uint32_t)k & o.ctrl_reg) == o.ctrl_reg; };
    // phase on the target's |1> half first (the pending diagonal terms on the target)
    if (o.flags & svk::F_PAIRS) {
        // pair phases: the |1> amplitude of pair c (the other register bits) gets
        // w0 * P[c], P[c] = exp(i * sum of the angles of the other bits set in c)
        uint32_t ang[4] = {0, 0, 0, 0};
        for (int i = 0; i < R - 1 && i < 3; ++i) std::memcpy(&ang[i], &o.m[1 + 2 * i], 4);
        const bool tw = (o.flags & svk::F_TW) != 0;
        if (tw) r += "const float2 w0 = " + phase_factor(o, gi) + ";\n";
        for (int k = 0; k < K; ++k) {
            if (!selected(k)) continue;
            const int c = (k & (bj - 1)) | ((k >> (j + 1)) << j);
            uint32_t t = 0;
            for (int i = 0; i < R - 1; ++i)
                if ((c >> i) & 1) t += ang[i];
            if (c == 0 && !tw) continue;   // (no other register bit set: no pair phase)
            std::string ph;
            if (c == 0) {
                ph = "w0";
            } else {
                const double rad = (double)t * (2.0 * M_PI / 4294967296.0);
                const int fi = A.F((float)std::cos(rad));
                A.F((float)std::sin(rad));
                ph = fmt("make_float2(S.f[%d], S.f[%d])", fi, fi + 1);
                if (tw) ph = "svj_cmul(w0, " + ph + ")";
            }
            for (int v = 0; v < NV; ++v) r += fmt("%s = svj_cmul(%s, %s);\n", amp(v, k | bj).c_str(), amp(v, k | bj).c_str(), ph.c_str());
        }
    } else if (o.flags & svk::F_TW) {
        r += "const float2 w0 = " + phase_factor(o, gi) + ";\n";
        for (int k = 0; k < K; ++k)
            if (selected(k))
                for (int v = 0; v < NV; ++v) r += fmt("%s = svj_cmul(%s, w0);\n", amp(v, k | bj).c_str(), amp(v, k | bj).c_str());
    }
    if (o.type == svk::OP_X) {
        for (int k = 0; k < K; ++k) {
            if (!selected(k)) continue;
            if (pred) {
                for (int v = 0; v < NV; ++v) r += fmt("svj_cswap(true, %s, %s);\n", amp(v, k).c_str(), amp(v, k | bj).c_str());
            } else {
                std::swap(perm[k], perm[k | bj]);   // a relabel of registers: no instruction
            }
        }
    } else if (o.type == svk::OP_UR && hdefer && h_like(o)) {
        hscale *= (double)o.m[0];
        for (int k = 0; k < K; ++k)
            if (selected(k)) r += fmt("svj_hb(%s, %s);\n", amp(0, k).c_str(), amp(0, k | bj).c_str());
    } else if (o.type == svk::OP_UR) {
        const int m0 = A.F(o.m[0]), m2 = A.F(o.m[2]), m4 = A.F(o.m[4]), m6 = A.F(o.m[6]);
        if (o.flags & svk::F_BIND) binds.push_back({m0, svk::OP_UR, o.u, (int)o.term_off});
        for (int k = 0; k < K; ++k)
            if (selected(k))
                for (int v = 0; v < NV; ++v)
                    r += fmt("svj_ur(%s, %s, S.f[%d], S.f[%d], S.f[%d], S.f[%d]);\n", amp(v, k).c_str(),
                             amp(v, k | bj).c_str(), m0, m2, m4, m6);
    } else {   // OP_U
        int m[8];
        for (int i = 0; i < 8; ++i) m[i] = A.F(o.m[i]);
        if (o.flags & svk::F_BIND) binds.push_back({m[0], svk::OP_U, o.u, (int)o.term_off});
        for (int k = 0; k < K; ++k)
            if (selected(k))
                for (int v = 0; v < NV; ++v)
                    r += fmt("svj_u(%s, %s, S.f[%d], S.f[%d], S.f[%d], S.f[%d], S.f[%d], S.f[%d], S.f[%d], S.f[%d]);\n",
                             amp(v, k).c_str(), amp(v, k | bj).c_str(), m[0], m[1], m[2], m[3], m[4], m[5], m[6], m[7]);
    }
    if (pred) r += "}\n";
    return r + "}\n";
}

std::string Gen::grad(const svk::DevOp<float>& o) {
    const int K = 1 << R;
    // full warps: the partial stays in a register until the group's end, where all of
    // the group's gradient partials are reduced across the warp together
    const bool defer = NT >= 32;
    std::string r;
    if (defer && pend.size() == 32) r += reduce_pending();   // at most 32 values per reduction
    const std::string acc = defer ? fmt("ga%d", ngvar++) : std::string("acc");
    r += defer ? "float " + acc + " = 0.f;\n{\n" : "{\nfloat acc = 0.f;\n";
    const char* A_ = acc.c_str();
    if (o.type == svk::OP_GRAD_Z) {
        // Im(conj(lambda_k) psi_k) per amplitude; diagonal ops multiply psi_k and lambda_k by
        // the same phase, which cancels here, so the products stay valid until a dense op
        // and consecutive Z gradients share them (register r's product in zi<g>_<r>)
        if (zgen < 0) {
            zgen = nzgen++;
            std::string d = "";
            for (int k = 0; k < K; ++k)
                d += fmt("const float zi%d_%d = svj_imc(%s, %s);\n", zgen, perm[k], amp(1, k).c_str(), amp(0, k).c_str());
            r = d + r;
        }
        std::string sum;
        for (int k = 0; k < K; ++k) {
            const bool neg = !o.u && ((k >> o.j) & 1);
            sum += fmt("%c zi%d_%d", k == 0 ? (neg ? '-' : ' ') : (neg ? '-' : '+'), zgen, perm[k]);
        }
        r += fmt("%s = %s;\n", A_, sum.c_str());
        if (o.u) r += "if " + fix_pred(o.ctrl_fix, false) + fmt(" %s = -%s;\n", A_, A_);   // Z on a non-register bit
    } else if (o.type == svk::OP_GRAD_Y) {   // Y|0> = i|1>, Y|1> = -i|0>: Re(conj(l1) p0) - Re(conj(l0) p1), packed
        const int bj = 1 << o.j;
        r += "float2 yp = make_float2(0.f, 0.f), ym = make_float2(0.f, 0.f);\n";
        for (int k = 0; k < K; ++k) {
            if (k & bj) continue;
            const int k1 = k | bj;
            r += fmt("yp = svj_rec2(yp, %s, %s);\nym = svj_rec2(ym, %s, %s);\n", amp(1, k1).c_str(), amp(0, k).c_str(),
                     amp(1, k).c_str(), amp(0, k1).c_str());
        }
        r += fmt("%s = (yp.x + yp.y) - (ym.x + ym.y);\n", A_);
    } else {
        const int bj = 1 << o.j;
        for (int k = 0; k < K; ++k) {
            if (k & bj) continue;
            const int k1 = k | bj;
            r += fmt("%s += svj_imc(%s, %s) + svj_imc(%s, %s);\n", A_, amp(1, k).c_str(), amp(0, k1).c_str(),
                     amp(1, k1).c_str(), amp(0, k).c_str());   // X
        }
    }
    if (defer) {
        pend.push_back({acc, o.slot});
        return r + "}\n";
    }
    for (int off = 16; off > 0; off >>= 1)
        if (off < NT) r += fmt("acc += __shfl_xor_sync(%s, acc, %d);\n", NT >= 32 ? "0xffffffffu" : fmt("0x%xu", (1u << NT) - 1u).c_str(), off);
    r += fmt("if ((tid & 31u) == 0u) gsm[%u * %d + (tid >> 5)] += (double)acc;\n}\n", o.slot, NW);
    return r;
}

// The group's m gradient partials (one per lane and op) summed over the warp together:
// a butterfly reduce-scatter halves the set at each of the first log2(m) exchange
// steps (a lane keeps the half its lane bit selects and adds its partner's copy), the
// remaining steps finish the sum; value i then sits in the lanes whose upper bits
// spell i, and one of them adds it in FP64 to the warp's slot sum.
std::string Gen::reduce_pending() {
    const int m = (int)pend.size();
    if (m == 0) return "";
    int P2 = 1;
    while (P2 < m) P2 <<= 1;
    const int id = nred++;
    std::string r = "{\n";
    std::vector<std::string> v(P2);
    for (int i = 0; i < P2; ++i) v[i] = i < m ? pend[i].first : std::string("0.f");
    r += "const u32 lane = tid & 31u;\n";
    int cnt = P2, step = 0;
    for (int off = 16; off > 0; off >>= 1) {
        if (cnt > 1) {
            const int h = cnt / 2;
            for (int i = 0; i < h; ++i) {
                const std::string nv = fmt("gr%d_%d_%d", id, step, i);
                r += fmt("const float %s = ((lane & %du) ? %s : %s) + __shfl_xor_sync(0xffffffffu, (lane & %du) ? %s : %s, %d);\n",
                         nv.c_str(), off, v[i + h].c_str(), v[i].c_str(), off, v[i].c_str(), v[i + h].c_str(), off);
                v[i] = nv;
            }
            cnt = h;
        } else {
            const std::string nv = fmt("gr%d_%d_0", id, step);
            r += fmt("const float %s = %s + __shfl_xor_sync(0xffffffffu, %s, %d);\n", nv.c_str(), v[0].c_str(), v[0].c_str(), off);
            v[0] = nv;
        }
        ++step;
    }
    // value index of this lane: the lane bits of the halving steps, highest first
    int lg = 0;
    while ((1 << lg) < P2) ++lg;
    r += fmt("const u32 gi = lane >> %d;\n", 5 - lg);
    r += fmt("if ((lane & %uu) == 0u && gi < %du) {\nu32 sl = 0u;\n", (1u << (5 - lg)) - 1u, m);
    for (int i = 0; i < m; ++i) r += fmt("sl = gi == %du ? %uu : sl;\n", i, pend[i].second);
    r += fmt("gsm[sl * %d + (tid >> 5)] += (double)%s;\n}\n}\n", NW, v[0].c_str());
    pend.clear();
    return r;
}

std::string Gen::op(const svk::DevOp<float>& o, int gi) {
    const int K = 1 << R;
    switch (o.type) {
        case svk::OP_U: case svk::OP_UR: case svk::OP_X:
            return dense(o, gi);
        case svk::OP_PHASE0: case svk::OP_PHASE1: {
            std::string r = "{\nconst float2 w = " + phase_factor(o, gi) + ";\n";
            for (int k = 0; k < K; ++k)
                if (o.type == svk::OP_PHASE0 || ((k >> o.j) & 1))
                    for (int v = 0; v < NV; ++v) r += fmt("%s = svj_cmul(%s, w);\n", amp(v, k).c_str(), amp(v, k).c_str());
            return r + "}\n";
        }
        case svk::OP_PHASE2: {
            const int c = A.F(o.m[0]);
            A.F(o.m[1]);
            std::string r = fmt("{\nconst float2 w = make_float2(S.f[%d], S.f[%d]);\n", c, c + 1);
            for (int k = 0; k < K; ++k)
                if (((k >> o.j) & 1) && ((k >> o.u) & 1))
                    for (int v = 0; v < NV; ++v) r += fmt("%s = svj_cmul(%s, w);\n", amp(v, k).c_str(), amp(v, k).c_str());
            return r + "}\n";
        }
        case svk::OP_GRAD_X: case svk::OP_GRAD_Y: case svk::OP_GRAD_Z:
            if (NV != 2) return "#error gradient op in a forward program\n";
            return grad(o);
        default:
            return "#error unknown op\n";
    }
}

std::string Gen::run() {
    T = (int)st.T;
    R = (int)st.R;
    TR = T - R;
    NT = 1 << TR;
    NV = V.nv;
    NW = (NT + 31) / 32;
    NPH = (int)st.n_phase;
    NSL = NV == 2 ? (int)st.n_slots : 0;
    const int n = V.n, NG = n - T;
    if (R < 1 || R > 5 || TR < 0 || TR > 9 || T > svk::kMaxT) return "jit: unsupported tile shape";
    if (st.tile_pos[0] != 0) return "jit: the tile must hold physical bit 0";
    BM = V.batched;
    // (not with lambda or gradients in the same kernel: those read the amplitudes mid-stage)
    hdefer = NV == 1 && !BM;
    ZI = V.zero_init;
    if (!BM)
        for (uint32_t i = 0; i < st.n_ops; ++i)
            if (V.ops[i].flags & svk::F_BIND) return "jit: bound (device-formed) ops need a batched stage";
    const size_t tile_b = (size_t)8 << T;
    // double-buffer the tiles when that still leaves the target residency
    // resident threads per SM the register budget is sized for (64 registers per thread
    // forward, 128 adjoint); SVGB_JIT_THR / SVGB_JIT_THR_BWD override for tuning
    int thr_per_sm = (NV == 2 || R >= 5) ? 512 : 1024;
    if (const char* e = getenv(NV == 2 ? "SVGB_JIT_THR_BWD" : "SVGB_JIT_THR"))
        thr_per_sm = std::max(64, std::min(2048, atoi(e)));
    const int ctas = std::max(1, thr_per_sm / std::max(NT, 32));
    NB = (NG > 0 && (size_t)ctas * 2 * NV * tile_b <= 200 * 1024) ? 2 : 1;
    if (const char* e = getenv("SVGB_JIT_NB")) NB = std::max(1, std::min(2, atoi(e)));
    if (NG == 0) NB = 1;
    ttab = (size_t)NPH * NT * 4 <= 16 * 1024;
    // Where per-op constants live: read from the parameter bank they are free operands
    // of the FP32 instructions, but in long stages the compiler hoists them out of the
    // tile loop into registers and spills; those stages read a shared-memory copy.
    int cbank_ops = 160;
    if (const char* e = getenv("SVGB_JIT_CBANK_OPS")) cbank_ops = atoi(e);
    cbank = NV == 1 && (int)st.n_ops <= cbank_ops;
    if (const char* e = getenv("SVGB_JIT_CBANK")) cbank = atoi(e) != 0;
    if (BM) {   // the per-circuit constants are written into the shared-memory copy
        cbank = false;
        NB = 1;
    }

    // ---- TMA eligibility: the tile holds physical bits 0..3, the tile is at least 1 KiB
    // (the 128-byte swizzle repeats every 1 KiB), and the runs of local / global physical
    // bits (local runs cut into pieces of at most 8 bits, the first piece exactly bits 0..3)
    // form at most 5 dimensions ----
    std::vector<Run> dims;
    const bool OUTP = V.dst != nullptr;
    if (OUTP && (NV != 1 || V.batched)) return "jit: an out-of-place permuted write-back needs a forward stage";
    tma = !V.batched && !OUTP && tma_runs(st, n, NV, &dims);
    // ring depth: one slot per CTA for the adjoint (psi and lambda tiles: a second slot
    // would take the shared memory of the SM's second CTA; measured HEA28 backward 92.3 ->
    // 82.5 ms), two otherwise
    NS = NV == 2 ? 1 : 2;
    if (const char* e = getenv("SVGB_JIT_NS")) NS = std::max(1, std::min(4, atoi(e)));
    if (tma) {   // coordinates of a tile along each dimension: (tile index >> shift) & mask
        B->tma = true;
        int gbits = 0;
        uint32_t sh[5] = {0, 0, 0, 0, 0}, mk[5] = {0, 0, 0, 0, 0};
        for (size_t d = 0; d < dims.size(); ++d) {
            B->gdim[d] = 1ull << dims[d].len;
            if (d > 0) B->gstride[d - 1] = 8ull << dims[d].start;
            B->box[d] = dims[d].local ? (1u << dims[d].len) : 1u;
            if (!dims[d].local) {
                sh[d] = (uint32_t)gbits;
                mk[d] = (uint32_t)((1ull << dims[d].len) - 1);
                gbits += dims[d].len;
            }
        }
        for (size_t d = dims.size(); d < 5; ++d) {   // unused dimensions of extent 1
            if (d > 0) B->gstride[d - 1] = 8ull << n;
        }
        for (int d = 0; d < 5; ++d) A.U(sh[d]);
        for (int d = 0; d < 5; ++d) A.U(mk[d]);
    }
    // thread-bit order of each register group: the tile's non-register bits, the first
    // lanes on bits whose shared-memory bank images are independent (TMA layout)
    tbo.assign(st.n_groups, std::vector<int>());
    for (uint32_t g = 0; g < st.n_groups; ++g) {
        const svk::Group& G = V.groups[g];
        std::vector<int> rest(G.thr_pos, G.thr_pos + TR);
        if (tma) {
            const bool pr = G.reg_pos[0] == 0;
            const uint32_t bmask = pr ? 0xEu : 0xFu;   // bank-select bits of a 16-byte / 8-byte access
            const int want = pr ? 3 : 4;
            std::vector<int> first;
            std::vector<uint32_t> basis;
            for (int round = 0; round < want; ++round) {
                int pick = -1;
                for (size_t i = 0; i < rest.size() && pick < 0; ++i) {
                    uint32_t img = swz(1u << rest[i]) & bmask;
                    for (uint32_t bv : basis)   // reduce against the chosen images
                        if ((img ^ bv) < img) img ^= bv;
                    if (img) {
                        pick = (int)i;
                        basis.push_back(img);
                        std::sort(basis.rbegin(), basis.rend());
                    }
                }
                if (pick < 0) break;
                first.push_back(rest[pick]);
                rest.erase(rest.begin() + pick);
            }
            first.insert(first.end(), rest.begin(), rest.end());
            rest = first;
        }
        tbo[g] = rest;
    }

    // ---- argument block layout: m0, m1 (tensor maps), v0, v1, partial, flag | q[] | u[] | f[] ----
    // q: global bit values (NG), tile bit values (T), then op masks
    for (int i = 0; i < NG; ++i) A.Q(1ull << st.glob_pos[i]);
    for (int b = 0; b < T; ++b) A.Q(1ull << st.tile_pos[b]);
    const int QG = 0, QT = NG;
    // phase slots: per slot [cangle, n_glob, first term] in u[], global-term masks in
    // q[] and their angles in u[]; thread-bit coefficients J[i] in u[]
    slot_thr.assign(NPH, -1);
    int slot_u = (int)A.u.size();
    for (int p = 0; p < NPH; ++p) {
        A.U(0);
        A.U(0);
        A.U(0);
    }
    for (int p = 0; p < NPH; ++p) {
        const svk::PhaseSlot<float>& ps = V.slots[p];
        A.u[slot_u + 3 * p] = ps.cangle;
        A.u[slot_u + 3 * p + 1] = ps.n_glob;
        A.u[slot_u + 3 * p + 2] = (uint32_t)A.q.size();   // first mask (angles follow in u at the same rank)
        for (uint32_t i = 0; i < ps.n_glob; ++i) A.Q(V.terms[ps.glob_off + i].mask);
    }
    int slot_ang_u = (int)A.u.size();   // angles of the global terms, in mask order from slot_q0
    const int slot_q0 = QT + T;
    for (int p = 0; p < NPH; ++p) {
        const svk::PhaseSlot<float>& ps = V.slots[p];
        for (uint32_t i = 0; i < ps.n_glob; ++i) A.U(V.terms[ps.glob_off + i].angle);
    }
    // J[i] is the slot's angle per thread bit i in the lowering's order of its group's
    // thread bits; the generated kernel may order them differently (tbo), so map them
    std::vector<int> slot_group(NPH, -1);
    for (uint32_t g = 0; g < st.n_groups; ++g)
        for (uint32_t oi = 0; oi < V.groups[g].n_ops; ++oi) {
            const svk::DevOp<float>& o = V.ops[V.groups[g].op_off + oi];
            if ((o.flags & svk::F_SLOT) && (int)o.slot < NPH) slot_group[o.slot] = (int)g;
        }
    for (int p = 0; p < NPH; ++p)
        if (V.slots[p].has_thr) {
            if (slot_group[p] < 0) return "jit: a phase slot without an op";
            const svk::Group& G = V.groups[slot_group[p]];
            slot_thr[p] = (int)A.u.size();
            for (int i = 0; i < TR; ++i) {
                int src = -1;
                for (int k = 0; k < TR; ++k)
                    if (G.thr_pos[k] == tbo[slot_group[p]][i]) src = k;
                if (src < 0) return "internal: thread-bit order";
                A.U(V.slots[p].J[src]);
            }
        }

    // ---- per-CTA setup ----
    std::string pre;
    pre += fmt("const u32 tid = threadIdx.x;\n");
    pre += fmt("const u64 ntiles = 1ull << %d;\n", NG);
    if (!BM) pre += "u64 t = blockIdx.x;\nif (t >= ntiles) return;\n";
    else pre += "u64 t = 0;\n";
    pre += "u64 base = 0, pstep = 0, gmask = 0;\n";
    if (NG > 0)
        pre += fmt("#pragma unroll 1\nfor (int i = 0; i < %d; ++i) {\nconst u64 b = a.q[%d + i];\ngmask |= b;\n"
                   "if ((t >> i) & 1ull) base |= b;\nif (((u64)gridDim.x >> i) & 1ull) pstep |= b;\n}\n", NG, QG);
    // this thread's 16-byte chunks: chunk c = tid + i * NT holds tile elements 2c, 2c + 1;
    // tile bit 1 + b <- tid bit b, tile bit 1 + TR + b <- i bit b
    if (!tma) {
        pre += "u64 ptid = 0;\nu32 stid = 0;\n";
        for (int b = 0; b < TR; ++b)
            pre += fmt("if ((tid >> %d) & 1u) { ptid |= a.q[%d]; stid ^= %uu; }\n", b, QT + 1 + b, svk::swizzle8(1u << (1 + b)));
    }
    const int NCH = 1 << (R - 1);
    std::vector<uint32_t> chs(NCH);
    std::vector<std::string> chp(NCH);
    for (int i = 0; i < NCH; ++i) {
        uint32_t sw = 0;
        std::string pe = "0ull";
        for (int b = 0; (1 << b) < NCH; ++b)
            if ((i >> b) & 1) {
                sw ^= svk::swizzle8(1u << (1 + TR + b));
                pe += fmt(" | S.q[%d]", QT + 1 + TR + b);
            }
        chs[i] = sw;
        chp[i] = pe;
    }
    // register groups: per group the thread's swizzled offset and (if used) its physical part
    const int ng = (int)st.n_groups;
    std::vector<bool> needfix(ng, false);
    for (int g = 0; g < ng; ++g) {
        const svk::Group& G = V.groups[g];
        for (uint32_t oi = 0; oi < G.n_ops; ++oi) {
            const svk::DevOp<float>& o = V.ops[G.op_off + oi];
            if (o.ctrl_fix || ((o.flags & svk::F_TERMS) && o.n_terms)) needfix[g] = true;
        }
    }
    // Each group's thread offsets (the swizzled shared-memory offset of the thread's
    // amplitudes, and the physical value of its thread bits where ops test it) would
    // stay live in registers for the whole kernel; they go to a per-CTA table in shared
    // memory instead, or, for stages with very many groups, are recomputed per tile.
    int nfix = 0;
    for (int g = 0; g < ng; ++g) nfix += needfix[g] ? 1 : 0;
    bool gtab = ng > 4 && (size_t)NT * (4 * (size_t)ng + 8 * (size_t)nfix) <= 24 * 1024;
    if (const char* e = getenv("SVGB_JIT_GTAB")) gtab = atoi(e) != 0 && (size_t)NT * (4 * (size_t)ng + 8 * (size_t)nfix) <= 24 * 1024;
    std::vector<int> fixrow(ng, -1);
    {
        int r = 0;
        for (int g = 0; g < ng; ++g)
            if (needfix[g]) fixrow[g] = r++;
    }
    auto so_expr = [&](int g) {
        std::string e = "(0u";
        for (int i = 0; i < TR; ++i) e += fmt(" ^ ((tid >> %d) & 1u ? %uu : 0u)", i, swz(1u << tbo[g][i]));
        return e + ")";
    };
    auto pf_expr = [&](int g, const char* src) {
        std::string e = "(0ull";
        for (int i = 0; i < TR; ++i) e += fmt(" | ((tid >> %d) & 1u ? %s.q[%d] : 0ull)", i, src, QT + tbo[g][i]);
        return e + ")";
    };
    // shared memory: tiles | mbarriers (TMA) | sang[NPH] | tang[NPH][NT] | gsm[NSL][NW]
    size_t o = (size_t)NV * (tma ? NS : NB) * tile_b;
    const size_t o_bar = o;
    if (tma) o += 8 * (size_t)NS;
    o = (o + 15) & ~(size_t)15;
    const size_t o_sang = o;
    o = (o + 4 * (size_t)NPH + 15) & ~(size_t)15;
    const size_t o_tang = o;
    if (ttab) o = (o + 4 * (size_t)NPH * NT + 15) & ~(size_t)15;
    const size_t o_gpf = o;   // u64 [nfix][NT]
    if (gtab) o += 8 * (size_t)nfix * NT;
    const size_t o_gso = o;   // u32 [ng][NT]
    if (gtab) o = (o + 4 * (size_t)ng * NT + 15) & ~(size_t)15;
    const size_t o_gsm = o;
    o += 8 * (size_t)NSL * NW;
    o = (o + 15) & ~(size_t)15;
    const size_t o_args = o;   // the argument block's shared-memory copy (size known at the end)
    pre += fmt("float2* const tl = reinterpret_cast<float2*>(smem);\n");
    pre += fmt("u32* const sang = reinterpret_cast<u32*>(smem + %zu);\n", o_sang);
    pre += fmt("u32* const tang = reinterpret_cast<u32*>(smem + %zu);\n", o_tang);
    pre += fmt("double* const gsm = reinterpret_cast<double*>(smem + %zu);\n", o_gsm);
    // per-op constants are read from a shared-memory copy of the arguments: read from
    // the parameter bank they would be hoisted out of the tile loop into registers
    if (cbank) {
        pre += "const Args& S = a;\n";
    } else {
        pre += fmt("{\nconst uint4* src = reinterpret_cast<const uint4*>(&a);\nuint4* dst = reinterpret_cast<uint4*>(smem + %zu);\n"
                   "for (u32 i = tid; i < (u32)(sizeof(Args) / 16); i += %du) dst[i] = src[i];\n}\n", o_args, NT);
        pre += fmt("const Args& S = *reinterpret_cast<const Args*>(smem + %zu);\n", o_args);
    }
    if (gtab) {
        pre += fmt("u64* const gpf = reinterpret_cast<u64*>(smem + %zu);\n", o_gpf);
        pre += fmt("u32* const gso = reinterpret_cast<u32*>(smem + %zu);\n", o_gso);
        for (int g = 0; g < ng; ++g) {
            pre += fmt("gso[%d * %d + tid] = %s;\n", g, NT, so_expr(g).c_str());
            if (needfix[g]) pre += fmt("gpf[%d * %d + tid] = %s;\n", fixrow[g], NT, pf_expr(g, "a").c_str());
        }
    } else {   // few groups: the offsets stay in registers
        for (int g = 0; g < ng; ++g) {
            pre += fmt("const u32 so%d = %s;\n", g, so_expr(g).c_str());
            if (needfix[g]) pre += fmt("const u64 pf%d = %s;\n", g, pf_expr(g, "a").c_str());
        }
    }
    if (tma) {
        pre += fmt("u64* const bars = reinterpret_cast<u64*>(smem + %zu);\n", o_bar);
        pre += fmt("if (tid == 0) {\nfor (int s = 0; s < %d; ++s) svj_mbar_init(&bars[s], 1u);\nsvj_fence_barrier_init();\n}\n", NS);
    }
    pre += "__syncthreads();\n";
    if (ttab)
        for (int p = 0; p < NPH; ++p)
            if (slot_thr[p] >= 0) {
                pre += fmt("{ u32 x = 0;\n");
                for (int i = 0; i < TR; ++i) pre += fmt("if ((tid >> %d) & 1u) x += a.u[%d];\n", i, slot_thr[p] + i);
                pre += fmt("tang[%d * %d + tid] = x; }\n", p, NT);
            }
    if (NSL) pre += fmt("for (u32 i = tid; i < %du; i += %du) gsm[i] = 0.0;\n", NSL * NW, NT);

    // tile load / store
    auto load = [&](const char* buf, const char* bexpr) {
        std::string r;
        for (int i = 0; i < NCH; ++i)
            for (int v = 0; v < NV; ++v)
                r += fmt("svj_cp_async16(tl + ((%d * %d + (%s)) << %d) + (stid ^ %uu), a.v%d + (%s | ptid | %s));\n", v,
                         NB, buf, T, chs[i], v, bexpr, chp[i].c_str());
        return r + "svj_cp_commit();\n";
    };
    // the register groups (also collects the bound ops of a batched stage)
    std::string gcode;
    for (int g = 0; g < ng; ++g) {
        const svk::Group& G = V.groups[g];
        const int K = 1 << R;
        for (int k = 0; k < K; ++k) perm[k] = k;
        std::vector<uint32_t> sr(K);
        for (int k = 0; k < K; ++k) {
            uint32_t x = 0;
            for (int j = 0; j < R; ++j)
                if ((k >> j) & 1) x ^= swz(1u << G.reg_pos[j]);
            sr[k] = x;
        }
        const bool pairs = G.reg_pos[0] == 0;
        gcode += fmt("{ // group %d\n", g);
        if (gtab) gcode += fmt("const u32 so%d = gso[%d * %d + tid];\n", g, g, NT);
        fixvar = "";
        if (needfix[g]) {
            if (gtab) gcode += fmt("const u64 fix = base ^ gpf[%d * %d + tid];\n", fixrow[g], NT);
            else gcode += fmt("const u64 fix = base ^ pf%d;\n", g);
            fixvar = "fix";
        }
        for (int v = 0; v < NV; ++v) {
            for (int k = 0; k < K; ++k) gcode += fmt("float2 %c%d;\n", v ? 'l' : 'p', k);
            if (pairs) {
                for (int k = 0; k < K; k += 2)
                    gcode += fmt("{ const float4 q = *reinterpret_cast<const float4*>(T%d + (so%d ^ %uu)); %c%d = make_float2(q.x, q.y); %c%d = make_float2(q.z, q.w); }\n",
                                v, g, sr[k], v ? 'l' : 'p', k, v ? 'l' : 'p', k + 1);
            } else {
                for (int k = 0; k < K; ++k) gcode += fmt("%c%d = T%d[so%d ^ %uu];\n", v ? 'l' : 'p', k, v, g, sr[k]);
            }
        }
        pend.clear();
        zgen = -1;
        for (uint32_t oi = 0; oi < G.n_ops; ++oi) gcode += op(V.ops[G.op_off + oi], g);
        gcode += reduce_pending();
        if (g == ng - 1 && hscale != 1.0) {   // the deferred Hadamard factors, once
            const int fi = A.F((float)hscale);
            for (int k = 0; k < K; ++k)
                gcode += fmt("%s = __fmul2_rn(make_float2(S.f[%d], S.f[%d]), %s);\n", amp(0, k).c_str(), fi, fi, amp(0, k).c_str());
        }
        for (int v = 0; v < NV; ++v) {
            if (pairs) {
                for (int k = 0; k < K; k += 2)
                    gcode += fmt("*reinterpret_cast<float4*>(T%d + (so%d ^ %uu)) = make_float4(%s.x, %s.y, %s.x, %s.y);\n", v, g,
                                sr[k], amp(v, k).c_str(), amp(v, k).c_str(), amp(v, k + 1).c_str(), amp(v, k + 1).c_str());
            } else {
                for (int k = 0; k < K; ++k) gcode += fmt("T%d[so%d ^ %uu] = %s;\n", v, g, sr[k], amp(v, k).c_str());
            }
        }
        // the last group's writes become visible to the tile's TMA store
        gcode += (tma && g == ng - 1) ? "}\nsvj_fence_async_smem();\n__syncthreads();\n" : "}\n__syncthreads();\n";
    }
    std::string body;
    // TMA: a tile is one box of the 5-D view; its coordinates come from the tile index
    auto crd = [&](const char* tt) {
        std::string r;
        for (int d = 0; d < 5; ++d) r += fmt("%s(int)(((%s) >> S.u[%d]) & (u64)S.u[%d])", d ? ", " : "", tt, d, 5 + d);
        return r;
    };
    auto tma_load = [&](const char* slot, const char* tt) {
        std::string r = fmt("svj_mbar_expect_tx(&bars[%s], %zuu);\n", slot, (size_t)NV * tile_b);
        for (int v = 0; v < NV; ++v)
            r += fmt("svj_tma_load(tl + ((%s * %d + %d) << %d), &a.m%d, %s, &bars[%s]);\n", slot, NV, v, T, v, crd(tt).c_str(), slot);
        return r;
    };
    if (BM) {
        // ---- batched: work items w = (circuit << NG) | tile, a contiguous range per CTA;
        // a new circuit rebinds the parametric matrices and restarts the tile walk ----
        const int bt = (int)A.u.size();
        for (const Bind& b : binds) {
            A.U((uint32_t)b.fi);
            A.U((uint32_t)((b.type << 8) | b.kind));
            A.U((uint32_t)b.param);
        }
        const int nbind = (int)binds.size();
        body += fmt("Args& Sw = *reinterpret_cast<Args*>(smem + %zu);\n", o_args);
        body += fmt("const u64 W = a.ncirc << %d;\n", NG);
        body += "const u64 w0 = (W * blockIdx.x) / gridDim.x, w1 = (W * ((u64)blockIdx.x + 1)) / gridDim.x;\n";
        body += "u32 cc = 0xffffffffu;\nu64 tfirst = 0;\n";
        auto flush = [&]() {
            if (!NSL) return std::string();
            return fmt("if (cc != 0xffffffffu)\nfor (u32 sl = tid; sl < %du; sl += %du) {\ndouble x = 0.0;\n"
                       "for (int wv = 0; wv < %d; ++wv) {\nx += gsm[sl * %d + wv];\ngsm[sl * %d + wv] = 0.0;\n}\n"
                       "a.partial[(((u64)cc << %d) | tfirst) * %d + sl] = x;\n}\n", NSL, NT, NW, NW, NW, NG, NSL);
        };
        body += "#pragma unroll 1\nfor (u64 w = w0; w < w1; ++w) {\n";
        body += fmt("const u32 c = (u32)(w >> %d);\nconst u64 tt = w & (ntiles - 1ull);\n", NG);
        body += "if (c != cc) {\n" + flush() + "cc = c;\ntfirst = tt;\n__syncthreads();\n";
        if (nbind) {
            body += fmt("{\nconst double* pp = a.params + a.pofs[c];\n#pragma unroll 1\nfor (u32 i = tid; i < %du; i += %du) {\n"
                        "const u32 fi = Sw.u[%d + 3 * i], kd = Sw.u[%d + 3 * i + 1], pi = Sw.u[%d + 3 * i + 2];\n"
                        "double sd, cd;\nsincos(0.5 * pp[pi], &sd, &cd);\n"
                        "const float cs = (float)cd, sn = (kd & 4u) ? -(float)sd : (float)sd;\nfloat* f = Sw.f + fi;\n"
                        "if ((kd >> 8) == %du) {\nf[0] = cs; f[1] = -sn; f[2] = sn; f[3] = cs;\n} else {\n"
                        "f[0] = cs; f[1] = 0.f; f[2] = 0.f; f[3] = 0.f; f[4] = 0.f; f[5] = 0.f; f[6] = cs; f[7] = 0.f;\n"
                        "const u32 k = kd & 3u;\nif (k == 1u) { f[3] = -sn; f[5] = -sn; }\n"
                        "else if (k == 2u) { f[2] = -sn; f[4] = sn; }\nelse { f[1] = -sn; f[7] = sn; }\n}\n}\n}\n",
                        nbind, NT, bt, bt, bt, (unsigned)svk::OP_UR);
        }
        body += fmt("base = 0;\n#pragma unroll 1\nfor (int i = 0; i < %d; ++i)\nif ((tt >> i) & 1ull) base |= a.q[%d + i];\n", NG, QG);
        body += "__syncthreads();\n}\n";
        for (int v = 0; v < NV; ++v) body += fmt("float2* const g%d = a.v%d + ((u64)c << %d);\n", v, v, n);
        if (ZI) {   // |0...0> restricted to this tile: element 0 (storage 0) of the tile with base 0
            for (int i = 0; i < NCH; ++i)
                body += fmt("*reinterpret_cast<float4*>(tl + (stid ^ %uu)) = make_float4((base == 0ull && tid == 0u && %d == 0) ? 1.f : 0.f, 0.f, 0.f, 0.f);\n",
                            chs[i], i);
        } else {
            for (int i = 0; i < NCH; ++i)
                for (int v = 0; v < NV; ++v)
                    body += fmt("svj_cp_async16(tl + ((%d << %d) + (stid ^ %uu)), g%d + (base | ptid | %s));\n", v, T, chs[i], v,
                                chp[i].c_str());
            body += "svj_cp_commit();\nsvj_cp_wait0();\n";
        }
        if (NPH) {
            body += fmt("#pragma unroll 1\nfor (u32 p = tid; p < %du; p += %du) {\nu32 x = S.u[%d + 3 * p];\nconst u32 ng = S.u[%d + 3 * p + 1], q0 = S.u[%d + 3 * p + 2];\n",
                        NPH, NT, slot_u, slot_u, slot_u);
            body += fmt("#pragma unroll 1\nfor (u32 i = 0; i < ng; ++i)\nif (base & S.q[q0 + i]) x += S.u[%d + (q0 - %d) + i];\nsang[p] = x;\n}\n",
                        slot_ang_u, slot_q0);
        }
        body += "__syncthreads();\n";
        for (int v = 0; v < NV; ++v) body += fmt("float2* const T%d = tl + (%d << %d);\n", v, v, T);
        body += gcode;
        for (int i = 0; i < NCH; ++i)
            for (int v = 0; v < NV; ++v)
                body += fmt("*reinterpret_cast<float4*>(g%d + (base | ptid | %s)) = *reinterpret_cast<const float4*>(T%d + (stid ^ %uu));\n",
                            v, chp[i].c_str(), v, chs[i]);
        body += fmt("base = ((base | ~gmask) + a.q[%d]) & gmask;\n__syncthreads();\n}\n", QG);
        body += flush();
    } else {
        if (tma) {
            body += "if (tid == 0) {\n";
            for (int sl = 0; sl < NS; ++sl)
                body += fmt("if (t + %du * (u64)gridDim.x < ntiles) {\nconst u64 tt = t + %du * (u64)gridDim.x;\n", sl, sl) +
                        tma_load(std::to_string(sl).c_str(), "tt") + "}\n";
            body += "}\n";
        } else {
            body += load("0", "base");
        }
        if (tma) body += "u32 brk = 0xffffffffu;   // iteration whose tile wait gave up\n";
        body += "#pragma unroll 1\nfor (u32 it = 0; t < ntiles; t += gridDim.x, ++it) {\n";
        body += "const u64 bn = ((base | ~gmask) + pstep) & gmask;\n";
        if (tma) {
            body += fmt("const u32 cb = it %% %du;\n", NS);
            body += fmt("if (!__syncthreads_and(svj_mbar_wait(&bars[cb], (it / %du) & 1u, a.flag))) {\nbrk = it;\nbreak;\n}\n", NS);
        } else if (NB == 2) {
            body += "const u32 cb = it & 1u;\n";
            body += "if (t + gridDim.x < ntiles) {\n" + load("cb ^ 1u", "bn") + "svj_cp_wait1();\n} else {\nsvj_cp_wait0();\n}\n";
        } else {
            body += "const u32 cb = 0u;\n";
            body += "if (it > 0) {\n" + load("0", "base") + "}\nsvj_cp_wait0();\n";
        }
        if (NPH) {   // per-tile slot angles: the constant plus the global-bit terms set in this tile
            body += fmt("#pragma unroll 1\nfor (u32 p = tid; p < %du; p += %du) {\nu32 x = S.u[%d + 3 * p];\nconst u32 ng = S.u[%d + 3 * p + 1], q0 = S.u[%d + 3 * p + 2];\n",
                        NPH, NT, slot_u, slot_u, slot_u);
            body += fmt("#pragma unroll 1\nfor (u32 i = 0; i < ng; ++i)\nif (base & S.q[q0 + i]) x += S.u[%d + (q0 - %d) + i];\nsang[p] = x;\n}\n",
                        slot_ang_u, slot_q0);
        }
        body += "__syncthreads();\n";
        for (int v = 0; v < NV; ++v) {
            if (tma) body += fmt("float2* const T%d = tl + ((cb * %d + %d) << %d);\n", v, NV, v, T);
            else body += fmt("float2* const T%d = tl + ((%d * %d + cb) << %d);\n", v, v, NB, T);
        }
        body += gcode;
        if (tma) {
            // one thread stores the tile (bulk tensor copy) and refills the slot with the tile
            // NS steps ahead once the store has read it
            body += "if (tid == 0) {\n";
            for (int v = 0; v < NV; ++v) body += fmt("svj_tma_store(&a.m%d, %s, T%d);\n", v, crd("t").c_str(), v);
            body += "svj_bulk_commit();\n";
            body += fmt("const u64 tn = t + %du * (u64)gridDim.x;\nif (tn < ntiles) {\nsvj_bulk_wait_read0();\n", NS) +
                    tma_load("cb", "tn") + "}\n}\n";
            body += "base = bn;\n}\n";
            // a wait that gave up leaves loads in flight: wait for them (bounded) before the
            // CTA's shared memory goes away; then for the tile stores
            body += fmt("if (tid == 0) {\nif (brk != 0xffffffffu)\nfor (u32 k = 0; k < %du; ++k) {\nconst u32 i2 = brk + k;\n"
                        "if ((u64)blockIdx.x + (u64)i2 * gridDim.x < ntiles) svj_mbar_wait(&bars[i2 %% %du], (i2 / %du) & 1u, nullptr);\n}\n"
                        "svj_bulk_wait0();\n}\n", NS, NS, NS);
        } else if (OUTP) {
            // out of place through the bit map: output element e enumerates the tile bits in
            // order of their destination bits (o[0] lowest), so a thread writes the pair
            // e, e + 1 and consecutive threads consecutive pairs of the destination
            std::vector<std::pair<int, int>> od;
            for (int b = 0; b < T; ++b) od.push_back({V.dst[st.tile_pos[b]], b});
            std::sort(od.begin(), od.end());
            const int QD = (int)A.q.size();
            for (int i = 0; i < NG; ++i) A.Q(1ull << V.dst[st.glob_pos[i]]);
            for (int k = 0; k < T; ++k) A.Q(1ull << od[k].first);
            pre += "u64 dtid = 0;\nu32 otid = 0;\n";
            for (int j = 0; j < TR; ++j)
                pre += fmt("if ((tid >> %d) & 1u) { dtid |= a.q[%d]; otid ^= %uu; }\n", j, QD + NG + 1 + j,
                           swz(1u << od[1 + j].second));
            const bool rd4 = od[0].second == 0, wr4 = od[0].first == 0;
            const uint32_t s1 = swz(1u << od[0].second);
            body += fmt("{\nu64 dbase = 0;\n#pragma unroll 1\nfor (int i = 0; i < %d; ++i)\nif ((t >> i) & 1ull) dbase |= S.q[%d + i];\n",
                        NG, QD);
            for (int i = 0; i < NCH; ++i) {
                uint32_t so = 0;
                std::string pe = "dbase | dtid";
                for (int b = 0; (1 << b) < NCH; ++b)
                    if ((i >> b) & 1) {
                        so ^= swz(1u << od[1 + TR + b].second);
                        pe += fmt(" | S.q[%d]", QD + NG + 1 + TR + b);
                    }
                body += "{\n";
                if (rd4) body += fmt("const float4 x = *reinterpret_cast<const float4*>(T0 + (otid ^ %uu));\n", so);
                else body += fmt("const float2 x0 = T0[otid ^ %uu], x1 = T0[otid ^ %uu];\n", so, so ^ s1);
                body += fmt("float2* const d = a.v1 + (%s);\n", pe.c_str());
                if (wr4) body += rd4 ? "*reinterpret_cast<float4*>(d) = x;\n"
                                     : "*reinterpret_cast<float4*>(d) = make_float4(x0.x, x0.y, x1.x, x1.y);\n";
                else if (rd4) body += fmt("d[0] = make_float2(x.x, x.y);\nd[S.q[%d]] = make_float2(x.z, x.w);\n", QD + NG);
                else body += fmt("d[0] = x0;\nd[S.q[%d]] = x1;\n", QD + NG);
                body += "}\n";
            }
            body += "}\nbase = bn;\n__syncthreads();\n}\n";
        } else {
            // write the tile back in place
            for (int i = 0; i < NCH; ++i)
                for (int v = 0; v < NV; ++v)
                    body += fmt("*reinterpret_cast<float4*>(a.v%d + (base | ptid | %s)) = *reinterpret_cast<const float4*>(T%d + (stid ^ %uu));\n",
                                v, chp[i].c_str(), v, chs[i]);
            body += "base = bn;\n__syncthreads();\n}\n";
        }
        if (NSL)
            body += fmt("for (u32 sl = tid; sl < %du; sl += %du) {\ndouble x = 0.0;\nfor (int w = 0; w < %d; ++w) x += gsm[sl * %d + w];\n"
                        "a.partial[(u64)blockIdx.x * %d + sl] = x;\n}\n", NSL, NT, NW, NW, NSL);
    }

    // ---- assemble ----
    const int nq = std::max<int>(1, (int)A.q.size()), nu = std::max<int>(1, (int)A.u.size()),
              nf = std::max<int>(1, (int)A.f.size());
    const int minb = std::max(1, std::min(32, thr_per_sm / NT));
    std::string head;
    head += "#include \"jit_prelude.cuh\"\n";
    head += fmt("struct alignas(64) Args {\nSvjTmap m0;\nSvjTmap m1;\nfloat2* v0;\nfloat2* v1;\ndouble* partial;\nint* flag;\n"
                "const double* params;\nconst u32* pofs;\nu64 ncirc;\nu64 q[%d];\nu32 u[%d];\nfloat f[%d];\n};\n", nq, nu, nf);
    std::string src = head + "extern \"C\" __global__ void __launch_bounds__(" + std::to_string(NT) + ", " +
                      std::to_string(minb) + ") KNAME(const __grid_constant__ Args a) {\n"
                      "extern __shared__ __attribute__((aligned(1024))) unsigned char smem[];\n" + pre + body + "}\n";
    const std::string name = fmt("svj_%s_%016llx", NV == 2 ? "adj" : "fwd", (unsigned long long)fnv1a(src));
    size_t pos;
    while ((pos = src.find("KNAME")) != std::string::npos) src.replace(pos, 5, name);
    B->src = src;
    B->name = name;
    B->nthr = (uint32_t)NT;
    B->n_slots = (uint32_t)NSL;
    B->ntiles = 1ull << NG;
    // argument bytes, matching the struct: two 128-byte tensor maps, four pointers, q, u,
    // f, padded to the struct's 64-byte alignment
    const size_t off_q = kArgQ;
    size_t bytes = off_q + 8 * (size_t)nq + 4 * (size_t)nu;
    bytes = (bytes + 3) & ~(size_t)3;
    const size_t off_f = bytes;
    bytes += 4 * (size_t)nf;
    bytes = (bytes + 63) & ~(size_t)63;
    if (bytes > 32000) return "jit: stage constants exceed the kernel argument space";
    B->smem = (uint32_t)(cbank ? o_args : o_args + bytes);
    B->args.assign(bytes, 0);
    std::memcpy(B->args.data() + off_q, A.q.data(), 8 * A.q.size());
    std::memcpy(B->args.data() + off_q + 8 * nq, A.u.data(), 4 * A.u.size());
    std::memcpy(B->args.data() + off_f, A.f.data(), 4 * A.f.size());
    return "";
}

// The generated source depends on a stage's structure only: tile and register-group
// shapes (tile-bit indices), op kinds, register bits, flags and counts, and which
// masks are empty.  The key below holds exactly those fields (plus the tuning
// variables the generator reads), so stages that differ in values only — angles,
// matrices, physical bit positions, control masks — share one source, and a new
// stage of a known structure needs only its argument block (a quiet re-walk).
std::string structure_key(const StageView& v) {
    std::string k;
    auto put = [&](uint64_t x) { k.append((const char*)&x, sizeof(x)); };
    const svk::Stage& st = *v.st;
    put((uint64_t)v.nv);
    put((uint64_t)v.n);
    put((uint64_t)v.batched << 1 | (uint64_t)v.zero_init);
    put(st.T);
    put(st.R);
    put(st.n_groups);
    put(v.nv == 2 ? st.n_slots : 0);
    put(st.n_phase);
    put(st.n_ops);
    put(st.tile_pos[0]);
    put(st.R);
    {
        std::vector<Run> dims;
        put(!v.dst && tma_runs(st, v.n, v.nv, &dims) ? 1 : 0);
    }
    if (v.dst) {   // the write-back order: tile bits by destination, and whether it starts at bit 0
        std::vector<std::pair<int, int>> od;
        for (uint32_t b = 0; b < st.T; ++b) od.push_back({v.dst[st.tile_pos[b]], (int)b});
        std::sort(od.begin(), od.end());
        put(2 + (od[0].first == 0 ? 1 : 0));
        for (auto& x : od) put((uint64_t)x.second);
    } else {
        put(0);
    }
    for (const char* e : {"SVGB_JIT_TMA", "SVGB_JIT_NS", "SVGB_JIT_NB", "SVGB_JIT_THR", "SVGB_JIT_THR_BWD", "SVGB_JIT_CBANK", "SVGB_JIT_CBANK_OPS", "SVGB_JIT_GTAB"}) {
        const char* x = getenv(e);
        k += x ? x : "-";
        k += '|';
    }
    const int TR = (int)st.T - (int)st.R;
    for (uint32_t g = 0; g < st.n_groups; ++g) {
        const svk::Group& G = v.groups[g];
        put(G.op_off);
        put(G.n_ops);
        for (uint32_t j = 0; j < st.R; ++j) put(G.reg_pos[j]);
        for (int i = 0; i < TR; ++i) put(G.thr_pos[i]);
    }
    for (uint32_t i = 0; i < st.n_ops; ++i) {
        const svk::DevOp<float>& o = v.ops[i];
        put(o.type | (uint64_t)o.j << 8 | (uint64_t)o.u << 16 | (uint64_t)o.flags << 24 | (uint64_t)(o.ctrl_fix != 0) << 32);
        put(o.ctrl_reg);
        put(h_like(o) ? 1 : 0);
        put(o.slot);
        put(o.n_terms);
        if (o.flags & (svk::F_TERMS | svk::F_TW))
            for (uint32_t t = 0; t < o.n_terms; ++t) put(v.terms[o.term_off + t].mask == 0);
    }
    for (uint32_t p = 0; p < st.n_phase; ++p) {
        put(v.slots[p].n_glob);
        put(v.slots[p].has_thr);
    }
    return k;
}

struct Shape {
    std::string src, name;
};
std::mutex g_shape_mu;
std::unordered_map<std::string, std::shared_ptr<Shape>> g_shapes;   // structure key -> source

}  // namespace

std::string generate(const StageView& v, Built* out) {
    const std::string key = structure_key(v);
    std::shared_ptr<Shape> sh;
    {
        std::lock_guard<std::mutex> lk(g_shape_mu);
        auto it = g_shapes.find(key);
        if (it != g_shapes.end()) sh = it->second;
    }
    if (sh) {   // known structure: fill the argument block only
        g_quiet = true;
        Gen g(v, out);
        std::string err = g.run();
        g_quiet = false;
        if (!err.empty()) return err;
        out->src = sh->src;
        out->name = sh->name;
        return "";
    }
    Gen g(v, out);
    std::string err = g.run();
    if (!err.empty()) return err;
    auto ns = std::make_shared<Shape>();
    ns->src = out->src;
    ns->name = out->name;
    std::lock_guard<std::mutex> lk(g_shape_mu);
    if (g_shapes.size() > 8192) g_shapes.clear();
    g_shapes[key] = ns;
    return "";
}

static std::string nvrtc_compile(const std::string& src, const std::string& name, std::vector<char>* cubin) {
    if (const char* dir = getenv("SVGB_JIT_DUMP")) {   // keep the generated source (profiling, reading)
        if (FILE* f = fopen((std::string(dir) + "/" + name + ".cu").c_str(), "w")) {
            fwrite(src.data(), 1, src.size(), f);
            fclose(f);
        }
    }
    nvrtcProgram prog;
    const char* hdrs[1] = {kJitPrelude};
    const char* hnames[1] = {"jit_prelude.cuh"};
    if (nvrtcCreateProgram(&prog, src.c_str(), (name + ".cu").c_str(), 1, hdrs, hnames) != NVRTC_SUCCESS)
        return "nvrtcCreateProgram failed";
    const char* opts[] = {"-arch=sm_103a", "-std=c++17", "-default-device", "-lineinfo"};
    nvrtcResult r = nvrtcCompileProgram(prog, 4, opts);
    std::string err;
    if (r != NVRTC_SUCCESS) {
        size_t n = 0;
        nvrtcGetProgramLogSize(prog, &n);
        std::string log(n, '\0');
        nvrtcGetProgramLog(prog, &log[0]);
        err = std::string("NVRTC: ") + nvrtcGetErrorString(r) + "\n" + log.substr(0, 4000);
    } else {
        size_t n = 0;
        nvrtcGetCUBINSize(prog, &n);
        cubin->resize(n);
        nvrtcGetCUBIN(prog, cubin->data());
    }
    nvrtcDestroyProgram(&prog);
    return err;
}

std::string compile(std::vector<Built*>& kernels) {
    std::vector<std::pair<Built*, Kernel*>> todo;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        std::unordered_map<std::string, Kernel*> fresh;
        for (Built* b : kernels) {
            auto it = g_cache.find(b->src);
            if (it != g_cache.end()) {
                b->kernel = it->second;
                g_hits++;
                continue;
            }
            auto jt = fresh.find(b->src);
            if (jt != fresh.end()) {
                b->kernel = jt->second;
                continue;
            }
            Kernel* k = new Kernel();
            fresh[b->src] = k;
            b->kernel = k;
            todo.push_back({b, k});
        }
    }
    if (!todo.empty()) {
        const auto t0 = std::chrono::steady_clock::now();
        std::vector<std::vector<char>> bins(todo.size());
        std::vector<std::string> errs(todo.size());
        std::atomic<size_t> next{0};
        const unsigned nth = std::max(1u, std::min<unsigned>((unsigned)todo.size(), std::thread::hardware_concurrency()));
        std::vector<std::thread> pool;
        for (unsigned w = 0; w < nth; ++w)
            pool.emplace_back([&]() {
                for (size_t i; (i = next++) < todo.size();)
                    errs[i] = nvrtc_compile(todo[i].first->src, todo[i].first->name, &bins[i]);
            });
        for (auto& th : pool) th.join();
        std::string first_err;
        for (size_t i = 0; i < todo.size(); ++i) {
            Kernel* k = todo[i].second;
            k->cubin.swap(bins[i]);
            k->err = errs[i];
            if (!errs[i].empty() && first_err.empty()) first_err = errs[i];
        }
        g_compiles += todo.size();
        g_compile_us += (uint64_t)std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0).count();
        std::lock_guard<std::mutex> lk(g_mu);
        for (auto& p : todo) g_cache[p.first->src] = p.second;
        if (!first_err.empty()) return first_err;
    }
    for (Built* b : kernels)
        if (!b->kernel->err.empty()) return b->kernel->err;
    return "";
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (the
// library links the runtime only)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// the stage's 5-D view of a state vector at ptr (8-byte elements, 128-byte swizzle)
static cudaError_t encode_map(const Built& b, void* ptr, void* out) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const cuuint32_t estride[5] = {1, 1, 1, 1, 1};
    cuuint64_t gdim[5], gstr[4];
    cuuint32_t box[5];
    for (int d = 0; d < 5; ++d) {
        gdim[d] = b.gdim[d];
        box[d] = b.box[d];
    }
    for (int d = 0; d < 4; ++d) gstr[d] = b.gstride[d];
    const CUresult r = fn((CUtensorMap*)out, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5, ptr, gdim, gstr, box, estride,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// load the kernel's library on first use and (re)size its launch attributes for the
// current device; returns the resident CTAs per SM in *per_sm
static cudaError_t ready(const Built& b, int* per_sm) {
    Kernel* k = b.kernel;
    if (!k || !k->err.empty() || k->cubin.empty()) return cudaErrorInvalidDeviceFunction;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(k->mu);
    if (!k->fn) {   // context-independent load: the library is usable on every device
        e = cudaLibraryLoadData(&k->lib, k->cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
        if (e != cudaSuccess) return e;
        e = cudaLibraryGetKernel(&k->fn, k->lib, b.name.c_str());
        if (e != cudaSuccess) return e;
    }
    if (k->dev != dev || k->smem_set < b.smem) {
        e = cudaFuncSetAttribute((const void*)k->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b.smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k->fn, (int)b.nthr, b.smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        k->per_sm_dev = per_sm;
        k->dev = dev;
        k->smem_set = b.smem;
    }
    *per_sm = k->per_sm_dev;
    return cudaSuccess;
}

cudaError_t preload(const Built& b) {
    int per_sm = 0;
    return ready(b, &per_sm);
}

static uint8_t* fill_args(const Built& b, void* v0, void* v1, double* partial, int* flag) {
    alignas(64) static thread_local uint8_t argbuf[32768];
    if (b.args.size() > sizeof(argbuf)) return nullptr;
    std::memcpy(argbuf, b.args.data(), b.args.size());
    std::memcpy(argbuf + kArgV0, &v0, 8);
    std::memcpy(argbuf + kArgV1, &v1, 8);
    std::memcpy(argbuf + kArgPartial, &partial, 8);
    std::memcpy(argbuf + kArgFlag, &flag, 8);
    return argbuf;
}

cudaError_t launch_batched(const Built& b, void* v0, void* v1, double* partial, int* flag, const double* params,
                           const uint32_t* pofs, uint32_t ncirc, cudaStream_t s) {
    int per_sm = 0;
    cudaError_t e = ready(b, &per_sm);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const uint64_t W = (uint64_t)ncirc * b.ntiles;
    if (W == 0) return cudaSuccess;
    const uint64_t grid = std::min<uint64_t>(W, (uint64_t)per_sm * (uint64_t)nsm);
    uint8_t* args = fill_args(b, v0, v1, partial, flag);
    if (!args) return cudaErrorInvalidValue;
    const uint64_t nc = ncirc;
    std::memcpy(args + kArgParams, &params, 8);
    std::memcpy(args + kArgPofs, &pofs, 8);
    std::memcpy(args + kArgNcirc, &nc, 8);
    void* p[1] = {args};
    return cudaLaunchKernel((const void*)b.kernel->fn, dim3((unsigned)grid), dim3(b.nthr), p, b.smem, s);
}

cudaError_t launch(const Built& b, void* v0, void* v1, double* partial, int* flag, cudaStream_t s,
                   uint32_t* grid_out) {
    int per_sm = 0;
    cudaError_t e = ready(b, &per_sm);
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    Kernel* k = b.kernel;
    int nsm = 0;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const uint64_t grid = std::min<uint64_t>(b.ntiles, (uint64_t)per_sm * (uint64_t)nsm);
    if (grid_out) *grid_out = (uint32_t)grid;
    // the argument block, 64-byte aligned (the tensor maps inside must be)
    uint8_t* args = fill_args(b, v0, v1, partial, flag);
    if (!args) return cudaErrorInvalidValue;
    if (b.tma) {
        e = encode_map(b, v0, args + 0);
        if (e != cudaSuccess) return e;
        if (v1) {
            e = encode_map(b, v1, args + 128);
            if (e != cudaSuccess) return e;
        }
    }
    void* params[1] = {args};
    return cudaLaunchKernel((const void*)k->fn, dim3((unsigned)grid), dim3(b.nthr), params, b.smem, s);
}

void stats(uint64_t* compiles, uint64_t* hits, double* compile_ms) {
    if (compiles) *compiles = g_compiles.load();
    if (hits) *hits = g_hits.load();
    if (compile_ms) *compile_ms = g_compile_us.load() / 1000.0;
}


// ---------------------------------------------------------------------------
// Pauli-sum expectation sweeps (the observable of Sec. 4.2): one sweep's terms compiled
// into a kernel, expectation only.  Per tile a thread holds 16 amplitudes a_k (register
// bits = tile bits 4..7 of the sweep's layout) and sums |a_k|^2 times the diagonal weight,
// plus, for each X / Y term, Re(conj(a_k) f s_k p_k) with p_k the partner amplitude (in a
// register, or in the tile staged in shared memory); terms whose X / Y qubits all sit on
// the top 4 tile bits are evaluated from a second read of the tile with those bits as the
// register bits.  A Pauli string is Hermitian, so the
// two amplitudes of a register pair contribute complex-conjugate terms: one is
// evaluated, twice.  Tiles are double-buffered with cp.async; FP32 per tile, compensated
// FP32 across a thread's tiles, FP64 across threads.
// ---------------------------------------------------------------------------
std::string generate_pauli(const svk::PauliSweep& sw, const svk::PauliTerm* terms, int n, Built* B) {
    const int T = (int)sw.T, R = (int)sw.R, L = (int)sw.L, NG = (int)sw.n_glob;
    if (L != 4 || R != 4 || T < 9 || T > 13 || n - T != NG) return "pauli jit: unsupported sweep shape";
    const int NT = 1 << (T - R), K = 1 << R;
    // tile buffers per CTA (2: the next tile's copy overlaps this one) and CTAs per SM the
    // registers are budgeted for; SVGB_PAULI_NB / SVGB_PAULI_MINB override for tuning
    int NBUF = 2, MINB = 1;
    if (const char* e = getenv("SVGB_PAULI_NB")) NBUF = std::max(1, std::min(2, atoi(e)));
    if (const char* e = getenv("SVGB_PAULI_MINB")) MINB = std::max(1, std::min(4, atoi(e)));
    const svk::PauliTerm* tl = terms + sw.term_off;
    const uint32_t nterm = sw.n_terms, d0 = sw.n_dstat, d1 = d0 + sw.n_dglob, d2 = d1 + sw.n_dmix;
    const uint32_t regmask = ((1u << R) - 1u) << L;
    ArgBuilder A;
    for (int i = 0; i < NG; ++i) A.Q(1ull << sw.glob_pos[i]);
    const int QT = NG;
    for (int b = 0; b < T; ++b) A.Q(sw.ptile[b]);
    auto tmask = [&](uint64_t z) {
        uint32_t m = 0;
        for (int b = 0; b < T; ++b)
            if (z & sw.ptile[b]) m |= 1u << b;
        return m;
    };
    auto amp = [](int k) { return fmt("x%d", k); };
    std::string pre, body;
    pre += "const u32 tid = threadIdx.x;\n";
    pre += fmt("const u64 ntiles = 1ull << %d;\nu64 t = blockIdx.x;\nif (t >= ntiles) return;\n", NG);
    pre += fmt("float2* const tb0 = reinterpret_cast<float2*>(smem);\nfloat2* const tb1 = tb0 + %d;\n", NBUF == 2 ? 1 << T : 0);
    pre += fmt("const u32 te = (tid & 15u) | ((tid >> 4) << %d);\n", L + R);
    pre += fmt("u64 tphys = 0;\n#pragma unroll\nfor (int b = 0; b < %d; ++b)\nif ((te >> b) & 1u) tphys |= a.q[%d + b];\n", T, QT);
    const int rounds = (1 << T) / 2 / NT;
    pre += fmt("u64 ld_tid = 0;\n#pragma unroll\nfor (int b = 1; b < %d; ++b)\nif (((2u * tid) >> b) & 1u) ld_tid |= a.q[%d + b];\n", T, QT);
    pre += fmt("u64 jp[%d];\n#pragma unroll\nfor (int j = 0; j < %d; ++j) {\nu64 p = 0;\nconst u32 e = %du * (u32)j;\n", rounds, rounds, 2 * NT);
    pre += fmt("#pragma unroll\nfor (int b = 1; b < %d; ++b)\nif ((e >> b) & 1u) p |= a.q[%d + b];\njp[j] = p;\n}\n", T, QT);
    pre += "u64 base = 0, pstep = 0, gmask = 0;\n";
    if (NG > 0)
        pre += fmt("#pragma unroll 1\nfor (int i = 0; i < %d; ++i) {\nconst u64 b = a.q[i];\ngmask |= b;\nif ((t >> i) & 1ull) base |= b;\n"
                   "if (((u64)gridDim.x >> i) & 1ull) pstep |= b;\n}\n", NG);
    // static diagonal weights (Z on tile bits only): w_k = sum c (-1)^(|te & zthr|) (-1)^(|k & zreg|)
    pre += fmt("float w[%d];\n#pragma unroll\nfor (int k = 0; k < %d; ++k) w[k] = 0.f;\n", K, K);
    for (uint32_t i = 0; i < d0; ++i) {
        const svk::PauliTerm& pt = tl[i];
        const uint32_t zthr = tmask(pt.zmask) & ~regmask;
        const int c = A.F(pt.fre32);
        pre += zthr ? fmt("{\nconst float c = (__popc(te & %uu) & 1) ? -a.f[%d] : a.f[%d];\n", zthr, c, c)
                    : fmt("{\nconst float c = a.f[%d];\n", c);
        for (int k = 0; k < K; ++k) pre += fmt("w[%d] %s= c;\n", k, (__builtin_popcount((unsigned)k & pt.zreg) & 1) ? "-" : "+");
        pre += "}\n";
    }
    auto issue = [&](const char* bexpr, const char* buf) {
        std::string r;
        for (int j = 0; j < rounds; ++j)
            r += fmt("svj_cp_async16(%s + 2u * (tid + %du), a.v0 + (%s | ld_tid | jp[%d]));\n", buf, j * NT, bexpr, j);
        return r + "svj_cp_commit();\n";
    };
    pre += "float es = 0.f, ec = 0.f;\n";
    pre += issue("base", "tb0");
    body += "#pragma unroll 1\nfor (u32 cur = 0; t < ntiles; t += gridDim.x, cur ^= 1u) {\n";
    body += "const u64 bn = ((base | ~gmask) + pstep) & gmask;\n";
    if (NBUF == 2)
        body += "if (t + gridDim.x < ntiles) {\n" + issue("bn", "(cur ? tb0 : tb1)") + "svj_cp_wait1();\n} else {\nsvj_cp_wait0();\n}\n__syncthreads();\n";
    else
        body += "svj_cp_wait0();\n__syncthreads();\n";
    body += "const float2* const tb = cur ? tb1 : tb0;\n";
    for (int k = 0; k < K; ++k) body += fmt("const float2 %s = tb[te | %du];\n", amp(k).c_str(), (unsigned)k << L);
    body += "const u64 fix = base | tphys;\n";
    // diagonal: global-only terms give one weight per tile, mixed terms a signed sum
    // (the global-only terms are shared by every thread of the tile: lane i of each warp
    // evaluates terms i, i + 32, ..., then the warp sums them)
    if (d1 > d0) {
        int zq0 = -1, cf0 = -1;
        for (uint32_t i = d0; i < d1; ++i) {
            const int zi = A.Q(tl[i].zmask), c = A.F(tl[i].fre32);
            if (i == d0) zq0 = zi, cf0 = c;
        }
        body += "float wc = 0.f;\n{\nconst u32 ln = tid & 31u;\n";
        for (uint32_t c0 = 0; c0 < d1 - d0; c0 += 32) {
            const uint32_t m = std::min<uint32_t>(32u, d1 - d0 - c0);
            body += fmt("if (ln < %uu) {\nconst u32 j = %uu + ln;\nwc += (__popcll(base & a.q[%d + j]) & 1) ? -a.f[%d + j] : a.f[%d + j];\n}\n",
                        m, c0, zq0, cf0, cf0);
        }
        body += "#pragma unroll\nfor (int o = 16; o > 0; o >>= 1) wc += __shfl_xor_sync(0xffffffffu, wc, o);\n}\n";
    } else {
        body += "float wc = 0.f;\n";
    }
    body += "float e = 0.f;\n";
    for (int k = 0; k < K; ++k)
        body += fmt("e = fmaf(fmaf(%s.x, %s.x, %s.y * %s.y), w[%d] + wc, e);\n", amp(k).c_str(), amp(k).c_str(), amp(k).c_str(),
                    amp(k).c_str(), k);
    for (uint32_t i = d1; i < d2; ++i) {
        const svk::PauliTerm& pt = tl[i];
        const int zi = A.Q(pt.zmask), c = A.F(pt.fre32);
        body += fmt("{\nfloat m = 0.f;\n");
        for (int k = 0; k < K; ++k)
            body += fmt("m = fmaf(%s%s.x, %s.x, fmaf(%s%s.y, %s.y, m));\n", ((pt.smask >> k) & 1) ? "-" : "", amp(k).c_str(),
                        amp(k).c_str(), ((pt.smask >> k) & 1) ? "-" : "", amp(k).c_str(), amp(k).c_str());
        body += fmt("e = fmaf((__popcll(fix & a.q[%d]) & 1) ? -a.f[%d] : a.f[%d], m, e);\n}\n", zi, c, c);
    }
    // X / Y terms.  A term whose X / Y qubits are all register bits of the first layout
    // (tile bits L..L+R-1) pairs registers of that layout; one whose X / Y qubits are all
    // on the top R tile bits pairs registers of a second layout, in which a thread holds
    // the amplitudes along those bits (threads on tile bits 0..T-R-1, so the lanes still
    // read consecutive amplitudes); any other term reads its partners from the tile.
    const int RB0 = T - R;
    const bool lb = RB0 >= L + R;
    const uint32_t regmaskB = lb ? ((1u << R) - 1u) << RB0 : 0u;
    uint64_t regphysB = 0;
    for (int b = RB0; lb && b < T; ++b) regphysB |= sw.ptile[b];
    auto in_b = [&](const svk::PauliTerm& pt) { return lb && pt.xtile != 0 && (pt.xtile & ~regmaskB) == 0; };
    // a third layout for terms whose X / Y qubits are all among tile bits 0..L-1: a thread
    // holds the 2^L amplitudes of one run (threads on tile bits L..T-1); lane l reads
    // element j ^ (l mod 2^L) of its run into register j, so that the lanes of each load
    // fall on distinct banks; a term's partner is then register j ^ x, and the lane's
    // XOR enters only the Z sign (through the fixed-bit value, which includes it)
    const bool lc = L == R && T - L == T - R;
    auto in_c = [&](const svk::PauliTerm& pt) {
        return lc && pt.xtile != 0 && (pt.xtile & ~((1u << L) - 1u)) == 0 && !in_b(pt);
    };
    // one term: Re(f sum_k conj(a_k) s_k p_k), with p_k a register of the same layout
    // (xr: the term's X / Y bits among the layout's register bits) or a tile read
    auto emit_xy = [&](const svk::PauliTerm& pt, const char* vn, const char* fixn, uint32_t xr, uint32_t sm, bool noz,
                       uint32_t xthr) {
        const bool real = (pt.flags & svk::PT_REAL) != 0;
        const int cr = A.F(pt.fre32), ci = real ? -1 : A.F(pt.fim32);
        auto av = [&](int k) { return fmt("%s%d", vn, k); };
        body += "{\nfloat ar = 0.f, ai = 0.f;\n";
        const uint32_t low = xr & (~xr + 1u);
        if (xthr) body += fmt("const float2* const pb = tb + (te ^ %uu);\n", xthr);
        for (int k = 0; k < K; ++k) {
            if (!xthr && (k & (int)low)) continue;   // the pair's other amplitude: its conjugate term
            const std::string p = xthr ? fmt("pb[%du]", (unsigned)((k ^ xr) << L)) : av(k ^ (int)xr);
            const char* sg = ((sm >> k) & 1) ? "-" : "";
            if (xthr) body += fmt("{\nconst float2 p = %s;\n", p.c_str());
            const std::string pp = xthr ? std::string("p") : p;
            body += fmt("ar = fmaf(%s%s.x, %s.x, fmaf(%s%s.y, %s.y, ar));\n", sg, av(k).c_str(), pp.c_str(), sg, av(k).c_str(),
                        pp.c_str());
            if (!real)
                body += fmt("ai = fmaf(%s%s.x, %s.y, fmaf(%s%s.y, %s.x, ai));\n", sg, av(k).c_str(), pp.c_str(),
                            ((sm >> k) & 1) ? "" : "-", av(k).c_str(), pp.c_str());
            if (xthr) body += "}\n";
        }
        const std::string v = real ? fmt("a.f[%d] * ar", cr) : fmt("fmaf(a.f[%d], ar, -a.f[%d] * ai)", cr, ci);
        const float scale = xthr ? 1.f : 2.f;
        if (noz) body += fmt("e = fmaf(%.1ff, %s, e);\n", scale, v.c_str());
        else body += fmt("e = fmaf((__popcll(%s & a.q[%d]) & 1) ? %.1ff : %.1ff, %s, e);\n", fixn, A.Q(pt.zmask), -scale, scale,
                         v.c_str());
        body += "}\n";
    };
    bool any_b = false, any_c = false;
    for (uint32_t i = d2; i < nterm; ++i) {
        const svk::PauliTerm& pt = tl[i];
        if (in_b(pt)) {
            any_b = true;
            continue;
        }
        if (in_c(pt)) {
            any_c = true;
            continue;
        }
        emit_xy(pt, "x", "fix", pt.xreg, pt.smask, (pt.flags & svk::PT_NOZ) != 0, pt.xtile & ~regmask);
    }
    if (any_b) {
        pre += fmt("u64 tphysb = 0;\n#pragma unroll\nfor (int b = 0; b < %d; ++b)\nif ((tid >> b) & 1u) tphysb |= a.q[%d + b];\n",
                   RB0, QT);
        body += "{\n";
        for (int k = 0; k < K; ++k) body += fmt("const float2 y%d = tb[tid | %du];\n", k, (unsigned)k << RB0);
        body += "const u64 fixb = base | tphysb;\n";
        for (uint32_t i = d2; i < nterm; ++i) {
            const svk::PauliTerm& pt = tl[i];
            if (!in_b(pt)) continue;
            const uint32_t zr = (tmask(pt.zmask) & regmaskB) >> RB0;
            uint32_t sm = 0;
            for (int k = 0; k < K; ++k)
                if (__builtin_popcount((unsigned)k & zr) & 1) sm |= 1u << k;
            emit_xy(pt, "y", "fixb", pt.xtile >> RB0, sm, (pt.zmask & ~regphysB) == 0, 0u);
        }
        body += "}\n";
    }
    if (any_c) {
        pre += fmt("u64 tphysc = tid & %uu;\n#pragma unroll\nfor (int b = %d; b < %d; ++b)\nif ((tid >> (b - %d)) & 1u) tphysc |= a.q[%d + b];\n",
                   (1u << L) - 1u, L, T, L, QT);
        pre += fmt("const u32 tcx = (tid << %d) | (tid & %uu);\n", L, (1u << L) - 1u);
        body += "{\n";
        for (int k = 0; k < K; ++k) body += fmt("const float2 z%d = tb[tcx ^ %du];\n", k, k);
        body += "const u64 fixc = base | tphysc;\n";
        for (uint32_t i = d2; i < nterm; ++i) {
            const svk::PauliTerm& pt = tl[i];
            if (!in_c(pt)) continue;
            const uint32_t zr = (uint32_t)(pt.zmask & ((1u << L) - 1u));
            uint32_t sm = 0;
            for (int k = 0; k < K; ++k)
                if (__builtin_popcount((unsigned)k & zr) & 1) sm |= 1u << k;
            emit_xy(pt, "z", "fixc", pt.xtile, sm, pt.zmask == 0, 0u);
        }
        body += "}\n";
    }
    body += "{\nconst float y = e - ec, s2 = es + y;\nec = (s2 - es) - y;\nes = s2;\n}\n";
    body += "base = bn;\n__syncthreads();\n";
    if (NBUF == 1) body += "if (t + gridDim.x < ntiles) {\n" + issue("bn", "tb0") + "}\n";
    body += "}\n";
    // CTA partial in FP64, fixed order
    body += "double d = (double)es - (double)ec;\n";
    body += "#pragma unroll\nfor (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);\n";
    body += "__shared__ double s_w[32];\nif ((tid & 31u) == 0u) s_w[tid >> 5] = d;\n__syncthreads();\n";
    body += fmt("if (tid == 0) {\ndouble s2 = 0.0;\nfor (int i = 0; i < %d; ++i) s2 += s_w[i];\na.partial[blockIdx.x] = s2;\n}\n", NT / 32);
    // assemble (the argument block has the stage kernels' layout, so launch() serves both)
    const int nq = std::max<int>(1, (int)A.q.size()), nu = 1, nf = std::max<int>(1, (int)A.f.size());
    std::string src = "#include \"jit_prelude.cuh\"\n";
    src += fmt("struct alignas(64) Args {\nSvjTmap m0;\nSvjTmap m1;\nfloat2* v0;\nfloat2* v1;\ndouble* partial;\nint* flag;\n"
               "const double* params;\nconst u32* pofs;\nu64 ncirc;\nu64 q[%d];\nu32 u[%d];\nfloat f[%d];\n};\n", nq, nu, nf);
    src += "extern \"C\" __global__ void __launch_bounds__(" + std::to_string(NT) + ", " + std::to_string(MINB) +
           ") KNAME(const __grid_constant__ Args a) {\n"
           "extern __shared__ __attribute__((aligned(16))) unsigned char smem[];\n" + pre + body + "}\n";
    const std::string name = fmt("svj_pauli_%016llx", (unsigned long long)fnv1a(src));
    size_t pos;
    while ((pos = src.find("KNAME")) != std::string::npos) src.replace(pos, 5, name);
    B->src = src;
    B->name = name;
    B->nthr = (uint32_t)NT;
    B->n_slots = 1;
    B->ntiles = 1ull << NG;
    B->tma = false;
    size_t bytes = kArgQ + 8 * (size_t)nq + 4 * (size_t)nu;
    bytes = (bytes + 3) & ~(size_t)3;
    const size_t off_f = bytes;
    bytes += 4 * (size_t)nf;
    bytes = (bytes + 63) & ~(size_t)63;
    if (bytes > 32000) return "pauli jit: terms exceed the kernel argument space";
    B->smem = (uint32_t)((8u * NBUF) << T);   // tile buffers of 2^T complex64
    B->args.assign(bytes, 0);
    std::memcpy(B->args.data() + kArgQ, A.q.data(), 8 * A.q.size());
    std::memcpy(B->args.data() + off_f, A.f.data(), 4 * A.f.size());
    return "";
}

}  // namespace svj
