// Host emulator of the packed forward program (test infrastructure).  Runs the
// library's host planner (SWAP relabel, closeness-centrality partition, lowering into
// register groups and micro-ops, packing) on a circuit and executes the packed device
// program tile by tile, thread by thread, in double precision, following the op
// semantics the kernels implement.  The test compares the result with the CPU oracle,
// so the lowering is checked on the CPU.
//
//   stage_emu fwd  <in.bin> <out.bin>     forward program
//   stage_emu grad <in.bin> <out.bin>     forward, lambda = O psi, adjoint program
//   stage_emu bind <in.bin> <out.bin>     as grad, lowered the way batches are: the
//                                         parametric rotations stay symbolic (bound
//                                         dense ops) and their matrices are formed from
//                                         the parameters after packing
//   stage_emu gemm <in.bin> <out.bin>     tensor-core plan (header L = fusion width k,
//                                         rmax = precision 1 TF32x3 / 2 BF16x3): each
//                                         stage's B operand is decoded from the packed
//                                         blob (hi + lo halves, 128-byte-swizzled rows)
//                                         and applied to every state column in FP64;
//                                         out: double n_stages, then the state
// in:  int32 n, L, n_fixed, n_params, n_gates, elem_bytes (8 | 16), rmax;
//      n_params doubles; n_gates x (int32 kind, nq, q0, q1, param; double a0, a1, a2);
//      2^n x (re, im) doubles (the input state);
//      grad only: int32 n_terms; n_terms x (double coeff, n uint8 Pauli codes 0..3 = I X Y Z)
// out: fwd:  2^n x (re, im) doubles in canonical qubit order;
//      grad: double E, n_params doubles dE/dtheta, then the state after the adjoint
//      program (the input state again) as 2^n x (re, im) doubles;
//      exit status 0, or 2 with a message on stderr when the planner rejects the circuit
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "gemm.h"
#include "hier.h"
#include "planner.h"

using namespace svh;
using namespace svk;
typedef std::complex<double> cd;

static double ang(uint32_t k) { return (double)(int32_t)k * (2 * M_PI / 4294967296.0); }
static double ang(double a) { return a; }
static uint64_t deposit(uint64_t x, const uint8_t* pos, int n) {
    uint64_t r = 0;
    for (int i = 0; i < n; ++i)
        if ((x >> i) & 1) r |= 1ull << pos[i];
    return r;
}

// lam / slot_param / grad: adjoint programs carry lambda beside psi and accumulate
// gradient ops (slot += Im <lam| P |psi>) into grad[slot_param[slot]]
// bound: the parameters of bound dense ops (F_BIND: term_off = parameter index, u = the
// rotation kind, | BK_DAGGER for the adjoint, i.e. the angle negated), whose matrices
// are written from the rotations' definitions, RX(t) = [[c, -i s], [-i s, c]],
// RY(t) = [[c, -s], [s, c]], RZ(t) = diag(e^{-i t/2}, e^{i t/2}) with c = cos(t/2),
// s = sin(t/2)
template <typename Real>
static void run_packed(const Program& prog, int n, std::vector<cd>& psi, std::vector<cd>* lam = nullptr,
                       std::vector<double>* grad = nullptr, const double* bound = nullptr) {
    Packed pk;
    std::string err = pack(prog, n, sizeof(Real) == 8 ? 16 : 8, &pk);
    if (!err.empty()) {
        fprintf(stderr, "pack: %s\n", err.c_str());
        exit(2);
    }
    if (bound) {
        DevOp<Real>* bops = (DevOp<Real>*)(pk.blob.data() + pk.op_off);
        for (size_t i = 0; i < pk.n_ops; ++i) {
            DevOp<Real>& o = bops[i];
            if (!(o.flags & F_BIND)) continue;
            const double t = (o.u & BK_DAGGER) ? -bound[o.term_off] : bound[o.term_off];
            const cd c(std::cos(0.5 * t), 0), is(0, std::sin(0.5 * t));
            cd M[4];
            switch (o.u & 3) {
                case BK_RX: M[0] = c; M[1] = -is; M[2] = -is; M[3] = c; break;
                case BK_RY: M[0] = c; M[1] = -std::sin(0.5 * t); M[2] = std::sin(0.5 * t); M[3] = c; break;
                default: M[0] = c - is; M[1] = 0; M[2] = 0; M[3] = c + is; break;   // BK_RZ
            }
            for (int e = 0; e < 4; ++e) {
                o.m[2 * e] = (Real)M[e].real();
                o.m[2 * e + 1] = (Real)M[e].imag();
            }
        }
    }
    const uint8_t* b = pk.blob.data();
    const Stage* stages = (const Stage*)(b + pk.stage_off);
    const Group* groups = (const Group*)(b + pk.group_off);
    const DevOp<Real>* ops = (const DevOp<Real>*)(b + pk.op_off);
    const DevTerm<Real>* terms = (const DevTerm<Real>*)(b + pk.term_off);
    const PhaseSlot<Real>* slots = (const PhaseSlot<Real>*)(b + pk.slot_off);
    for (size_t si = 0; si < pk.stages.size(); ++si) {
        const Stage& st = stages[si];
        const int R = (int)st.R, TR = (int)st.T - R;
        for (uint64_t tile = 0; tile < (1ull << st.n_glob); ++tile) {
            const uint64_t base = deposit(tile, st.glob_pos, (int)st.n_glob);
            std::vector<double> wg(st.n_phase);   // per-tile angle of each phase slot
            for (uint32_t p = 0; p < st.n_phase; ++p) {
                const PhaseSlot<Real>& ps = slots[st.phase_off + p];
                double a = ang(ps.cangle);
                for (uint32_t i = 0; i < ps.n_glob; ++i)
                    if (base & terms[ps.glob_off + i].mask) a += ang(terms[ps.glob_off + i].angle);
                wg[p] = a;
            }
            for (uint32_t gi = 0; gi < st.n_groups; ++gi) {
                const Group& G = groups[st.group_off + gi];
                for (uint32_t tid = 0; tid < (1u << TR); ++tid) {
                    uint64_t fix = base;
                    for (int i = 0; i < TR; ++i)
                        if ((tid >> i) & 1) fix |= 1ull << st.tile_pos[G.thr_pos[i]];
                    const int NV = lam ? 2 : 1;
                    std::vector<uint64_t> addr(1u << R);
                    std::vector<cd> av[2] = {std::vector<cd>(1u << R), std::vector<cd>(1u << R)};
                    for (int k = 0; k < (1 << R); ++k) {
                        uint64_t x = fix;
                        for (int j = 0; j < R; ++j)
                            if ((k >> j) & 1) x |= 1ull << st.tile_pos[G.reg_pos[j]];
                        addr[k] = x;
                        av[0][k] = psi[x];
                        if (lam) av[1][k] = (*lam)[x];
                    }
                    for (uint32_t oi = 0; oi < G.n_ops; ++oi) {
                        const DevOp<Real>& o = ops[st.op_off + G.op_off + oi];
                        if (o.type >= OP_GRAD_X) {
                            if (!lam) {
                                fprintf(stderr, "gradient op in a forward program\n");
                                exit(3);
                            }
                            const std::vector<cd>&ps = av[0], &la = av[1];
                            double acc = 0;
                            if (o.type == OP_GRAD_Z && o.u) {   // Z on the bit in ctrl_fix: one sign per thread
                                for (int k = 0; k < (1 << R); ++k) acc += std::imag(std::conj(la[k]) * ps[k]);
                                if (fix & o.ctrl_fix) acc = -acc;
                            } else {
                                for (int k = 0; k < (1 << R); ++k) {
                                    if ((k >> o.j) & 1) continue;
                                    const int k1 = k | (1 << o.j);
                                    if (o.type == OP_GRAD_X)
                                        acc += std::imag(std::conj(la[k]) * ps[k1] + std::conj(la[k1]) * ps[k]);
                                    else if (o.type == OP_GRAD_Y)
                                        acc += std::imag(std::conj(la[k]) * cd(0, -1) * ps[k1] + std::conj(la[k1]) * cd(0, 1) * ps[k]);
                                    else
                                        acc += std::imag(std::conj(la[k]) * ps[k] - std::conj(la[k1]) * ps[k1]);
                                }
                            }
                            (*grad)[st.slot_off + o.slot] += acc;
                            continue;
                        }
                        for (int v = 0; v < NV; ++v) {
                        std::vector<cd>& a = av[v];
                        cd M[4] = {cd(o.m[0], o.m[1]), cd(o.m[2], o.m[3]), cd(o.m[4], o.m[5]), cd(o.m[6], o.m[7])};
                        if (o.type == OP_UR) {
                            M[0] = o.m[0];
                            M[1] = o.m[2];
                            M[2] = o.m[4];
                            M[3] = o.m[6];
                        }
                        // the op's phase factor: a phase slot (per-tile angle plus the thread
                        // bits' part), or a constant with optional per-thread terms
                        auto phase = [&]() {
                            if (o.flags & F_SLOT) {
                                double x = wg[o.slot];
                                const PhaseSlot<Real>& ps = slots[st.phase_off + o.slot];
                                for (int i = 0; i < TR; ++i)
                                    if ((tid >> i) & 1) x += ang(ps.J[i]);
                                return std::polar(1.0, x);
                            }
                            cd w = (o.flags & F_TW) ? cd(1, 0) : cd(o.m[0], o.m[1]);
                            if (o.flags & F_TERMS) {
                                double x = 0;
                                for (uint32_t i = 0; i < o.n_terms; ++i) {
                                    const uint64_t m = terms[o.term_off + i].mask;
                                    if ((fix & m) == m) x += ang(terms[o.term_off + i].angle);
                                }
                                w *= std::polar(1.0, x);
                            }
                            return w;
                        };
                        if (o.type <= OP_X) {
                            if ((fix & o.ctrl_fix) != o.ctrl_fix) continue;
                            if (o.flags & F_PAIRS) {   // pair phases on the target's |1> half
                                const cd w0 = (o.flags & F_TW) ? phase() : cd(1, 0);
                                double pa[3];
                                for (int i = 0; i < 3; ++i) {
                                    typename AngT<Real>::type t;
                                    memcpy(&t, &o.m[1 + 2 * i], sizeof(t));
                                    pa[i] = ang(t);
                                }
                                for (int k = 0; k < (1 << R); ++k) {
                                    if (!((k >> o.j) & 1)) continue;
                                    const int kk = k & ~(1 << o.j);
                                    const int c = (kk & ((1 << o.j) - 1)) | ((kk >> (o.j + 1)) << o.j);
                                    double ph = 0;
                                    for (int i = 0; i < R - 1; ++i)
                                        if ((c >> i) & 1) ph += pa[i];
                                    a[k] *= w0 * std::polar(1.0, ph);
                                }
                            } else if (o.flags & F_TW) {
                                const cd w = phase();
                                for (int k = 0; k < (1 << R); ++k)
                                    if ((k >> o.j) & 1) a[k] *= w;
                            }
                            for (int k = 0; k < (1 << R); ++k) {
                                if ((k >> o.j) & 1) continue;
                                if ((k & (int)o.ctrl_reg) != (int)o.ctrl_reg) continue;
                                const int k1 = k | (1 << o.j);
                                const cd x0 = a[k], x1 = a[k1];
                                if (o.type == OP_X) {
                                    a[k] = x1;
                                    a[k1] = x0;
                                } else {
                                    a[k] = M[0] * x0 + M[1] * x1;
                                    a[k1] = M[2] * x0 + M[3] * x1;
                                }
                            }
                        } else if (o.type == OP_PHASE1) {
                            const cd w = phase();
                            for (int k = 0; k < (1 << R); ++k)
                                if ((k >> o.j) & 1) a[k] *= w;
                        } else if (o.type == OP_PHASE2) {
                            const cd w(o.m[0], o.m[1]);
                            for (int k = 0; k < (1 << R); ++k)
                                if (((k >> o.j) & 1) && ((k >> o.u) & 1)) a[k] *= w;
                        } else if (o.type == OP_PHASE0) {
                            const cd w = phase();
                            for (int k = 0; k < (1 << R); ++k) a[k] *= w;
                        } else {
                            fprintf(stderr, "unknown op type %d\n", (int)o.type);
                            exit(3);
                        }
                        }
                    }
                    for (int k = 0; k < (1 << R); ++k) {
                        psi[addr[k]] = av[0][k];
                        if (lam) (*lam)[addr[k]] = av[1][k];
                    }
                }
            }
        }
    }
}

// Tensor-core stages: D = X Ut^T per column (X: the column's 2^keff local amplitudes as
// interleaved (re, im) floats; Ut: the real embedding of the fused unitary, read back as
// hi + lo from the 128-byte-swizzled K-major blob).
static void run_gemm(const GemmProgram& gp, int prec, int n, std::vector<cd>& psi) {
    auto sw = [](uint32_t r, uint32_t b) -> size_t {   // byte b of row r in an operand block
        return (size_t)(r / 8) * 1024 + (r % 8) * 128 + ((((b / 16) ^ (r % 8)) % 8) * 16) + b % 16;
    };
    for (const GemmStage& st : gp.stages) {
        const uint32_t N = st.N, kc = prec == 1 ? 32u : 64u;   // K elements per chunk
        const size_t block = (size_t)N * 128;
        const uint8_t* base = gp.ublob.data() + st.b_off;
        std::vector<double> U((size_t)N * N);
        for (uint32_t r = 0; r < N; ++r)
            for (uint32_t kk = 0; kk < N; ++kk) {
                const uint8_t* ch = base + (size_t)(kk / kc) * st.b_chunk_bytes;
                const uint32_t kl = kk % kc;
                double v = 0;
                for (int half = 0; half < 2; ++half) {
                    const uint8_t* q = ch + half * block;
                    if (prec == 1) {
                        float x;
                        memcpy(&x, q + sw(r, kl * 4), 4);
                        v += x;
                    } else {
                        uint16_t h;
                        memcpy(&h, q + sw(r, kl * 2), 2);
                        const uint32_t b = (uint32_t)h << 16;   // bfloat16: the top half of an FP32
                        float x;
                        memcpy(&x, &b, 4);
                        v += x;
                    }
                }
                U[(size_t)r * N + kk] = v;
            }
        const uint32_t D = 1u << st.keff;
        std::vector<double> x(N), y(N);
        for (uint64_t g = 0; g < (1ull << st.n_glob); ++g)
            for (uint64_t c = 0; c < (1ull << st.ncol_bits); ++c) {
                const uint64_t col = deposit(g, st.glob_pos, (int)st.n_glob) | deposit(c, st.col_pos, (int)st.ncol_bits);
                for (uint32_t j = 0; j < D; ++j) {
                    const cd a = psi[col | deposit(j, st.local_pos, (int)st.keff)];
                    x[2 * j] = a.real();
                    x[2 * j + 1] = a.imag();
                }
                for (uint32_t r = 0; r < N; ++r) {
                    double acc = 0;
                    for (uint32_t kk = 0; kk < N; ++kk) acc += U[(size_t)r * N + kk] * x[kk];
                    y[r] = acc;
                }
                for (uint32_t j = 0; j < D; ++j) psi[col | deposit(j, st.local_pos, (int)st.keff)] = cd(y[2 * j], y[2 * j + 1]);
            }
    }
}


// The hierarchical tensor-core stage, emulated byte for byte: every tile's amplitudes are
// split into (hi, lo) halves and stored at the A-operand offsets the layout tables give,
// the operands are read back through the 128-byte-swizzled K-major layout, each
// sub-partition's three products are summed in double, and the epilogue stores through
// the next layout (the last one into the FP32 output tile, read back by its own table).
static float emu_tf32(float x) {
    uint32_t b;
    memcpy(&b, &x, 4);
    b = (b + 0x0FFFu + ((b >> 13) & 1u)) & 0xFFFFE000u;
    memcpy(&x, &b, 4);
    return x;
}
static float emu_bf16(float x) {
    uint32_t b;
    memcpy(&b, &x, 4);
    b = (b + 0x7FFFu + ((b >> 16) & 1u)) & 0xFFFF0000u;
    memcpy(&x, &b, 4);
    return x;
}
static void run_hier(const HierProgram& hp, int prec, std::vector<cd>& psi) {
    const bool tf32 = prec == 1;
    auto sw = [](uint32_t r, uint32_t b) -> size_t {
        return (size_t)(r / 8) * 1024 + (r % 8) * 128 + ((((b / 16) ^ (r % 8)) % 8) * 16) + b % 16;
    };
    auto rnd = [&](float x) { return tf32 ? emu_tf32(x) : emu_bf16(x); };
    const uint32_t esz = tf32 ? 4 : 2, kc = tf32 ? 32u : 64u;
    for (const HierStage& st : hp.launches) {
        const uint32_t T = st.T, N = st.N, K = N, D2 = 1u << st.k;
        auto off = [&](int layout, uint32_t x) {
            uint32_t o = 0;
            for (uint32_t b = 0; b < T; ++b)
                if ((x >> b) & 1) o ^= st.ao[layout][b];
            return o;
        };
        // operand element store / load (byte images of hi / lo halves)
        std::vector<uint8_t> A(st.a_bytes);
        auto put = [&](uint32_t o, float v) {   // v at A offset o: hi there, lo 16384 above
            const float hi = rnd(v), lo = rnd(v - hi);
            if (tf32) {
                memcpy(&A[o], &hi, 4);
                memcpy(&A[o + 16384], &lo, 4);
            } else {
                uint32_t bh, bl;
                memcpy(&bh, &hi, 4);
                memcpy(&bl, &lo, 4);
                const uint16_t h = (uint16_t)(bh >> 16), l = (uint16_t)(bl >> 16);
                memcpy(&A[o], &h, 2);
                memcpy(&A[o + 16384], &l, 2);
            }
        };
        auto get = [&](const uint8_t* p) -> double {
            if (tf32) {
                float x;
                memcpy(&x, p, 4);
                return x;
            }
            uint16_t h;
            memcpy(&h, p, 2);
            const uint32_t b = (uint32_t)h << 16;
            float x;
            memcpy(&x, &b, 4);
            return x;
        };
        std::vector<double> Ah(128 * K), Al(128 * K), Bh((size_t)N * K), Bl((size_t)N * K), Dm(128 * N);
        std::vector<double> outre(1u << T), outim(1u << T);
        for (uint64_t g = 0; g < (1ull << st.n_glob); ++g) {
            const uint64_t base = deposit(g, st.glob_pos, (int)st.n_glob);
            for (uint32_t x = 0; x < (1u << T); ++x) {   // load: pair element x at layout 0
                const cd a = psi[base | deposit(x, st.tile_pos, (int)T)];
                const uint32_t o = off(0, x);
                put(o, (float)a.real());
                put(o + esz, (float)a.imag());
            }
            for (uint32_t s = 0; s < st.n_sub; ++s) {
                const uint8_t* B = hp.ublob.data() + st.b_off + (size_t)s * st.b_bytes;
                for (uint32_t r = 0; r < 128; ++r)
                    for (uint32_t kk = 0; kk < K; ++kk) {
                        const size_t o = (size_t)(kk / kc) * 32768 + sw(r, (kk % kc) * esz);
                        Ah[r * K + kk] = get(&A[o]);
                        Al[r * K + kk] = get(&A[o + 16384]);
                    }
                for (uint32_t r = 0; r < N; ++r)
                    for (uint32_t kk = 0; kk < K; ++kk) {
                        const size_t o = (size_t)(kk / kc) * 2 * N * 128 + sw(r, (kk % kc) * esz);
                        Bh[r * K + kk] = get(B + o);
                        Bl[r * K + kk] = get(B + o + (size_t)N * 128);
                    }
                for (uint32_t m = 0; m < 128; ++m)
                    for (uint32_t c = 0; c < N; ++c) {
                        double acc = 0;
                        for (uint32_t kk = 0; kk < K; ++kk)
                            acc += Ah[m * K + kk] * Bh[c * K + kk] + Al[m * K + kk] * Bh[c * K + kk] +
                                   Ah[m * K + kk] * Bl[c * K + kk];
                        Dm[m * N + c] = (float)acc;   // the accumulator is FP32
                    }
                for (uint32_t m = 0; m < 128; ++m)
                    for (uint32_t j = 0; j < D2; ++j) {
                        const uint32_t x = (uint32_t)(deposit(m, st.col_bits[s], 7) | deposit(j, st.amp_bits[s], (int)st.k));
                        const double re = Dm[m * N + 2 * j], im = Dm[m * N + 2 * j + 1];
                        if (s + 1 < st.n_sub) {
                            const uint32_t o = off((int)s + 1, x);
                            put(o, (float)re);
                            put(o + esz, (float)im);
                        } else {
                            const uint32_t o = off((int)st.n_sub, x) / 8;
                            outre[o] = re;
                            outim[o] = im;
                        }
                    }
            }
            for (uint32_t x = 0; x < (1u << T); ++x) {
                const uint32_t o = off((int)st.n_sub, x) / 8;
                psi[base | deposit(x, st.tile_pos, (int)T)] = cd(outre[o], outim[o]);
            }
        }
    }
}

template <typename T>
static T rd(FILE* f) {
    T v;
    if (fread(&v, sizeof(T), 1, f) != 1) {
        fprintf(stderr, "short input\n");
        exit(1);
    }
    return v;
}

int main(int argc, char** argv) {
    if (argc != 4 || (strcmp(argv[1], "fwd") != 0 && strcmp(argv[1], "grad") != 0 && strcmp(argv[1], "bind") != 0 &&
                      strcmp(argv[1], "gemm") != 0 && strcmp(argv[1], "fuse") != 0 && strcmp(argv[1], "hier") != 0)) {
        fprintf(stderr, "usage: stage_emu fwd|grad|bind|gemm|fuse|hier in.bin out.bin\n");
        return 1;
    }
    const bool bind = strcmp(argv[1], "bind") == 0;
    const bool hier = strcmp(argv[1], "hier") == 0;   // L = k + 7, strict, qubits 0..3 fixed
    const bool gemm = hier || strcmp(argv[1], "gemm") == 0;
    const bool fuse = strcmp(argv[1], "fuse") == 0;   // forward with the output-permutation retile
    const bool want_grad = bind || strcmp(argv[1], "grad") == 0;
    FILE* f = fopen(argv[2], "rb");
    if (!f) return 1;
    const int n = rd<int32_t>(f), L = rd<int32_t>(f), nf = rd<int32_t>(f), np = rd<int32_t>(f);
    const int ng = rd<int32_t>(f), eb = rd<int32_t>(f), rmax = rd<int32_t>(f);
    std::vector<double> params(np);
    for (auto& p : params) p = rd<double>(f);
    Plan P;
    P.n = n;
    P.n_params = np;
    P.L = L;
    P.n_fixed = nf;
    for (int i = 0; i < ng; ++i) {
        GateRec g;
        g.kind = rd<int32_t>(f);
        g.nq = rd<int32_t>(f);
        g.q[0] = rd<int32_t>(f);
        g.q[1] = rd<int32_t>(f);
        g.param = rd<int32_t>(f);
        for (int k = 0; k < 3; ++k) g.angle[k] = rd<double>(f);
        P.gates.push_back(g);
    }
    std::vector<cd> psi(1ull << n);
    for (auto& x : psi) {
        const double re = rd<double>(f), im = rd<double>(f);
        x = cd(re, im);
    }
    std::vector<double> coeff;
    std::vector<std::vector<uint8_t>> pauli;
    if (want_grad) {
        const int nt = rd<int32_t>(f);
        for (int t = 0; t < nt; ++t) {
            coeff.push_back(rd<double>(f));
            std::vector<uint8_t> c(n);
            for (int q = 0; q < n; ++q) c[q] = rd<uint8_t>(f);
            pauli.push_back(c);
        }
    }
    fclose(f);
    relabel(n, P.gates, &P.phys, &P.final_map);
    if (bind)   // a bound RZ is a dense op: its qubit must be local
        for (size_t g = 0; g < P.gates.size(); ++g)
            if (P.gates[g].kind == K_RZ && P.gates[g].param >= 0) P.phys[g].bound = true;
    const uint64_t fixed = (nf && (!gemm || hier)) ? ((1ull << nf) - 1) : 0;
    std::string err = partition_core(n, P.phys, L, fixed, (1ull << n) - 1, &P.top, &P.cc, gemm);
    if (!err.empty()) {
        fprintf(stderr, "partition: %s\n", err.c_str());
        return 2;
    }
    if (hier) {
        P.n_fixed = nf;
        HierProgram hp;
        err = plan_hier(P, np ? params.data() : nullptr, rmax, &hp);
        if (!err.empty()) {
            fprintf(stderr, "plan_hier: %s\n", err.c_str());
            return 2;
        }
        run_hier(hp, rmax, psi);
        FILE* o = fopen(argv[3], "wb");
        if (!o) return 1;
        const double nst = (double)hp.n_sub;
        fwrite(&nst, sizeof(double), 1, o);
        for (uint64_t y = 0; y < psi.size(); ++y) {   // physical -> canonical order
            uint64_t x = 0;
            for (int q = 0; q < n; ++q)
                if ((y >> q) & 1) x |= 1ull << P.final_map[q];
            const double v[2] = {psi[x].real(), psi[x].imag()};
            fwrite(v, sizeof(double), 2, o);
        }
        fclose(o);
        return 0;
    }
    if (gemm) {
        P.gemm_k = L;
        GemmProgram gp;
        err = plan_gemm(P, np ? params.data() : nullptr, rmax, &gp);
        if (!err.empty()) {
            fprintf(stderr, "plan_gemm: %s\n", err.c_str());
            return 2;
        }
        run_gemm(gp, rmax, n, psi);
        FILE* o = fopen(argv[3], "wb");
        if (!o) return 1;
        const double nst = (double)gp.stages.size();
        fwrite(&nst, sizeof(double), 1, o);
        for (uint64_t y = 0; y < psi.size(); ++y) {   // physical -> canonical order
            uint64_t x = 0;
            for (int q = 0; q < n; ++q)
                if ((y >> q) & 1) x |= 1ull << P.final_map[q];
            const double v[2] = {psi[x].real(), psi[x].imag()};
            fwrite(v, sizeof(double), 2, o);
        }
        fclose(o);
        return 0;
    }
    Program prog;
    const double* lp = (np && !bind) ? params.data() : nullptr;   // bind: parameters stay symbolic
    const double* bp = (np && bind) ? params.data() : nullptr;
    err = lower(P, lp, eb, rmax, false, &prog, bind, 0, fuse);
    if (!err.empty()) {
        fprintf(stderr, "lower: %s\n", err.c_str());
        return 2;
    }
    if (eb == 8) run_packed<float>(prog, n, psi, nullptr, nullptr, bp);
    else run_packed<double>(prog, n, psi, nullptr, nullptr, bp);
    FILE* o = fopen(argv[3], "wb");
    if (!o) return 1;
    if (want_grad) {
        // lambda = O psi in the physical layout (qubit q sits at bit final_map[q]);
        // (P psi)_x = f(x) psi_{x ^ xmask} for a Pauli string P
        const uint64_t dim = psi.size();
        std::vector<cd> lam(dim, 0.0);
        for (size_t t = 0; t < pauli.size(); ++t) {
            uint64_t xm = 0;
            for (int q = 0; q < n; ++q)
                if (pauli[t][q] == 1 || pauli[t][q] == 2) xm |= 1ull << P.final_map[q];
            for (uint64_t x = 0; x < dim; ++x) {
                const uint64_t y = x ^ xm;   // (P psi)_x = prod_q p_q(x_q <- y_q) psi_y
                cd f = coeff[t];
                for (int q = 0; q < n; ++q) {
                    const int bx = (int)((x >> P.final_map[q]) & 1);
                    if (pauli[t][q] == 2) f *= bx ? cd(0, 1) : cd(0, -1);   // Y|0> = i|1>, Y|1> = -i|0>
                    else if (pauli[t][q] == 3 && bx) f = -f;
                }
                lam[x] += f * psi[y];
            }
        }
        double E = 0;
        for (uint64_t x = 0; x < dim; ++x) E += std::real(std::conj(psi[x]) * lam[x]);
        Program bprog;
        err = lower(P, lp, eb, rmax, true, &bprog, bind);
        if (!err.empty()) {
            fprintf(stderr, "lower (adjoint): %s\n", err.c_str());
            return 2;
        }
        std::vector<double> slots(bprog.slot_param.size(), 0.0), grad(np, 0.0);
        if (eb == 8) run_packed<float>(bprog, n, psi, &lam, &slots, bp);
        else run_packed<double>(bprog, n, psi, &lam, &slots, bp);
        for (size_t i = 0; i < slots.size(); ++i) grad[bprog.slot_param[i]] += slots[i];
        fwrite(&E, sizeof(double), 1, o);
        fwrite(grad.data(), sizeof(double), grad.size(), o);
        for (uint64_t x = 0; x < dim; ++x) {
            const double v[2] = {psi[x].real(), psi[x].imag()};
            fwrite(v, sizeof(double), 2, o);
        }
        fclose(o);
        return 0;
    }
    for (uint64_t y = 0; y < psi.size(); ++y) {   // physical -> canonical order
        uint64_t x = 0;
        for (int q = 0; q < n; ++q)
            if ((y >> q) & 1) x |= 1ull << P.final_map[q];
        const double v[2] = {psi[x].real(), psi[x].imag()};
        fwrite(v, sizeof(double), 2, o);
    }
    fclose(o);
    return 0;
}
