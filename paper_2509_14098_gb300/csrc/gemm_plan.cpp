// gemm_plan.cpp — host side of the split-precision tensor-core stage.
//
// A plan partitioned without exemptions (every gate's qubits local) makes each
// partition one fixed unitary U on its k local qubits.  U is formed in FP64 by
// applying the partition's gates, in order, to the 2^k basis vectors (local index bit
// j = the j-th lowest local physical bit).  Its real embedding acts on columns of
// interleaved (re, im) floats: Ut[2i+a][2j+b] = Re U_ij if a == b, Im U_ij if (a, b) =
// (1, 0), -Im U_ij if (a, b) = (0, 1).  Ut is split as Ut ~ hi + lo with both halves
// rounded to nearest (TF32: hi = rn(x), lo = rn(x - hi); BF16 likewise) and stored per
// K chunk of 128 bytes per row in the tensor cores' 128-byte-swizzled K-major layout.
#include <algorithm>
#include <cmath>
#include <functional>
#include <complex>
#include <cstring>
#include <vector>

#include "gemm.h"
#include "planner.h"

namespace svh {

typedef std::complex<double> cd;

static void gate_full(const GateRec& g, const double* params, int* nq, cd m[16]) {
    auto th = [&](int i) { return g.param >= 0 ? params[g.param] : g.angle[i]; };
    const cd I(0, 1);
    const double r = 1.0 / std::sqrt(2.0);
    cd u[4] = {1, 0, 0, 1};
    *nq = kind_nq(g.kind);
    switch (g.kind) {
        case K_H: u[0] = r; u[1] = r; u[2] = r; u[3] = -r; break;
        case K_X: case K_CX: u[0] = 0; u[1] = 1; u[2] = 1; u[3] = 0; break;
        case K_Y: case K_CY: u[0] = 0; u[1] = -I; u[2] = I; u[3] = 0; break;
        case K_Z: case K_CZ: u[3] = -1; break;
        case K_S: u[3] = I; break;
        case K_SDG: u[3] = -I; break;
        case K_T: u[3] = std::polar(1.0, M_PI / 4); break;
        case K_TDG: u[3] = std::polar(1.0, -M_PI / 4); break;
        case K_RX: { double c = std::cos(th(0) / 2), s = std::sin(th(0) / 2); u[0] = c; u[1] = -I * s; u[2] = -I * s; u[3] = c; break; }
        case K_RY: { double c = std::cos(th(0) / 2), s = std::sin(th(0) / 2); u[0] = c; u[1] = -s; u[2] = s; u[3] = c; break; }
        case K_RZ: u[0] = std::polar(1.0, -th(0) / 2); u[3] = std::polar(1.0, th(0) / 2); break;
        case K_P: case K_CP: u[3] = std::polar(1.0, th(0)); break;
        case K_U3: {
            double t = g.angle[0], p = g.angle[1], l = g.angle[2];
            u[0] = std::cos(t / 2); u[1] = -std::polar(1.0, l) * std::sin(t / 2);
            u[2] = std::polar(1.0, p) * std::sin(t / 2); u[3] = std::polar(1.0, p + l) * std::cos(t / 2);
            break;
        }
        default: break;
    }
    if (*nq == 1) {
        for (int i = 0; i < 4; ++i) m[i] = u[i];
        return;
    }
    // two-qubit: index 2*b(q0) + b(q1); controlled gates act with u on q1 when q0 = 1
    for (int i = 0; i < 16; ++i) m[i] = 0;
    if (g.kind == K_SWAP) {
        m[0] = 1; m[1 * 4 + 2] = 1; m[2 * 4 + 1] = 1; m[15] = 1;
        return;
    }
    m[0] = 1; m[5] = 1;
    m[2 * 4 + 2] = u[0]; m[2 * 4 + 3] = u[1]; m[3 * 4 + 2] = u[2]; m[3 * 4 + 3] = u[3];
}

// round to the nearest TF32 value (ties to even)
static float rn_tf32(float x) {
    uint32_t b;
    std::memcpy(&b, &x, 4);
    b = (b + 0x0FFFu + ((b >> 13) & 1u)) & 0xFFFFE000u;
    float r;
    std::memcpy(&r, &b, 4);
    return r;
}
static void split_tf32(float x, float* hi, float* lo) {
    *hi = rn_tf32(x);
    *lo = rn_tf32(x - *hi);
}
static uint16_t to_bf16(float x) {   // round to nearest even
    uint32_t b;
    std::memcpy(&b, &x, 4);
    uint32_t r = b + 0x7FFFu + ((b >> 16) & 1u);
    return (uint16_t)(r >> 16);
}
static float from_bf16(uint16_t h) {
    uint32_t b = (uint32_t)h << 16;
    float x;
    std::memcpy(&x, &b, 4);
    return x;
}

// 128-byte-swizzled K-major position of byte b of row r inside one operand block
static size_t sw128(uint32_t r, uint32_t b) {
    return (size_t)(r >> 3) * 1024 + (r & 7) * 128 + ((((b >> 4) ^ (r & 7)) & 7) << 4) + (b & 15);
}

std::string fuse_unitary(const Plan& P, const std::vector<uint32_t>& ids, const int* lp, int k, const double* params,
                         std::vector<cd>* Uout) {
    const int D = 1 << k;
    int lidx[64];
    for (int b = 0; b < 64; ++b) lidx[b] = -1;
    for (int j = 0; j < k; ++j) lidx[lp[j]] = j;
    std::vector<cd>& U = *Uout;
    U.assign((size_t)D * D, 0.0);
    for (int c = 0; c < D; ++c) U[(size_t)c * D + c] = 1.0;   // column-major: U[col][row]
    for (uint32_t gi : ids) {
        const GateRec& g = P.gates[gi];
        const PGate& pg = P.phys[gi];
        if (g.kind == K_SWAP) continue;   // relabel
        int nq;
        cd m[16];
        gate_full(g, params, &nq, m);
        if (nq == 1) {
            const int q = lidx[pg.p[0]];
            if (q < 0) return "internal: gate outside the local set";
            for (int c = 0; c < D; ++c) {
                cd* col = &U[(size_t)c * D];
                for (int i = 0; i < D; ++i)
                    if (!((i >> q) & 1)) {
                        cd a0 = col[i], a1 = col[i | (1 << q)];
                        col[i] = m[0] * a0 + m[1] * a1;
                        col[i | (1 << q)] = m[2] * a0 + m[3] * a1;
                    }
            }
        } else {
            const int q0 = lidx[pg.p[0]], q1 = lidx[pg.p[1]];
            if (q0 < 0 || q1 < 0) return "internal: gate outside the local set";
            for (int c = 0; c < D; ++c) {
                cd* col = &U[(size_t)c * D];
                for (int i = 0; i < D; ++i) {
                    if ((i >> q0) & 1 || (i >> q1) & 1) continue;
                    int idx[4] = {i, i | (1 << q1), i | (1 << q0), i | (1 << q0) | (1 << q1)};
                    cd v[4] = {col[idx[0]], col[idx[1]], col[idx[2]], col[idx[3]]};
                    for (int r = 0; r < 4; ++r) {
                        cd acc = 0;
                        for (int q = 0; q < 4; ++q) acc += m[r * 4 + q] * v[q];
                        col[idx[r]] = acc;
                    }
                }
            }
        }
    }
    return "";
}

// Real embedding Ut[n][kk] (n = 2i + a output float, kk = 2j + b input float), split
// into rounded hi / lo halves, one 128-byte K chunk per row per block: chunk c at
// c * 2 * (N x 128 bytes), hi block then lo block.
void emit_b(const std::vector<cd>& U, int k, bool tf32, uint8_t* base) {
    const int D = 1 << k;
    const uint32_t Nn = 2u << k;
    const size_t block = (size_t)Nn * 128;
    const size_t bcb = 2 * block;
    const uint32_t kc = tf32 ? 32u : 64u;   // K elements per chunk
    for (uint32_t r = 0; r < Nn; ++r) {
        const int i = (int)(r >> 1), a = (int)(r & 1);
        for (uint32_t kk = 0; kk < Nn; ++kk) {
            const int j = (int)(kk >> 1), b = (int)(kk & 1);
            const cd u = U[(size_t)j * D + i];
            const double v = (a == b) ? u.real() : (a == 1 ? u.imag() : -u.imag());
            const float x = (float)v;
            uint8_t* ch = base + (size_t)(kk / kc) * bcb;
            const uint32_t kl = kk % kc;
            if (tf32) {
                float hi, lo;
                split_tf32(x, &hi, &lo);
                const size_t off = sw128(r, kl * 4);
                std::memcpy(ch + off, &hi, 4);
                std::memcpy(ch + block + off, &lo, 4);
            } else {
                const uint16_t hi = to_bf16(x);
                const uint16_t lo = to_bf16(x - from_bf16(hi));
                const size_t off = sw128(r, kl * 2);
                std::memcpy(ch + off, &hi, 2);
                std::memcpy(ch + block + off, &lo, 2);
            }
        }
    }
}

std::string plan_gemm(const Plan& P, const double* params, int prec, GemmProgram* out) {
    out->stages.clear();
    out->ublob.clear();
    const int n = P.n;
    const bool tf32 = prec == 1;
    for (size_t s = 0; s < P.top.local.size(); ++s) {
        uint64_t local = P.top.local[s];
        int k = __builtin_popcountll(local);
        // widen to at least 6 local qubits (N = 128) with identity qubits
        for (int b = 0; b < n && k < 6; ++b)
            if (!((local >> b) & 1)) { local |= 1ull << b; ++k; }
        if (k < 6 || k > 7) return "tensor-core stages need 6 or 7 local qubits (k in 5..7, n >= 6)";
        if (n - k < 1) return "tensor-core stages need at least one column bit (n > k)";
        svk::GemmStage st;
        std::memset(&st, 0, sizeof(st));
        int lp[8], nl = 0;
        for (int b = 0; b < n; ++b)
            if ((local >> b) & 1) lp[nl++] = b;
        st.keff = (uint32_t)k;
        st.N = 2u << k;
        st.camp_bits = tf32 ? 4u : 5u;
        st.nchunk = (uint32_t)((1u << k) >> st.camp_bits);
        const int ncb = std::min(7, n - k);
        st.ncol_bits = (uint32_t)ncb;
        for (int j = 0; j < k; ++j) st.local_pos[j] = (uint8_t)lp[j];
        int nc = 0, ng = 0;
        for (int b = 0; b < n; ++b) {
            if ((local >> b) & 1) continue;
            if (nc < ncb) st.col_pos[nc++] = (uint8_t)b;
            else st.glob_pos[ng++] = (uint8_t)b;
        }
        st.n_glob = (uint32_t)ng;
        // chunk-varying bits (low local bits, column bits) in ascending physical order
        int var[12], role[12], nv = 0;
        for (uint32_t j = 0; j < st.camp_bits; ++j) { var[nv] = lp[j]; role[nv] = (int)j; ++nv; }
        for (int c = 0; c < ncb; ++c) { var[nv] = st.col_pos[c]; role[nv] = 8 + c; ++nv; }
        for (int a = 0; a < nv; ++a)
            for (int b2 = a + 1; b2 < nv; ++b2)
                if (var[b2] < var[a]) { std::swap(var[a], var[b2]); std::swap(role[a], role[b2]); }
        st.nvar = (uint32_t)nv;
        for (int a = 0; a < nv; ++a) {
            st.var_pos[a] = (uint8_t)var[a];
            st.var_role[a] = (uint8_t)role[a];
        }
        {
            // Producer mapping.  A store writes g bytes (one amplitude, or both amplitudes of
            // the pair when the pair bit is amplitude bit 0) at an offset XOR-linear in the
            // chunk-varying bits; the 128 / g lanes that share a shared-memory wavefront are
            // conflict-free when their 128-byte-slot images are independent.  The lane bits
            // take, lowest physical position first, the bits that extend that rank; the rest
            // follow in ascending order.
            auto aoff = [&](uint32_t jj, uint32_t m) -> uint32_t {
                const uint32_t rowo = (m >> 3) * 1024 + (m & 7) * 128;
                return tf32 ? rowo + ((((jj >> 1) ^ m) & 7u) << 4) + ((jj & 1u) << 3)
                            : rowo + ((((jj >> 2) ^ m) & 7u) << 4) + ((jj & 3u) << 2);
            };
            const bool pair_amp = role[0] == 0;
            const int g = (tf32 ? 8 : 4) * (pair_amp ? 2 : 1);
            const int lg = __builtin_ctz((unsigned)g);
            const int nphase = 7 - lg;                  // lane bits sharing a wavefront
            const uint32_t smask = (128u / (uint32_t)g) - 1u;
            auto slot = [&](int v) -> uint32_t {
                const int r = role[v];
                const uint32_t jj = r < 8 ? 1u << r : 0u, m = r >= 8 ? 1u << (r - 8) : 0u;
                return (aoff(jj, m) >> lg) & smask;
            };
            std::vector<int> left, perm;
            for (int v = 1; v < nv; ++v) left.push_back(v);
            std::vector<uint32_t> basis;   // reduced slot images of the chosen lane bits
            auto reduce = [&](uint32_t x) {
                for (uint32_t b : basis) x = std::min(x, x ^ b);
                return x;
            };
            for (int lane = 0; lane < nphase; ++lane) {
                size_t pick = left.size();
                for (size_t i = 0; i < left.size(); ++i)
                    if (reduce(slot(left[i])) != 0) { pick = i; break; }
                if (pick == left.size()) break;
                basis.push_back(reduce(slot(left[pick])));
                std::sort(basis.begin(), basis.end(), std::greater<uint32_t>());
                perm.push_back(left[pick]);
                left.erase(left.begin() + (long)pick);
            }
            for (int v : left) perm.push_back(v);
            for (size_t i = 0; i < perm.size(); ++i) st.pperm[i] = (uint8_t)perm[i];
        }
        std::vector<cd> U;
        std::string ferr = fuse_unitary(P, P.top.ids[s], lp, k, params, &U);
        if (!ferr.empty()) return ferr;
        const uint32_t Nn = st.N;
        const size_t block = (size_t)Nn * 128;
        st.b_chunk_bytes = (uint32_t)(2 * block);
        // B stays in shared memory when it fits beside the two A slots (k = 6)
        st.resident = ((size_t)st.nchunk * st.b_chunk_bytes + 2 * 32768 <= 192 * 1024) ? 1u : 0u;
        // ring depth: three slots when they fit in 224 KiB with the resident B, else two
        const size_t slot = 32768 + (st.resident ? 0 : (size_t)st.b_chunk_bytes);
        const size_t fixed = 1024 + (st.resident ? (size_t)st.nchunk * st.b_chunk_bytes : 0);
        st.nslot = (fixed + 3 * slot <= 224 * 1024) ? 3u : 2u;
        st.b_off = (uint64_t)((out->ublob.size() + 1023) & ~(size_t)1023);
        out->ublob.resize(st.b_off + (size_t)st.nchunk * st.b_chunk_bytes, 0);
        emit_b(U, k, tf32, out->ublob.data() + st.b_off);
        out->stages.push_back(st);
    }
    out->identity_map = true;
    for (int q = 0; q < n; ++q)
        if (P.final_map[q] != q) out->identity_map = false;
    return "";
}

}  // namespace svh
