// hier_plan.cpp — host side of the hierarchical tensor-core stage (hier.h).
//
// Each stage of a strict partition with L = k + 7 is partitioned again (the same
// closeness-centrality partitioner, Sec. 4.2, budget k, universe = the stage's tile):
// the sub-partitions' fused unitaries (FP64, then split hi / lo like the flat
// tensor-core stages) become B operands, and the layout tables tell the kernel where
// each amplitude of the tile goes in every sub-partition's A operand.
#include <algorithm>
#include <cstring>
#include <functional>

#include "gemm.h"
#include "hier.h"
#include "planner.h"

namespace svh {

namespace {

// byte offset of amplitude jj (inside its K chunk) of row m in a 128-byte-swizzled
// K-major block: XOR-linear in the bits of jj and m
uint32_t a_offset(bool tf32, uint32_t jj, uint32_t m) {
    const uint32_t rowo = (m >> 3) * 1024 + (m & 7) * 128;
    return tf32 ? rowo + ((((jj >> 1) ^ m) & 7u) << 4) + ((jj & 1u) << 3)
                : rowo + ((((jj >> 2) ^ m) & 7u) << 4) + ((jj & 3u) << 2);
}

}  // namespace

size_t hier_smem_bytes(const svk::HierStage& st) {
    // 1024 (alignment) + A region + B buffers + per-sub-partition amplitude-offset tables
    return 1024 + (size_t)st.a_bytes + (size_t)st.b_slots * st.b_bytes + (size_t)st.n_sub * (1u << st.k) * 4;
}

std::string plan_hier(const Plan& P, const double* params, int prec, HierProgram* out) {
    out->launches.clear();
    out->ublob.clear();
    out->n_sub = 0;
    const int n = P.n;
    const bool tf32 = prec == 1;
    const int k = P.L - 7;
    if (k != 5 && k != 6) return "hierarchical stages need k = 5 or 6 (tiles of 12 or 13 qubits)";
    if (tf32 && k == 6) return "TF32x3 hierarchical stages need k = 5 (the operands of k = 6 exceed shared memory)";
    if (n < P.L) return "hierarchical stages need at least k + 7 qubits";
    if (P.n_fixed < 4) return "hierarchical stages need qubits 0..3 in every tile";
    const int T = k + 7;
    const int camp = tf32 ? 4 : 5;                      // log2 amplitudes per K chunk
    const uint32_t nchunk = 1u << (k - camp);
    const uint32_t N = 2u << k;
    const uint32_t b_bytes = nchunk * 2 * N * 128;
    for (size_t s = 0; s < P.top.local.size(); ++s) {
        const uint64_t tile = P.top.local[s];
        if (__builtin_popcountll(tile) != T || (tile & 15ull) != 15ull) return "internal: stage tile is not k + 7 qubits with 0..3";
        std::vector<uint32_t> ids;
        for (uint32_t i : P.top.ids[s])
            if (P.gates[i].kind != K_SWAP) ids.push_back(i);
        if (ids.empty()) continue;   // relabels only
        int tpos[16], tidx[64];
        for (int b = 0; b < 64; ++b) tidx[b] = -1;
        {
            int t = 0;
            for (int b = 0; b < n; ++b)
                if ((tile >> b) & 1) {
                    tidx[b] = t;
                    tpos[t++] = b;
                }
        }
        // the second level: sub-partitions of at most k qubits inside the tile
        std::vector<PGate> sub;
        for (uint32_t i : ids) sub.push_back(P.phys[i]);
        Partition groups;
        std::string err = partition_core(n, sub, k, 0, tile, &groups, nullptr, true);
        if (!err.empty()) return "sub-partition: " + err;
        const size_t ns = groups.local.size();
        for (size_t g0 = 0; g0 < ns; g0 += svk::kHierMaxSub) {
            const size_t g1 = std::min(ns, g0 + (size_t)svk::kHierMaxSub);
            svk::HierStage st;
            std::memset(&st, 0, sizeof(st));
            st.T = (uint32_t)T;
            st.k = (uint32_t)k;
            st.N = N;
            st.nchunk = nchunk;
            st.n_sub = (uint32_t)(g1 - g0);
            st.b_bytes = b_bytes;
            st.a_bytes = nchunk * 32768;
            // one B buffer: a second one (the next operand's copy overlapping this one's
            // GEMM) measured no faster at BF16x3 k = 5 (it costs a CTA per SM) and slower
            // at TF32x3 k = 5
            st.b_slots = 1;
            for (int t = 0; t < T; ++t) st.tile_pos[t] = (uint8_t)tpos[t];
            int ng = 0;
            for (int b = 0; b < n; ++b)
                if (!((tile >> b) & 1)) st.glob_pos[ng++] = (uint8_t)b;
            st.n_glob = (uint32_t)ng;
            st.b_off = (uint64_t)((out->ublob.size() + 1023) & ~(size_t)1023);
            out->ublob.resize(st.b_off + (size_t)st.n_sub * b_bytes, 0);
            const int S = (int)st.n_sub;
            std::vector<std::vector<int>> cols(S);
            for (int sl = 0; sl < S; ++sl) {
                uint64_t loc = groups.local[g0 + (size_t)sl];
                // widen to exactly k qubits with identity qubits of the tile
                for (int t = 0; t < T && __builtin_popcountll(loc) < k; ++t) loc |= 1ull << tpos[t];
                int na = 0;
                for (int t = 0; t < T; ++t) {
                    if ((loc >> tpos[t]) & 1) st.amp_bits[sl][na++] = (uint8_t)t;
                    else cols[sl].push_back(t);
                }
                if (na != k || cols[sl].size() != 7) return "internal: sub-partition shape";
                // layout sl: amplitude bit i -> (K chunk, position in the row)
                for (int i = 0; i < k; ++i)
                    st.ao[sl][st.amp_bits[sl][i]] = i < camp ? a_offset(tf32, 1u << i, 0) : (32768u << (i - camp));
            }
            // the output tile's layout (pairs adjacent, bits 5.. folded onto 1..3)
            for (int t = 0; t < T; ++t) {
                const uint32_t x = 1u << t;
                st.ao[S][t] = 8u * (x ^ (((x >> 4) ^ (x >> 8)) & 14u));
            }
            // Row order of each layout, last to first.  The epilogue of sub-partition s has
            // thread m write row m's amplitudes into layout s + 1, so the lanes of a warp
            // are rows 0..4 of layout s: they take the column bits whose shared-memory bank
            // images in layout s + 1 are independent (4-byte stores: bank bits 0..4 over 32
            // lanes; 8-byte stores: bits 1..4 over a half warp), so the stores do not
            // conflict where the sub-partitions allow it.
            // Amplitude order of a layout: amplitude bits 0..4 are the only terms that reach
            // bank bits 0 and 1, so the amplitude bits that are lanes of the writing epilogue
            // (column bits of the sub-partition before) come first.
            auto amp_first = [&](int L, const std::vector<int>& pref) {
                std::vector<int> a(st.amp_bits[L], st.amp_bits[L] + k), o;
                for (int t : a)
                    if (std::find(pref.begin(), pref.end(), t) != pref.end()) o.push_back(t);
                for (int t : a)
                    if (std::find(pref.begin(), pref.end(), t) == pref.end()) o.push_back(t);
                for (int i = 0; i < k; ++i) {
                    st.amp_bits[L][i] = (uint8_t)o[i];
                    st.ao[L][o[i]] = i < camp ? a_offset(tf32, 1u << i, 0) : (32768u << (i - camp));
                }
            };
            for (int sl = S - 1; sl >= 0; --sl) {
                const int L = sl + 1;
                if (L < S) amp_first(L, cols[sl]);
                const bool wide = tf32 || L == S;   // 8-byte stores into layout L
                const uint32_t bmask = wide ? 0x1Eu : 0x1Fu;
                const int nl = wide ? 4 : 5;
                std::vector<int> order, rest = cols[sl];
                std::vector<uint32_t> basis;
                auto reduce = [&](uint32_t x) {
                    for (uint32_t bv : basis) x = std::min(x, x ^ bv);
                    return x;
                };
                for (int lane = 0; lane < nl; ++lane) {
                    size_t pick = rest.size();
                    for (size_t i = 0; i < rest.size(); ++i)
                        if (reduce((st.ao[L][rest[i]] >> 2) & bmask)) {
                            pick = i;
                            break;
                        }
                    if (pick == rest.size()) break;
                    basis.push_back(reduce((st.ao[L][rest[pick]] >> 2) & bmask));
                    std::sort(basis.begin(), basis.end(), std::greater<uint32_t>());
                    order.push_back(rest[pick]);
                    rest.erase(rest.begin() + (long)pick);
                }
                order.insert(order.end(), rest.begin(), rest.end());
                for (int i = 0; i < 7; ++i) {
                    st.col_bits[sl][i] = (uint8_t)order[i];
                    st.ao[sl][order[i]] = a_offset(tf32, 0, 1u << i);
                }
            }
            amp_first(0, {1, 2, 3});   // the loads' lanes 0..2 are tile bits 1..3
            // Load / store mapping: pair-index bits 0..2 are tile bits 1..3 (a warp's loads
            // cover 128-byte runs); bits 3, 4 (the other lanes of a warp) take the tile bits
            // whose layout-0 bank images extend those of tile bits 1..3, so the split
            // amplitudes' stores into sub-partition 0's operand conflict as little as they can.
            {
                const uint32_t bmask = tf32 ? 0x1Eu : 0x1Fu;
                std::vector<uint32_t> basis;
                auto reduce = [&](uint32_t x) {
                    for (uint32_t bv : basis) x = std::min(x, x ^ bv);
                    return x;
                };
                std::vector<int> order = {1, 2, 3}, rest;
                for (int t = 4; t < T; ++t) rest.push_back(t);
                for (int t : order) {
                    const uint32_t r = reduce((st.ao[0][t] >> 2) & bmask);
                    if (r) {
                        basis.push_back(r);
                        std::sort(basis.begin(), basis.end(), std::greater<uint32_t>());
                    }
                }
                for (int lane = 3; lane < 5; ++lane) {
                    size_t pick = 0;
                    for (size_t i = 0; i < rest.size(); ++i)
                        if (reduce((st.ao[0][rest[i]] >> 2) & bmask)) {
                            pick = i;
                            break;
                        }
                    const uint32_t r = reduce((st.ao[0][rest[pick]] >> 2) & bmask);
                    if (r) {
                        basis.push_back(r);
                        std::sort(basis.begin(), basis.end(), std::greater<uint32_t>());
                    }
                    order.push_back(rest[pick]);
                    rest.erase(rest.begin() + (long)pick);
                }
                order.insert(order.end(), rest.begin(), rest.end());
                for (int i = 0; i < T - 1; ++i) st.ld_bits[i] = (uint8_t)order[i];
            }
            for (int sl = 0; sl < S; ++sl) {
                int lp[8];
                for (int i = 0; i < k; ++i) lp[i] = tpos[st.amp_bits[sl][i]];
                std::vector<uint32_t> gid;
                for (uint32_t x : groups.ids[g0 + (size_t)sl]) gid.push_back(ids[x]);
                std::vector<std::complex<double>> U;
                err = fuse_unitary(P, gid, lp, k, params, &U);
                if (!err.empty()) return err;
                emit_b(U, k, tf32, out->ublob.data() + st.b_off + (size_t)sl * b_bytes);
            }
            out->n_sub += st.n_sub;
            out->launches.push_back(st);
        }
    }
    out->identity_map = true;
    for (int q = 0; q < n; ++q)
        if (P.final_map[q] != q) out->identity_map = false;
    return "";
}

}  // namespace svh
