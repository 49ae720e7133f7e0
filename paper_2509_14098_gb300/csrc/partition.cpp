// partition.cpp — contraction DAG, critical-path levels, exact closeness
// centrality and the forward frontier partitioner (Sec. 4.1-4.2).
//
// Step A (Sec. 4.1): one node per gate, an edge per shared qubit dimension; a gate
// depends on the previous gate on each of its qubits.  Level l_g = 1 + max level of
// its predecessors (psi is level 0), e.g. l_H = 1, l_CX = 2 in the GHZ-3 example.
//
// Step B, backward pass (Sec. 4.2): in reverse order, RN(v) = union over the
// downstream neighbours w of {w} u RN(w), kept as word bitsets.  The distance along
// any downstream path telescopes to l_x - l_v, so dist(v) = sum_{x in RN(v)} l_x -
// |RN(v)| l_v exactly (no overlap threshold needed).  CC(v) = |RN|/dist * |RN|/N;
// candidates are ranked by cross-multiplying |RN|^2 * dist in 128-bit integers, so
// the ranking is exact; ties go to the lower gate index.
//
// Step B, forward pass (Sec. 4.2, step 3): absorb to a fixed point (scanning in
// original order) every ready gate whose required bits are local; then make local
// the required bits of the highest-CC ready gate that still fits L; repeat; cut
// when nothing fits.  Required bits: none for diagonal gates and SWAP, the target
// only for controlled gates (non-local control allowed), the qubit for other
// one-qubit gates.  After the cut the local set is filled to min(L, |universe|)
// bits with the partition's other touched bits (ascending), then the lowest free
// universe bits.
#include <algorithm>
#include <cstring>

#include "planner.h"

namespace svh {

static inline int popc64(uint64_t x) { return __builtin_popcountll(x); }

static uint64_t need_mask(const PGate& g, bool strict) {
    if (g.kind == K_SWAP) return 0;
    if (strict || g.bound) {
        uint64_t m = 0;
        for (int i = 0; i < g.nq; ++i) m |= 1ull << g.p[i];
        return m;
    }
    if (kind_is_diagonal(g.kind)) return 0;
    if (kind_is_controlled(g.kind)) return 1ull << g.p[1];
    uint64_t m = 0;
    for (int i = 0; i < g.nq; ++i) m |= 1ull << g.p[i];
    return m;
}

void relabel(int n, const std::vector<GateRec>& gates, std::vector<PGate>* phys,
             std::vector<int>* final_map) {
    std::vector<int> where(n);
    for (int q = 0; q < n; ++q) where[q] = q;
    phys->clear();
    phys->reserve(gates.size());
    for (const GateRec& g : gates) {
        PGate p;
        p.kind = g.kind;
        p.nq = g.nq;
        p.p[0] = where[g.q[0]];
        p.p[1] = g.nq > 1 ? where[g.q[1]] : -1;
        phys->push_back(p);
        if (g.kind == K_SWAP) std::swap(where[g.q[0]], where[g.q[1]]);
    }
    *final_map = where;
}

std::string partition_core(int nbits, const std::vector<PGate>& gates, int L, uint64_t fixed,
                           uint64_t universe, Partition* out, Centrality* ccout, bool strict) {
    const int G = (int)gates.size();
    out->local.clear();
    out->ids.clear();
    if (popc64(fixed) > L) return "fixed bits exceed the local budget";

    // --- Step A: DAG on bit positions (identical to the DAG on circuit wires,
    // because a SWAP touches both of its positions) and levels.
    std::vector<int> last(nbits, -1);
    std::vector<std::vector<int>> preds(G), succs(G);
    std::vector<uint32_t> level(G, 0);
    for (int i = 0; i < G; ++i) {
        int ps[2];
        int np = 0;
        for (int k = 0; k < gates[i].nq; ++k) {
            int l = last[gates[i].p[k]];
            if (l >= 0 && !(np == 1 && ps[0] == l)) ps[np++] = l;
        }
        if (np == 2 && ps[0] > ps[1]) std::swap(ps[0], ps[1]);
        uint32_t lv = 0;
        for (int k = 0; k < np; ++k) {
            preds[i].push_back(ps[k]);
            succs[ps[k]].push_back(i);
            lv = std::max(lv, level[ps[k]]);
        }
        level[i] = lv + 1;
        for (int k = 0; k < gates[i].nq; ++k) last[gates[i].p[k]] = i;
    }

    // --- Step B backward: reachable sets and exact distance sums.
    const int W = (G + 63) / 64;
    std::vector<uint64_t> rn((size_t)G * (size_t)W, 0);
    std::vector<uint32_t> reach(G, 0);
    std::vector<uint64_t> dist(G, 0);
    for (int v = G - 1; v >= 0; --v) {
        uint64_t* r = &rn[(size_t)v * W];
        for (int w : succs[v]) {
            const uint64_t* rw = &rn[(size_t)w * W];
            for (int k = 0; k < W; ++k) r[k] |= rw[k];
            r[w >> 6] |= 1ull << (w & 63);
        }
        uint64_t sum_level = 0;
        uint32_t cnt = 0;
        for (int k = 0; k < W; ++k) {
            uint64_t x = r[k];
            while (x) {
                int b = __builtin_ctzll(x);
                x &= x - 1;
                sum_level += level[k * 64 + b];
                ++cnt;
            }
        }
        reach[v] = cnt;
        dist[v] = sum_level - (uint64_t)cnt * level[v];
    }
    if (ccout) {
        ccout->reach = reach;
        ccout->dist = dist;
        ccout->level = level;
    }
    // CC(a) > CC(b) exactly:  |RN_a|^2 / dist_a > |RN_b|^2 / dist_b  (N cancels).
    auto cc_greater = [&](int a, int b) -> bool {
        if (reach[a] == 0) return false;
        if (reach[b] == 0) return true;
        unsigned __int128 lhs = (unsigned __int128)((uint64_t)reach[a] * reach[a]) * dist[b];
        unsigned __int128 rhs = (unsigned __int128)((uint64_t)reach[b] * reach[b]) * dist[a];
        return lhs > rhs;
    };

    // --- Step B forward: frontier partition.
    std::vector<uint64_t> need(G);
    for (int i = 0; i < G; ++i) need[i] = need_mask(gates[i], strict);
    std::vector<char> done(G, 0);
    auto ready = [&](int i) {
        for (int p : preds[i])
            if (!done[p]) return false;
        return true;
    };
    const int width = std::min(L, popc64(universe | fixed));
    int n_done = 0;
    while (n_done < G) {
        uint64_t local = fixed;
        std::vector<uint32_t> stage;
        for (;;) {
            bool changed = true;
            while (changed) {
                changed = false;
                for (int i = 0; i < G; ++i) {
                    if (!done[i] && (need[i] & ~local) == 0 && ready(i)) {
                        done[i] = 1;
                        ++n_done;
                        stage.push_back((uint32_t)i);
                        changed = true;
                    }
                }
            }
            int best = -1;
            for (int i = 0; i < G; ++i) {
                if (done[i] || !ready(i)) continue;
                if (popc64(local | need[i]) > L) continue;
                if (best < 0 || cc_greater(i, best)) best = i;
            }
            if (best < 0) break;
            local |= need[best];
        }
        if (stage.empty()) return "a ready gate needs more local qubits than the budget L";
        uint64_t touched = 0;
        for (uint32_t i : stage)
            for (int k = 0; k < gates[i].nq; ++k) touched |= 1ull << gates[i].p[k];
        touched &= universe;
        for (int b = 0; b < 64 && popc64(local) < width; ++b)
            if ((touched >> b) & 1) local |= 1ull << b;
        for (int b = 0; b < 64 && popc64(local) < width; ++b)
            if ((universe >> b) & 1) local |= 1ull << b;
        out->local.push_back(local);
        out->ids.push_back(std::move(stage));
    }
    return "";
}

}  // namespace svh
