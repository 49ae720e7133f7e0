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
    // A gate acts on at most two bits, so it has at most two predecessors (the last
    // gate on each of its bits) and at most two successors (the next one on each).
    std::vector<int> last(nbits, -1);
    struct Adj {
        int n = 0;
        int v[2];
    };
    std::vector<Adj> preds(G), succs(G);
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
            preds[i].v[preds[i].n++] = ps[k];
            succs[ps[k]].v[succs[ps[k]].n++] = i;
            lv = std::max(lv, level[ps[k]]);
        }
        level[i] = lv + 1;
        for (int k = 0; k < gates[i].nq; ++k) last[gates[i].p[k]] = i;
    }

    // --- Step B backward: reachable sets and exact distance sums.  The bitsets index
    // gates by level order (pos), so a level band is a contiguous range of bits.  Every
    // gate reachable from v has a level above l_v and levels 1..max all occur, so
    //   dist(v) = sum over x in RN(v) of (l_x - l_v) = sum over l > l_v of |{x in RN(v): l_x >= l}|,
    // each term a suffix count of the bitset from the first position of level l.
    const int W = (G + 63) / 64;
    uint32_t max_level = 0;
    for (int i = 0; i < G; ++i) max_level = std::max(max_level, level[i]);
    std::vector<int> lstart(max_level + 2, 0), pos(G);   // lstart[l]: first position of level >= l
    for (int i = 0; i < G; ++i) ++lstart[level[i] + 1];
    for (uint32_t l = 1; l <= max_level + 1; ++l) lstart[l] += lstart[l - 1];
    {
        std::vector<int> next(lstart.begin(), lstart.end());   // counting sort by level
        for (int i = 0; i < G; ++i) pos[i] = next[level[i]]++;
    }
    std::vector<uint64_t> rn((size_t)G * (size_t)W, 0);
    std::vector<uint32_t> reach(G, 0), cum(W + 1, 0);
    std::vector<uint64_t> dist(G, 0);
    for (int v = G - 1; v >= 0; --v) {
        uint64_t* r = &rn[(size_t)v * W];
        for (int e = 0; e < succs[v].n; ++e) {
            const int w = succs[v].v[e];
            const uint64_t* rw = &rn[(size_t)w * W];
            for (int k = 0; k < W; ++k) r[k] |= rw[k];
            r[pos[w] >> 6] |= 1ull << (pos[w] & 63);
        }
        cum[W] = 0;   // cum[k]: bits set in words k.. of r
        for (int k = W - 1; k >= 0; --k) cum[k] = cum[k + 1] + (uint32_t)popc64(r[k]);
        uint64_t d = 0;
        for (uint32_t l = level[v] + 1; l <= max_level; ++l) {
            const int a = lstart[l];
            d += cum[(a >> 6) + 1] + (uint32_t)popc64(r[a >> 6] >> (a & 63));
        }
        reach[v] = cum[0];
        dist[v] = d;
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
    std::vector<int> pending(G);   // predecessors not yet done: ready <=> 0
    for (int i = 0; i < G; ++i) pending[i] = preds[i].n;
    auto finish = [&](int i) {
        done[i] = 1;
        for (int e = 0; e < succs[i].n; ++e) --pending[succs[i].v[e]];
    };
    const int width = std::min(L, popc64(universe | fixed));
    int n_done = 0;
    int first = 0;   // every gate below this index is done
    while (n_done < G) {
        uint64_t local = fixed;
        std::vector<uint32_t> stage;
        for (;;) {
            // Absorb to the fixed point in gate order.  Gates are in topological order
            // (predecessors have smaller indices) and the local set does not change
            // while absorbing, so one pass reaches the fixed point: a gate skipped
            // because a predecessor was not done stays blocked, since that predecessor
            // was visited earlier in the same pass and could not be absorbed either.
            for (int i = first; i < G; ++i) {
                if (!done[i] && pending[i] == 0 && (need[i] & ~local) == 0) {
                    finish(i);
                    ++n_done;
                    stage.push_back((uint32_t)i);
                }
            }
            while (first < G && done[first]) ++first;
            int best = -1;
            for (int i = first; i < G; ++i) {
                if (done[i] || pending[i] != 0) continue;
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
