// batch.cpp — C ABI of the batched form (sv_batch_create / sv_run_batch /
// sv_autotune): builds the shared programs, the largest-first queue and the HBM
// workspace, captures the evaluation as one CUDA graph, and times (L, k) candidates.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "batch.h"
#include "internal.h"
#include "jit.h"
#include "kernels.h"
#include "planner.h"
#include "sv.h"

namespace {

using svh::set_error;

#define BT_CUDA(x)                                                                              \
    do {                                                                                        \
        cudaError_t e_ = (x);                                                                   \
        if (e_ != cudaSuccess)                                                                  \
            return set_error(SV_ERR_CUDA, (std::string(#x) + ": " + cudaGetErrorString(e_)).c_str()); \
    } while (0)

constexpr uint32_t kMinQ = 7, kMaxQB = 30, kMaxL = 13;

struct CircIn {
    uint32_t n = 0, n_params = 0, param_off = 0;
    std::vector<svh::GateRec> gates;
    std::vector<std::pair<uint64_t, double>> obs;   // (logical Z mask, coefficient)
    std::string key;                                // structure: width, gates, fixed angles, slots
};

struct DevMem {
    void* p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t n) {
        if (n <= cap) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        cudaError_t e = cudaMalloc(&p, n);
        if (e == cudaSuccess) cap = n;
        return e;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};

// Host image of a built batch (the device blob and the launch description).
struct Built {
    std::vector<uint8_t> blob;
    size_t o_circ = 0, o_prog = 0, o_stage = 0, o_group = 0, o_op = 0, o_term = 0, o_slot = 0, o_sp = 0, o_obs = 0;
    uint32_t n_circ = 0, n_prog = 0, n_resident = 0;
    uint64_t ws_amps = 0;
    svk::BatchSmem sm{};
};

uint32_t tune_L(const sv_tune& t, uint32_t n) {
    uint32_t L = t.L[n] ? t.L[n] : std::min(n, kMaxL);
    return std::min(L, n);
}
uint32_t tune_k(const sv_tune& t, uint32_t n) { return t.k[n] ? t.k[n] : 4u; }

size_t align_to(size_t x, size_t a) { return (x + a - 1) / a * a; }

template <typename T>
size_t put(std::vector<uint8_t>* blob, const std::vector<T>& v) {
    size_t off = align_to(blob->size(), 128);
    blob->resize(off + v.size() * sizeof(T) + 16, 0);
    if (!v.empty()) std::memcpy(blob->data() + off, v.data(), v.size() * sizeof(T));
    return off;
}
template <typename T>
void append_section(std::vector<T>* dst, const svh::Packed& p, size_t off, size_t count) {
    const T* src = reinterpret_cast<const T*>(p.blob.data() + off);
    dst->insert(dst->end(), src, src + count);
}

// Build the programs, queue and shared-memory layout for the circuits `ids` under
// tuning table `tune`.  Circuit ids[j]'s expectation value goes to index ids[j].
sv_status build(const std::vector<CircIn>& in, const std::vector<uint32_t>& ids, const sv_tune& tune, Built* B) {
    *B = Built();
    std::vector<svk::BatchProg> progs;
    std::vector<svk::Stage> stages;
    std::vector<svk::Group> groups;
    std::vector<svk::DevOp<float>> ops;
    std::vector<svk::DevTerm<float>> terms;
    std::vector<svk::PhaseSlot<float>> slots;
    std::vector<int32_t> slot_param;
    std::vector<svk::ObsTerm> obs;
    std::vector<std::vector<int>> final_maps;
    std::map<std::string, uint32_t> by_key;
    std::vector<uint32_t> prog_of(ids.size());
    uint32_t maxG[2] = {0, 0}, maxO[2] = {0, 0}, maxP[2] = {0, 0}, max_slots = 0, maxT = 0;

    for (size_t j = 0; j < ids.size(); ++j) {
        const CircIn& c = in[ids[j]];
        auto it = by_key.find(c.key);
        if (it != by_key.end()) {
            prog_of[j] = it->second;
            continue;
        }
        const uint32_t L = tune_L(tune, c.n), k = tune_k(tune, c.n);
        if (L < kMinQ || L > kMaxL) return set_error(SV_ERR_ARG, "tile width L must be in [7, 13]");
        if (k < 2 || k > 4) return set_error(SV_ERR_ARG, "register width k must be in [2, 4]");
        svh::Plan P;
        P.n = (int)c.n;
        P.n_params = (int)c.n_params;
        P.L = (int)L;
        P.gates = c.gates;
        svh::relabel(P.n, P.gates, &P.phys, &P.final_map);
        for (size_t g = 0; g < P.gates.size(); ++g)
            if (P.gates[g].kind == svh::K_RZ && P.gates[g].param >= 0) P.phys[g].bound = true;
        // tiled circuits keep the coalescing low bits in every tile (as sv_partition does)
        const uint32_t nf = c.n > L ? std::min<uint32_t>(4, L - 1) : 0;
        const uint64_t fixed = nf ? ((1ull << nf) - 1) : 0;
        std::string err = svh::partition_core(P.n, P.phys, (int)L, fixed, (1ull << c.n) - 1, &P.top, nullptr);
        if (!err.empty()) return set_error(SV_ERR_PARTITION, err.c_str());
        // whole warps per register group: 2^(T - R) >= 32
        const int rmax = std::min<int>((int)k, (int)L - 5);
        svh::Program fp, bp;
        svh::Packed pf, pb;
        err = svh::lower(P, nullptr, 8, rmax, false, &fp, true);
        if (err.empty()) err = svh::lower(P, nullptr, 8, rmax, true, &bp, true);
        if (!err.empty()) return set_error(SV_ERR_UNSUPPORTED, err.c_str());
        svh::pack(fp, P.n, 8, &pf);
        svh::pack(bp, P.n, 8, &pb);
        if (pf.stages.size() != pb.stages.size()) return set_error(SV_ERR_UNSUPPORTED, "internal: stage count mismatch");
        svk::BatchProg bpg;
        std::memset(&bpg, 0, sizeof(bpg));
        bpg.n = c.n;
        bpg.Rf = pf.stages[0].R;
        bpg.Rb = pb.stages[0].R;
        bpg.f_stage = (uint32_t)stages.size();
        bpg.n_f = (uint32_t)pf.stages.size();
        stages.insert(stages.end(), pf.stages.begin(), pf.stages.end());
        bpg.b_stage = (uint32_t)stages.size();
        bpg.n_b = (uint32_t)pb.stages.size();
        stages.insert(stages.end(), pb.stages.begin(), pb.stages.end());
        const svh::Packed* pk[2] = {&pf, &pb};
        uint32_t* gbase[2] = {&bpg.f_group, &bpg.b_group};
        uint32_t* obase[2] = {&bpg.f_op, &bpg.b_op};
        uint32_t* tbase[2] = {&bpg.f_term, &bpg.b_term};
        uint32_t* sbase[2] = {&bpg.f_slot, &bpg.b_slot};
        for (int d = 0; d < 2; ++d) {
            const svh::Packed& p = *pk[d];
            *gbase[d] = (uint32_t)groups.size();
            *obase[d] = (uint32_t)ops.size();
            *tbase[d] = (uint32_t)terms.size();
            *sbase[d] = (uint32_t)slots.size();
            append_section(&groups, p, p.group_off, p.n_groups);
            append_section(&ops, p, p.op_off, p.n_ops);
            append_section(&terms, p, p.term_off, p.n_terms);
            append_section(&slots, p, p.slot_off, p.n_slots);
            for (const svk::Stage& st : p.stages) {
                maxG[d] = std::max(maxG[d], st.n_groups);
                maxO[d] = std::max(maxO[d], st.n_ops);
                maxP[d] = std::max(maxP[d], st.n_phase);
                maxT = std::max(maxT, st.T);
                if (d == 1) max_slots = std::max(max_slots, st.n_slots);
                if (st.T - st.R < 5) return set_error(SV_ERR_UNSUPPORTED, "internal: register group narrower than a warp");
            }
        }
        bpg.slot_param = (uint32_t)slot_param.size();
        for (int sp : bp.slot_param) slot_param.push_back(sp);
        const uint32_t pi = (uint32_t)progs.size();
        progs.push_back(bpg);
        final_maps.push_back(P.final_map);
        by_key[c.key] = pi;
        prog_of[j] = pi;
    }

    // queue: widest first (then more stages, then input order)
    std::vector<uint32_t> order(ids.size());
    for (size_t j = 0; j < order.size(); ++j) order[j] = (uint32_t)j;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) {
        const svk::BatchProg &pa = progs[prog_of[a]], &pb = progs[prog_of[b]];
        if (pa.n != pb.n) return pa.n > pb.n;
        return pa.n_f > pb.n_f;
    });
    std::vector<svk::BatchCirc> circs;
    for (uint32_t j : order) {
        const CircIn& c = in[ids[j]];
        const svk::BatchProg& P = progs[prog_of[j]];
        svk::BatchCirc bc;
        std::memset(&bc, 0, sizeof(bc));
        bc.prog = prog_of[j];
        bc.param_off = c.param_off;
        bc.out = ids[j];
        bc.obs_off = (uint32_t)obs.size();
        bc.n_obs = (uint32_t)c.obs.size();
        const std::vector<int>& fm = final_maps[prog_of[j]];
        for (auto& t : c.obs) {
            uint64_t m = 0;
            for (uint32_t q = 0; q < c.n; ++q)
                if ((t.first >> q) & 1) m |= 1ull << fm[q];
            obs.push_back(svk::ObsTerm{m, t.second});
        }
        if (P.n_f > 1) {   // psi and lambda live in HBM between stages
            bc.ws = B->ws_amps;
            B->ws_amps += 2ull << c.n;
        }
        const svk::Stage& s0 = stages[P.f_stage];
        if (P.n_f == 1 && s0.n_glob == 0) B->n_resident++;
        circs.push_back(bc);
    }

    // shared memory: tiles (psi and lambda of the widest tile), then per direction the
    // staged stage program, then the gradient and reduction scratch
    svk::BatchSmem& sm = B->sm;
    size_t o = (size_t)2 * 8 << maxT;
    sm.tiles = (uint32_t)o;
    for (int d = 0; d < 2; ++d) {
        sm.st[d] = (uint32_t)o;
        o = align_to(o + sizeof(svk::Stage), 16);
    }
    for (int d = 0; d < 2; ++d) {
        sm.grp[d] = (uint32_t)o;
        o += (size_t)maxG[d] * sizeof(svk::Group);
        sm.ops[d] = (uint32_t)o;
        o += (size_t)maxO[d] * sizeof(svk::DevOp<float>);
        sm.slots[d] = (uint32_t)o;
        o += (size_t)maxP[d] * sizeof(svk::PhaseSlot<float>);
        sm.ang[d] = (uint32_t)o;
        o = align_to(o + (size_t)maxP[d] * 4, 16);
    }
    const int nw = svk::batch_threads() / 32;
    sm.gsm = (uint32_t)o;
    o = align_to(o + (size_t)max_slots * nw * 4, 16);
    sm.gacc = (uint32_t)o;
    o += (size_t)max_slots * 8;
    sm.red = (uint32_t)o;
    o += (size_t)nw * 8;
    sm.total = (uint32_t)align_to(o, 16);
    sm.max_slots = max_slots;
    if (sm.total > 225 * 1024)
        return set_error(SV_ERR_UNSUPPORTED,
                         ("batch needs " + std::to_string(sm.total / 1024) + " KiB of shared memory per CTA; lower L").c_str());

    B->o_circ = put(&B->blob, circs);
    B->o_prog = put(&B->blob, progs);
    B->o_stage = put(&B->blob, stages);
    B->o_group = put(&B->blob, groups);
    B->o_op = put(&B->blob, ops);
    B->o_term = put(&B->blob, terms);
    B->o_slot = put(&B->blob, slots);
    B->o_sp = put(&B->blob, slot_param);
    B->o_obs = put(&B->blob, obs);
    B->n_circ = (uint32_t)circs.size();
    B->n_prog = (uint32_t)progs.size();
    return SV_OK;
}

// Circuits of at least this many qubits run as wide groups: all circuits of one
// structure sweep each stage together in one generated kernel (jit.h, batched mode),
// instead of one CTA per circuit in the persistent kernel (SVGB_BATCH_WIDE; 0 = never).
uint32_t wide_threshold() {
    const char* e = getenv("SVGB_BATCH_WIDE");
    return e ? (uint32_t)std::max(0, atoi(e)) : 14u;
}
constexpr uint32_t kWideL = 12;   // tile width of the wide groups' stages

struct WideGroup {
    uint32_t n = 0, ncirc = 0, np = 0, nst = 0, nblk = 0;
    std::vector<uint32_t> circ;                         // indices into the batch's circuits
    std::vector<std::shared_ptr<svj::Built>> fwd, bwd;  // generated batched stage kernels
    std::vector<svk::Stage> bst;                        // adjoint stages (T, slots)
    DevMem ws, tab, partial, slotsum, epart;
    size_t o_pofs = 0, o_out = 0, o_obsoff = 0, o_obs = 0, o_pidx = 0, o_plist = 0;
    size_t partial_bytes = 0;
};

}  // namespace

struct sv_batch_s {
    int dev = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<CircIn> in;
    uint32_t total_params = 0;
    sv_tune tune{};
    Built built;
    DevMem blob, ws, params, out, queue;
    double* h_params = nullptr;   // pinned
    double* h_out = nullptr;      // pinned: expval (n_circ) | grad (total_params)
    svk::BatchArgs args{};
    int grid = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double last_ms = 0.0;
    std::vector<std::unique_ptr<WideGroup>> wide;

    void drop_graph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
    }
    ~sv_batch_s() {
        drop_graph();
        blob.release();
        ws.release();
        params.release();
        out.release();
        queue.release();
        for (auto& g : wide) {
            g->ws.release();
            g->tab.release();
            g->partial.release();
            g->slotsum.release();
            g->epart.release();
        }
        if (h_params) cudaFreeHost(h_params);
        if (h_out) cudaFreeHost(h_out);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

namespace {

// Upload a built image and fill the launch arguments.
sv_status upload(sv_batch* b, const Built& B) {
    BT_CUDA(b->blob.ensure(B.blob.size()));
    BT_CUDA(cudaMemcpy(b->blob.p, B.blob.data(), B.blob.size(), cudaMemcpyHostToDevice));
    BT_CUDA(b->ws.ensure(std::max<size_t>(16, B.ws_amps * 8)));
    const uint8_t* base = (const uint8_t*)b->blob.p;
    svk::BatchArgs& a = b->args;
    std::memset(&a, 0, sizeof(a));
    a.circs = (const svk::BatchCirc*)(base + B.o_circ);
    a.n_circ = B.n_circ;
    a.progs = (const svk::BatchProg*)(base + B.o_prog);
    a.stages = (const svk::Stage*)(base + B.o_stage);
    a.groups = (const svk::Group*)(base + B.o_group);
    a.ops = (const svk::DevOp<float>*)(base + B.o_op);
    a.terms = (const svk::DevTerm<float>*)(base + B.o_term);
    a.slots = (const svk::PhaseSlot<float>*)(base + B.o_slot);
    a.slot_param = (const int32_t*)(base + B.o_sp);
    a.obs = (const svk::ObsTerm*)(base + B.o_obs);
    a.params = (const double*)b->params.p;
    a.ws = b->ws.p;
    a.expval = (double*)b->out.p;
    a.grad = (double*)b->out.p + b->in.size();
    a.queue = (uint32_t*)b->queue.p;
    a.sm = B.sm;
    int per_sm = 0, nsm = 0;
    BT_CUDA(svk::batch_occupancy(B.sm.total, &per_sm));
    if (per_sm < 1) return set_error(SV_ERR_UNSUPPORTED, "batch kernel does not fit on an SM");
    BT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->dev));
    b->grid = (int)std::min<uint64_t>((uint64_t)per_sm * nsm, std::max<uint32_t>(1, B.n_circ));
    return SV_OK;
}

// Build the wide groups: per structure, the partition (tile width kWideL), the bind-mode
// programs, their generated batched kernels (compiled and loaded here, before any
// capture), the per-circuit tables and the workspaces.
sv_status build_wide(sv_batch* b) {
    b->wide.clear();
    const uint32_t W = wide_threshold();
    if (W == 0) return SV_OK;
    std::map<std::string, size_t> by_key;
    for (uint32_t i = 0; i < b->in.size(); ++i) {
        const CircIn& c = b->in[i];
        if (c.n < W || c.n <= kWideL) continue;
        auto it = by_key.find(c.key);
        if (it == by_key.end()) {
            by_key[c.key] = b->wide.size();
            b->wide.emplace_back(new WideGroup());
            b->wide.back()->n = c.n;
            b->wide.back()->np = c.n_params;
            it = by_key.find(c.key);
        }
        b->wide[it->second]->circ.push_back(i);
    }
    std::vector<svj::Built*> to_compile;
    std::vector<std::vector<std::pair<uint64_t, double>>> gobs;
    for (auto& gp : b->wide) {
        WideGroup& G = *gp;
        const CircIn& c0 = b->in[G.circ[0]];
        G.ncirc = (uint32_t)G.circ.size();
        svh::Plan P;
        P.n = (int)c0.n;
        P.n_params = (int)c0.n_params;
        P.L = (int)kWideL;
        P.gates = c0.gates;
        svh::relabel(P.n, P.gates, &P.phys, &P.final_map);
        for (size_t g = 0; g < P.gates.size(); ++g)
            if (P.gates[g].kind == svh::K_RZ && P.gates[g].param >= 0) P.phys[g].bound = true;
        std::string err = svh::partition_core(P.n, P.phys, (int)kWideL, 15ull, (1ull << c0.n) - 1, &P.top, nullptr);
        if (!err.empty()) return set_error(SV_ERR_PARTITION, err.c_str());
        svh::Program fp, bp;
        err = svh::lower(P, nullptr, 8, 4, false, &fp, true);
        if (err.empty()) err = svh::lower(P, nullptr, 8, 4, true, &bp, true);
        if (!err.empty()) return set_error(SV_ERR_UNSUPPORTED, err.c_str());
        svh::Packed pf, pb;
        svh::pack(fp, P.n, 8, &pf);
        svh::pack(bp, P.n, 8, &pb);
        for (int d = 0; d < 2; ++d) {
            const svh::Packed& pk = d ? pb : pf;
            const uint8_t* blob = pk.blob.data();
            const auto* groups = (const svk::Group*)(blob + pk.group_off);
            const auto* ops = (const svk::DevOp<float>*)(blob + pk.op_off);
            const auto* terms = (const svk::DevTerm<float>*)(blob + pk.term_off);
            const auto* slots = (const svk::PhaseSlot<float>*)(blob + pk.slot_off);
            for (size_t si = 0; si < pk.stages.size(); ++si) {
                const svk::Stage& st = pk.stages[si];
                svj::StageView v{&st, groups + st.group_off, ops + st.op_off, terms, slots + st.phase_off, (int)c0.n, d + 1};
                v.batched = 1;
                v.zero_init = (d == 0 && si == 0) ? 1 : 0;
                auto bt = std::make_shared<svj::Built>();
                err = svj::generate(v, bt.get());
                if (!err.empty()) return set_error(SV_ERR_UNSUPPORTED, err.c_str());
                if (bt->smem > 227 * 1024) return set_error(SV_ERR_UNSUPPORTED, "wide batch stage exceeds shared memory");
                (d ? G.bwd : G.fwd).push_back(bt);
                to_compile.push_back(bt.get());
            }
        }
        G.bst = pb.stages;
        G.nst = (uint32_t)bp.slot_param.size();
        // parameter -> slots (CSR)
        std::vector<uint32_t> pidx(G.np + 1, 0), plist;
        for (int sp : bp.slot_param)
            if (sp >= 0 && (uint32_t)sp < G.np) pidx[sp + 1]++;
        for (uint32_t p = 0; p < G.np; ++p) pidx[p + 1] += pidx[p];
        plist.assign(pidx[G.np], 0);
        std::vector<uint32_t> fill(pidx.begin(), pidx.end() - 1);
        for (size_t sl = 0; sl < bp.slot_param.size(); ++sl) {
            const int sp = bp.slot_param[sl];
            if (sp >= 0 && (uint32_t)sp < G.np) plist[fill[sp]++] = (uint32_t)sl;
        }
        // per-circuit tables: parameter offsets, output index, observable terms (physical)
        std::vector<uint32_t> pofs, outidx, obs_off(1, 0);
        std::vector<svk::ObsTerm> obs;
        for (uint32_t ci : G.circ) {
            const CircIn& c = b->in[ci];
            pofs.push_back(c.param_off);
            outidx.push_back(ci);
            for (auto& t : c.obs) {
                uint64_t m = 0;
                for (uint32_t q = 0; q < c.n; ++q)
                    if ((t.first >> q) & 1) m |= 1ull << P.final_map[q];
                obs.push_back(svk::ObsTerm{m, t.second});
            }
            obs_off.push_back((uint32_t)obs.size());
        }
        std::vector<uint8_t> tab;
        auto place = [&](const void* src, size_t bytes) {
            size_t off = align_to(tab.size(), 16);
            tab.resize(off + bytes + 16, 0);
            if (bytes) std::memcpy(tab.data() + off, src, bytes);
            return off;
        };
        G.o_pofs = place(pofs.data(), pofs.size() * 4);
        G.o_out = place(outidx.data(), outidx.size() * 4);
        G.o_obsoff = place(obs_off.data(), obs_off.size() * 4);
        G.o_obs = place(obs.data(), obs.size() * sizeof(svk::ObsTerm));
        G.o_pidx = place(pidx.data(), pidx.size() * 4);
        G.o_plist = place(plist.data(), std::max<size_t>(1, plist.size()) * 4);
        BT_CUDA(G.tab.ensure(tab.size()));
        BT_CUDA(cudaMemcpy(G.tab.p, tab.data(), tab.size(), cudaMemcpyHostToDevice));
        BT_CUDA(G.ws.ensure((size_t)G.ncirc * 2 * 8 << c0.n));
        size_t pmax = 8;
        for (const svk::Stage& st : G.bst)
            pmax = std::max<size_t>(pmax, (size_t)G.ncirc * ((size_t)st.n_slots << (c0.n - st.T)) * 8);
        G.partial_bytes = pmax;
        BT_CUDA(G.partial.ensure(pmax));
        BT_CUDA(G.slotsum.ensure(std::max<size_t>(8, (size_t)G.ncirc * G.nst * 8)));
        G.nblk = (uint32_t)std::max<uint64_t>(1, (1ull << c0.n) / 4096);
        BT_CUDA(G.epart.ensure((size_t)G.ncirc * G.nblk * 8));
    }
    if (!to_compile.empty()) {
        std::string err = svj::compile(to_compile);
        if (!err.empty()) return set_error(SV_ERR_CUDA, ("compiling the wide batch kernels: " + err).c_str());
        for (svj::Built* bt : to_compile) BT_CUDA(svj::preload(*bt));
    }
    return SV_OK;
}

// the wide groups' part of one evaluation (stream-ordered after the persistent launch)
cudaError_t launch_wide(sv_batch* b) {
    for (auto& gp : b->wide) {
        WideGroup& G = *gp;
        const uint8_t* tab = (const uint8_t*)G.tab.p;
        float2* psi = (float2*)G.ws.p;
        float2* lam = psi + ((size_t)G.ncirc << G.n);
        const uint32_t* pofs = (const uint32_t*)(tab + G.o_pofs);
        const double* prm = (const double*)b->params.p;
        cudaError_t e = cudaSuccess;
        for (auto& k : G.fwd)
            if ((e = svj::launch_batched(*k, psi, nullptr, nullptr, nullptr, prm, pofs, G.ncirc, b->stream)) != cudaSuccess)
                return e;
        e = svk::launch_bgs_obs(psi, lam, (int)G.n, G.ncirc, (const svk::ObsTerm*)(tab + G.o_obs),
                                (const uint32_t*)(tab + G.o_obsoff), (double*)G.epart.p, G.nblk, b->stream);
        if (e != cudaSuccess) return e;
        for (size_t i = 0; i < G.bwd.size(); ++i) {
            const svk::Stage& st = G.bst[i];
            if (st.n_slots && (e = cudaMemsetAsync(G.partial.p, 0, G.partial_bytes, b->stream)) != cudaSuccess) return e;
            if ((e = svj::launch_batched(*G.bwd[i], psi, lam, (double*)G.partial.p, nullptr, prm, pofs, G.ncirc,
                                         b->stream)) != cudaSuccess)
                return e;
            if (st.n_slots &&
                (e = svk::launch_bgs_slotsum((const double*)G.partial.p, G.ncirc, 1u << (G.n - st.T), st.n_slots,
                                             st.slot_off, G.nst, (double*)G.slotsum.p, b->stream)) != cudaSuccess)
                return e;
        }
        e = svk::launch_bgs_finish((const double*)G.epart.p, G.nblk, (const double*)G.slotsum.p, G.nst,
                                   (const uint32_t*)(tab + G.o_pidx), (const uint32_t*)(tab + G.o_plist), G.np, pofs,
                                   (const uint32_t*)(tab + G.o_out), G.ncirc, b->args.expval, b->args.grad, b->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// one evaluation without the graph (queue and gradient reset, launch)
sv_status launch_direct(sv_batch* b) {
    BT_CUDA(cudaMemsetAsync(b->queue.p, 0, 4, b->stream));
    BT_CUDA(cudaMemsetAsync(b->args.grad, 0, std::max<size_t>(8, b->total_params * 8), b->stream));
    BT_CUDA(svk::launch_batch(b->args, b->grid, b->stream));
    return SV_OK;
}

sv_status capture(sv_batch* b) {
    b->drop_graph();
    const size_t n_out = b->in.size() + b->total_params;
    BT_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemcpyAsync(b->params.p, b->h_params, std::max<size_t>(8, b->total_params * 8),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->queue.p, 0, 4, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->args.grad, 0, std::max<size_t>(8, b->total_params * 8), b->stream);
    if (e == cudaSuccess && b->built.n_circ) e = svk::launch_batch(b->args, b->grid, b->stream);
    if (e == cudaSuccess) e = launch_wide(b);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_out, b->out.p, n_out * 8, cudaMemcpyDeviceToHost, b->stream);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return set_error(SV_ERR_CUDA, cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    b->graph = g;
    BT_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
    return SV_OK;
}

bool is_wide(const CircIn& c) {
    const uint32_t W = wide_threshold();
    return W && c.n >= W && c.n > kWideL;
}

sv_status rebuild(sv_batch* b) {
    std::vector<uint32_t> small;
    for (uint32_t i = 0; i < b->in.size(); ++i)
        if (!is_wide(b->in[i])) small.push_back(i);
    sv_status s = build(b->in, small, b->tune, &b->built);
    if (s != SV_OK) return s;
    b->drop_graph();
    s = upload(b, b->built);
    if (s != SV_OK) return s;
    if (b->wide.empty()) {
        s = build_wide(b);
        if (s != SV_OK) return s;
    }
    return capture(b);
}

}  // namespace

extern "C" {

sv_status sv_batch_create(const sv_circuit* circuits, const sv_observable* observables, uint32_t n_circuits,
                          const sv_tune* tune, void* cuda_stream, sv_batch** out) {
    if (!out) return set_error(SV_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!circuits || !observables || n_circuits == 0) return set_error(SV_ERR_ARG, "empty batch");
    std::vector<CircIn> in(n_circuits);
    uint32_t poff = 0;
    for (uint32_t i = 0; i < n_circuits; ++i) {
        const sv_circuit& c = circuits[i];
        const sv_observable& o = observables[i];
        const std::string at = "circuit " + std::to_string(i) + ": ";
        if (c.n_qubits < kMinQ || c.n_qubits > kMaxQB) return set_error(SV_ERR_ARG, (at + "n_qubits must be in [7, 30]").c_str());
        if (c.n_gates == 0 || !c.gates) return set_error(SV_ERR_ARG, (at + "empty circuit").c_str());
        if (c.n_gates > 32768) return set_error(SV_ERR_ARG, (at + "more than 32768 gates").c_str());
        std::string err = svh::gates_from_circuit(&c, &in[i].gates);
        if (!err.empty()) return set_error(SV_ERR_ARG, (at + err).c_str());
        for (const svh::GateRec& g : in[i].gates)
            if (g.param >= 0 && g.kind != svh::K_RX && g.kind != svh::K_RY && g.kind != svh::K_RZ)
                return set_error(SV_ERR_UNSUPPORTED, (at + "only RX / RY / RZ gates may carry parameters in a batch").c_str());
        if (o.n_qubits != c.n_qubits || (o.n_terms && (!o.pauli || !o.coeff)))
            return set_error(SV_ERR_ARG, (at + "observable does not match the circuit").c_str());
        for (uint32_t t = 0; t < o.n_terms; ++t) {
            uint64_t m = 0;
            for (uint32_t q = 0; q < c.n_qubits; ++q) {
                const uint8_t f = o.pauli[(size_t)t * c.n_qubits + q];
                if (f == 3) m |= 1ull << q;
                else if (f != 0)
                    return set_error(SV_ERR_UNSUPPORTED, (at + "batched observables are sums of Z strings").c_str());
            }
            in[i].obs.push_back({m, o.coeff[t]});
        }
        in[i].n = c.n_qubits;
        in[i].n_params = c.n_params;
        in[i].param_off = poff;
        poff += c.n_params;
        std::string& key = in[i].key;
        key.append((const char*)&c.n_qubits, 4);
        key.append((const char*)&c.n_params, 4);
        for (const svh::GateRec& g : in[i].gates) {
            key.append((const char*)&g.kind, sizeof(g.kind));
            key.append((const char*)g.q, sizeof(g.q));
            key.append((const char*)&g.param, sizeof(g.param));
            key.append((const char*)g.angle, sizeof(g.angle));
        }
    }
    sv_batch* b = new (std::nothrow) sv_batch();
    if (!b) return set_error(SV_ERR_OOM, "host allocation failed");
    b->in = std::move(in);
    b->total_params = poff;
    if (tune) b->tune = *tune;
    auto bail = [&](sv_status s) {
        delete b;
        return s;
    };
    cudaError_t e = cudaGetDevice(&b->dev);
    if (e != cudaSuccess) return bail(set_error(SV_ERR_CUDA, cudaGetErrorString(e)));
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {   // the legacy default stream cannot be captured: use a private one
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(set_error(SV_ERR_CUDA, cudaGetErrorString(e)));
        b->own_stream = true;
    }
    const size_t n_out = b->in.size() + b->total_params;
    if (cudaMallocHost(&b->h_params, std::max<size_t>(8, b->total_params * 8)) != cudaSuccess ||
        cudaMallocHost(&b->h_out, n_out * 8) != cudaSuccess)
        return bail(set_error(SV_ERR_OOM, "pinned host allocation failed"));
    std::memset(b->h_params, 0, std::max<size_t>(8, b->total_params * 8));
    if (b->params.ensure(std::max<size_t>(8, b->total_params * 8)) != cudaSuccess || b->out.ensure(n_out * 8) != cudaSuccess ||
        b->queue.ensure(16) != cudaSuccess)
        return bail(set_error(SV_ERR_OOM, "device allocation failed"));
    if (cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess)
        return bail(set_error(SV_ERR_CUDA, "event creation failed"));
    sv_status s = rebuild(b);
    if (s != SV_OK) return bail(s);
    *out = b;
    return SV_OK;
}

sv_status sv_run_batch(sv_batch* b, const double* params, double* expval_out, double* grad_out) {
    if (!b || !expval_out || (b->total_params && !params)) return set_error(SV_ERR_ARG, "null argument");
    if (!b->exec) return set_error(SV_ERR_CUDA, "batch graph is not instantiated");
    if (b->total_params) std::memcpy(b->h_params, params, (size_t)b->total_params * 8);
    BT_CUDA(cudaEventRecord(b->ev0, b->stream));
    BT_CUDA(cudaGraphLaunch(b->exec, b->stream));
    BT_CUDA(cudaEventRecord(b->ev1, b->stream));
    BT_CUDA(cudaStreamSynchronize(b->stream));
    float ms = 0.f;
    BT_CUDA(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
    b->last_ms = ms;
    std::memcpy(expval_out, b->h_out, b->in.size() * 8);
    if (grad_out && b->total_params) std::memcpy(grad_out, b->h_out + b->in.size(), (size_t)b->total_params * 8);
    return SV_OK;
}

sv_status sv_autotune(sv_batch* b, const double* params, sv_tune* table_out) {
    if (!b || (b->total_params && !params)) return set_error(SV_ERR_ARG, "null argument");
    b->drop_graph();
    if (b->total_params)
        BT_CUDA(cudaMemcpy(b->params.p, params, (size_t)b->total_params * 8, cudaMemcpyHostToDevice));
    // probe each width with at most one wave of its circuits (one per SM)
    int nsm = 0;
    BT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->dev));
    std::map<uint32_t, std::vector<uint32_t>> by_n;
    for (uint32_t i = 0; i < b->in.size(); ++i)
        if (!is_wide(b->in[i]) && by_n[b->in[i].n].size() < (size_t)nsm) by_n[b->in[i].n].push_back(i);
    sv_tune best_table = b->tune;
    for (auto& kv : by_n) {
        const uint32_t n = kv.first;
        std::vector<uint32_t> Ls;
        if (n <= kMaxL) Ls.push_back(n);
        else
            for (uint32_t L = 11; L <= kMaxL; ++L) Ls.push_back(L);
        double best = 1e30;
        uint32_t bL = tune_L(b->tune, n), bk = tune_k(b->tune, n);
        for (uint32_t L : Ls)
            for (uint32_t k = (n <= kMaxL ? 2u : 3u); k <= 4; ++k) {
                sv_tune t = best_table;
                t.L[n] = (uint8_t)L;
                t.k[n] = (uint8_t)k;
                Built B;
                if (build(b->in, kv.second, t, &B) != SV_OK) continue;   // e.g. over the shared-memory limit
                if (upload(b, B) != SV_OK) continue;
                float tmin = 1e30f;
                bool ok = true;
                for (int r = 0; r < 2 && ok; ++r) {   // one warm-up, one timed run
                    ok = cudaEventRecord(b->ev0, b->stream) == cudaSuccess && launch_direct(b) == SV_OK &&
                         cudaEventRecord(b->ev1, b->stream) == cudaSuccess &&
                         cudaStreamSynchronize(b->stream) == cudaSuccess;
                    float ms = 0.f;
                    if (ok && cudaEventElapsedTime(&ms, b->ev0, b->ev1) == cudaSuccess && r > 0) tmin = std::min(tmin, ms);
                }
                if (!ok) {
                    BT_CUDA(cudaGetLastError());
                    return set_error(SV_ERR_CUDA, "autotune run failed");
                }
                if (tmin < best) {
                    best = tmin;
                    bL = L;
                    bk = k;
                }
            }
        best_table.L[n] = (uint8_t)bL;
        best_table.k[n] = (uint8_t)bk;
    }
    b->tune = best_table;
    sv_status s = rebuild(b);
    if (s != SV_OK) return s;
    if (table_out) *table_out = best_table;
    return SV_OK;
}

sv_status sv_batch_info_get(const sv_batch* b, sv_batch_info* out) {
    if (!b || !out) return set_error(SV_ERR_ARG, "null argument");
    std::memset(out, 0, sizeof(*out));
    out->n_circuits = (uint32_t)b->in.size();
    out->n_programs = b->built.n_prog + (uint32_t)b->wide.size();
    out->n_resident = b->built.n_resident;
    out->total_params = b->total_params;
    out->workspace_bytes = b->built.ws_amps * 8;
    for (const auto& g : b->wide) out->workspace_bytes += (uint64_t)g->ncirc * 2 * 8 << g->n;
    out->smem_bytes = b->built.sm.total;
    out->grid = (uint32_t)b->grid;
    out->graph = b->exec ? 1u : 0u;
    out->last_ms = b->last_ms;
    return SV_OK;
}

sv_status sv_batch_destroy(sv_batch* b) {
    if (!b) return set_error(SV_ERR_ARG, "null batch");
    delete b;
    return SV_OK;
}

}  // extern "C"
