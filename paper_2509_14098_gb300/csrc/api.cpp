// api.cpp — the C ABI declared in include/sv.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <memory>
#include <mutex>
#include <unordered_map>

#include "gemm.h"
#include "hier.h"
#include "jit.h"
#include "kernels.h"
#include "planner.h"
#include "internal.h"
#include "sv.h"

namespace {

thread_local std::string g_err;

sv_status fail(sv_status s, const std::string& m) {
    g_err = m;
    return s;
}

#define SV_CUDA(x)                                                                             \
    do {                                                                                       \
        cudaError_t e_ = (x);                                                                  \
        if (e_ != cudaSuccess)                                                                 \
            return fail(SV_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_));        \
    } while (0)

struct DevBuf {
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

// Device copy of a lowered, packed program (see svh::Packed for the layout).
struct DevProgram {
    DevBuf buf;
    svh::Packed packed;
    svk::StageLaunch launch(size_t s, void* psi, void* lam, double* partial) const {
        const uint8_t* b = (const uint8_t*)buf.p;
        svk::StageLaunch L;
        L.psi = psi;
        L.lam = lam;
        L.stage = (const svk::Stage*)(b + packed.stage_off) + s;
        L.groups = (const svk::Group*)(b + packed.group_off);
        L.ops = b + packed.op_off;
        L.terms = b + packed.term_off;
        L.slots = b + packed.slot_off;
        L.partial = partial;
        return L;
    }
};

size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

}  // namespace

namespace svh {
// error reporting for entry points defined in other translation units
sv_status set_error(sv_status s, const char* msg) { return fail(s, msg); }

std::string gates_from_circuit(const sv_circuit* c, std::vector<GateRec>* out) {
    out->clear();
    out->reserve(c->n_gates);
    for (uint32_t i = 0; i < c->n_gates; ++i) {
        const sv_gate& g = c->gates[i];
        const std::string at = "gate " + std::to_string(i) + ": ";
        GateRec r;
        r.kind = g.kind;
        if (g.kind < K_H || g.kind > K_LAST) return at + "unknown kind";
        r.nq = kind_nq(g.kind);
        if (g.nq != r.nq) return at + "wrong qubit count";
        for (int k = 0; k < r.nq; ++k) {
            if (g.q[k] >= c->n_qubits) return at + "qubit out of range";
            r.q[k] = g.q[k];
        }
        if (r.nq == 1) r.q[1] = -1;
        if (r.nq == 2 && r.q[0] == r.q[1]) return at + "repeated qubit";
        r.param = g.param;
        if (g.param >= 0) {
            bool ok = g.kind == K_RX || g.kind == K_RY || g.kind == K_RZ || g.kind == K_P || g.kind == K_CP;
            if (!ok || (uint32_t)g.param >= c->n_params) return at + "bad parameter slot";
        } else if (g.param != -1) {
            return at + "param must be -1 or a slot";
        }
        for (int k = 0; k < 3; ++k) r.angle[k] = g.angle[k];
        out->push_back(r);
    }
    return "";
}
}  // namespace svh

struct sv_plan_s {
    svh::Plan plan;
};

struct sv_handle_s {
    uint32_t n = 0;
    sv_dtype dt = SV_C64;
    int eb = 8;
    void* psi = nullptr;
    bool owns = false;
    cudaStream_t stream = nullptr;
    DevBuf scratch;      // state-sized: permutation target / adjoint lambda
    DevProgram fwd, bwd;
    DevBuf partial;      // per-tile gradient partial sums
    DevBuf slot_sum;     // per-slot gradient sums
    DevBuf red;          // reduction partials and results
    DevBuf aux;          // Pauli sweeps / permutation descriptors
    DevBuf gemm;         // tensor-core stage descriptors + operand chunks
    DevBuf status;       // device-side error flag (bounded waits)
    DevBuf jflag;        // generated stage kernels' bounded-wait flag (sticky until reported)
    bool jflag_pending = false;   // a generated kernel ran since the flag was last read
    std::vector<uint8_t> gemm_host;
    std::vector<uint8_t> aux_host;
    sv_run_info info{};
    // kernel timing: event pairs recorded around sweep launches
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    struct Rec { cudaEvent_t a, b; int kind; };
    std::vector<Rec> recs;
    size_t ev_used = 0;
};

enum { TK_STAGE = 0, TK_BWD = 1, TK_PERM = 2, TK_OBS = 3 };

static cudaEvent_t next_event(sv_handle h) {
    if (h->ev_used == h->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        h->ev_pool.push_back(e);
    }
    return h->ev_pool[h->ev_used++];
}
// RAII-free helpers: tick() before a launch, tock() after it.
static cudaEvent_t tick(sv_handle h) {
    if (!h->timing) return nullptr;
    cudaEvent_t e = next_event(h);
    if (e) cudaEventRecord(e, h->stream);
    return e;
}
static void tock(sv_handle h, cudaEvent_t a, int kind) {
    if (!h->timing || !a) return;
    cudaEvent_t b = next_event(h);
    if (!b) return;
    cudaEventRecord(b, h->stream);
    h->recs.push_back({a, b, kind});
}

static sv_status upload_program(sv_handle h, const svh::Program& p, DevProgram* d, bool backward) {
    std::string err = svh::pack(p, (int)h->n, h->eb, &d->packed);
    if (!err.empty()) return fail(SV_ERR_ARG, err);
    for (auto& st : d->packed.stages)
        if (svk::stage_smem_bytes(h->eb, st, backward) > 227 * 1024)
            return fail(SV_ERR_UNSUPPORTED, "a stage needs more shared memory than a CTA has (lower L or split the circuit)");
    SV_CUDA(d->buf.ensure(d->packed.blob.size()));
    // pageable source: the call returns once the data is staged, so the host blob may
    // be reused immediately; the device copy is stream-ordered.
    SV_CUDA(cudaMemcpyAsync(d->buf.p, d->packed.blob.data(), d->packed.blob.size(),
                            cudaMemcpyHostToDevice, h->stream));
    return SV_OK;
}

static sv_status check_handle(sv_handle h) {
    if (!h) return fail(SV_ERR_ARG, "null handle");
    return SV_OK;
}

static size_t state_bytes(sv_handle h) { return ((size_t)1 << h->n) * (size_t)h->eb; }

// The generated stage kernels bound their waits for tile copies; a kernel that gave
// up sets the handle's flag.  sv_run stays asynchronous, so the flag is read at the
// next call that synchronises the stream (and then cleared).
static sv_status jflag_device(sv_handle h, int** out) {
    if (!h->jflag.p) {
        SV_CUDA(h->jflag.ensure(sizeof(int)));
        SV_CUDA(cudaMemsetAsync(h->jflag.p, 0, sizeof(int), h->stream));
    }
    *out = (int*)h->jflag.p;
    h->jflag_pending = true;
    return SV_OK;
}
static sv_status jflag_check(sv_handle h) {
    if (!h->jflag_pending) return SV_OK;
    h->jflag_pending = false;
    int v = 0;
    SV_CUDA(cudaMemcpyAsync(&v, h->jflag.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    SV_CUDA(cudaStreamSynchronize(h->stream));
    if (v) {
        SV_CUDA(cudaMemsetAsync(h->jflag.p, 0, sizeof(int), h->stream));
        return fail(SV_ERR_TIMEOUT, "a stage kernel gave up waiting for its tile copies (bounded wait); the state is invalid");
    }
    return SV_OK;
}

// ---------------------------------------------------------------------------
// permutation sweep: new[y] = old[x], bit phys_of_qubit[q] of x = bit q of y
// ---------------------------------------------------------------------------
// Tile of the permutation sweep (input physical bits): the input's 4 lowest bits and the
// input bits that land on output bits 0..3, then alternately the next input bit above
// the contiguous input run and the input bit that lands just above the contiguous output
// run, so that both the reads and the writes are runs of at least 512 bytes (2^12
// complex64 / 2^11 complex128).  dst[p] = the output bit of input bit p.
static uint64_t perm_tile(int n, int eb, const uint32_t* phys_of_qubit, const int* dst, int* T) {
    const int c = std::min(4, n);
    uint64_t B = (1ull << c) - 1;
    for (int p = 0; p < n; ++p)
        if (dst[p] < c) B |= 1ull << p;
    const int Tp = std::min(n, eb == 8 ? 12 : 11);
    for (int turn = 0, ri = 0, ro = 0; __builtin_popcountll(B) < Tp; turn ^= 1) {
        while (ri < n && ((B >> ri) & 1)) ++ri;
        while (ro < n && ((B >> phys_of_qubit[ro]) & 1)) ++ro;
        if (turn == 0 && ri < n) B |= 1ull << ri;
        else if (ro < n) B |= 1ull << phys_of_qubit[ro];
        else if (ri < n) B |= 1ull << ri;
    }
    *T = Tp;
    return B;
}

// dst[p] from phys_of_qubit (false: not a permutation of 0..n-1)
static bool perm_dst(int n, const uint32_t* phys_of_qubit, int* dst) {
    uint64_t seen = 0;
    for (int q = 0; q < n; ++q) {
        const uint32_t p = phys_of_qubit[q];
        if (p >= (uint32_t)n || ((seen >> p) & 1)) return false;
        seen |= 1ull << p;
        dst[p] = q;
    }
    return true;
}

static sv_status do_permute(sv_handle h, const uint32_t* phys_of_qubit) {
    const int n = (int)h->n;
    int dst[64];
    if (!perm_dst(n, phys_of_qubit, dst)) return fail(SV_ERR_ARG, "not a permutation");
    bool ident = true;
    for (int p = 0; p < n; ++p)
        if (dst[p] != p) ident = false;
    if (ident) return SV_OK;
    int Tp = 0;
    const uint64_t B = perm_tile(n, h->eb, phys_of_qubit, dst, &Tp);
    svk::PermDesc d;
    std::memset(&d, 0, sizeof(d));
    d.T = (uint32_t)Tp;
    int nt = 0, ng = 0;
    for (int p = 0; p < n; ++p) {
        if ((B >> p) & 1) {
            d.tile_pos[nt] = (uint8_t)p;
            d.ptile[nt] = 1ull << p;
            d.swbit[nt] = svk::swizzle(1u << nt, h->eb);
            ++nt;
        } else {
            d.glob_pos[ng] = (uint8_t)p;
            d.gout[ng] = 1ull << dst[p];
            ++ng;
        }
    }
    d.n_glob = (uint32_t)ng;
    // output tile positions ascending; sig = swizzled input element offset
    std::vector<std::pair<int, int>> outs;   // (output position, input tile bit)
    for (int b = 0; b < nt; ++b) outs.push_back({dst[d.tile_pos[b]], b});
    std::sort(outs.begin(), outs.end());
    for (int c2 = 0; c2 < nt; ++c2) {
        d.pout[c2] = 1ull << outs[c2].first;
        d.sig[c2] = d.swbit[outs[c2].second];
    }
    SV_CUDA(h->scratch.ensure(state_bytes(h)));
    const uint64_t ntiles = 1ull << (n - Tp);
    cudaEvent_t t0 = tick(h);
    SV_CUDA(svk::launch_permute(h->eb, h->psi, h->scratch.p, d, ntiles, h->stream));
    tock(h, t0, TK_PERM);
    // a handle that owns its state takes the permuted buffer as the state; a caller's
    // buffer receives a copy
    if (h->owns) {
        std::swap(h->psi, h->scratch.p);
    } else {
        SV_CUDA(cudaMemcpyAsync(h->psi, h->scratch.p, state_bytes(h), cudaMemcpyDeviceToDevice, h->stream));
        h->info.hbm_bytes += 2.0 * (double)state_bytes(h);
    }
    h->info.permutation_sweeps += 1;
    h->info.kernel_launches += 1;
    h->info.hbm_bytes += 2.0 * (double)state_bytes(h);
    return SV_OK;
}

// ---------------------------------------------------------------------------
// Pauli sweeps
// ---------------------------------------------------------------------------
struct PauliPlan {
    std::vector<svk::PauliSweep> sweeps;
    std::vector<svk::PauliTerm> terms;
};

// Split the observable into sweeps: each sweep's tile holds the L lowest physical bits
// and the X / Y qubits of its terms; the diagonal terms go to sweep 0.  Within a sweep
// the register bits are the tile qubits that carry X / Y most often.
static sv_status plan_pauli(int n, int eb, const sv_observable* obs, const std::vector<int>& where,
                            PauliPlan* out) {
    if (!obs || obs->n_qubits != (uint32_t)n || (obs->n_terms && (!obs->pauli || !obs->coeff)))
        return fail(SV_ERR_ARG, "bad observable");
    struct Raw { uint64_t x, z; double fre, fim; };
    std::vector<Raw> diag, off;
    for (uint32_t t = 0; t < obs->n_terms; ++t) {
        uint64_t x = 0, z = 0;
        int ny = 0;
        for (int q = 0; q < n; ++q) {
            uint8_t c = obs->pauli[(size_t)t * n + q];
            uint64_t b = 1ull << where[q];
            if (c == 1) x |= b;
            else if (c == 2) { x |= b; z |= b; ++ny; }
            else if (c == 3) z |= b;
            else if (c != 0) return fail(SV_ERR_ARG, "pauli code must be 0..3");
        }
        double fr = obs->coeff[t], fi = 0;   // coeff * i^ny
        for (int k = 0; k < (ny & 3); ++k) { double r = -fi, i2 = fr; fr = r; fi = i2; }
        if (__builtin_popcountll(x & z) & 1) { fr = -fr; fi = -fi; }   // (-1)^{|x & z|}
        (x ? off : diag).push_back(Raw{x, z, fr, fi});
    }
    // tiles of 13 qubits for complex64 (512 threads x 16 amplitudes), 12 for complex128
    int tc64 = 13;
    if (const char* e = getenv("SVGB_PAULI_T")) tc64 = std::max(9, std::min(13, atoi(e)));
    const int T = std::min(n, eb == 8 ? tc64 : 12);
    const int L = std::min(4, T - 1);
    const int R = std::min(eb == 8 ? 4 : 3, T - L);
    std::vector<char> used(off.size(), 0);
    size_t left = off.size();
    bool first = true;
    while (first || left) {
        uint64_t tile = (1ull << L) - 1;
        for (size_t i = 0; i < off.size(); ++i)
            if (!used[i] && __builtin_popcountll(tile | off[i].x) <= T) tile |= off[i].x;
        for (int p = 0; p < n && __builtin_popcountll(tile) < T; ++p) tile |= 1ull << p;
        std::vector<size_t> mine;
        for (size_t i = 0; i < off.size(); ++i)
            if (!used[i] && (off[i].x & ~tile) == 0) mine.push_back(i);
        if (!first && mine.empty())
            return fail(SV_ERR_UNSUPPORTED, "a Pauli term has X/Y on more qubits than a tile holds");
        // register bits: the non-low tile qubits with the most X / Y among this sweep's terms
        std::vector<int> cand;
        for (int p = L; p < n; ++p)
            if ((tile >> p) & 1) cand.push_back(p);
        std::vector<int> cnt(n, 0);
        for (size_t i : mine)
            for (uint64_t m = off[i].x; m; m &= m - 1) cnt[__builtin_ctzll(m)]++;
        std::vector<int> byc = cand;
        std::stable_sort(byc.begin(), byc.end(), [&](int u, int v) { return cnt[u] > cnt[v]; });
        std::vector<int> reg(byc.begin(), byc.begin() + R);
        std::sort(reg.begin(), reg.end());
        std::vector<int> pos;
        for (int p = 0; p < L; ++p) pos.push_back(p);
        for (int p : reg) pos.push_back(p);
        // the other tile qubits, fewest X / Y first: the qubits that carry X / Y take the
        // top tile bits, which the generated sweeps also read as register bits
        std::vector<int> rest;
        for (int p : cand)
            if (std::find(reg.begin(), reg.end(), p) == reg.end()) rest.push_back(p);
        std::stable_sort(rest.begin(), rest.end(), [&](int u, int v) { return cnt[u] < cnt[v]; });
        for (int p : rest) pos.push_back(p);
        svk::PauliSweep sw;
        std::memset(&sw, 0, sizeof(sw));
        sw.T = (uint32_t)T;
        sw.R = (uint32_t)R;
        sw.L = (uint32_t)L;
        int tidx[64];
        for (int p = 0; p < 64; ++p) tidx[p] = -1;
        for (int b = 0; b < T; ++b) {
            tidx[pos[b]] = b;
            sw.ptile[b] = 1ull << pos[b];
        }
        int ng = 0;
        for (int p = 0; p < n; ++p)
            if (tidx[p] < 0) sw.glob_pos[ng++] = (uint8_t)p;
        sw.n_glob = (uint32_t)ng;
        sw.term_off = (uint32_t)out->terms.size();
        const uint32_t regmask = ((1u << R) - 1u) << L;
        auto add = [&](const Raw& r, uint32_t flags) {
            svk::PauliTerm pt;
            std::memset(&pt, 0, sizeof(pt));
            pt.zmask = r.z;
            for (uint64_t m = r.x; m; m &= m - 1) pt.xtile |= 1u << tidx[__builtin_ctzll(m)];
            pt.xreg = (uint16_t)((pt.xtile & regmask) >> L);
            for (int j = 0; j < R; ++j)
                if ((r.z >> pos[L + j]) & 1) pt.zreg |= (uint16_t)(1u << j);
            for (int k = 0; k < (1 << R); ++k)
                if (__builtin_popcount((unsigned)k & pt.zreg) & 1) pt.smask |= 1u << k;
            if (pt.xtile & ~regmask) flags |= svk::PT_SMEM;
            if (r.fim == 0.0) flags |= svk::PT_REAL;
            uint64_t regphys = 0;
            for (int j = 0; j < R; ++j) regphys |= 1ull << pos[L + j];
            if ((r.z & ~regphys) == 0) flags |= svk::PT_NOZ;
            pt.flags = flags;
            pt.fre = r.fre;
            pt.fim = r.fim;
            pt.fre32 = (float)r.fre;
            pt.fim32 = (float)r.fim;
            out->terms.push_back(pt);
        };
        if (first) {
            // diagonal terms: Z on tile bits only, on global bits only, on both; the
            // first and last classes grouped by their register-bit Z mask (one
            // 2^R-wide update per group)
            std::vector<size_t> cls[3];
            for (size_t i = 0; i < diag.size(); ++i) {
                const uint64_t zt = diag[i].z & tile, zg = diag[i].z & ~tile;
                cls[zg == 0 ? 0 : (zt == 0 ? 1 : 2)].push_back(i);
            }
            auto zreg_of = [&](size_t i) {
                uint32_t zr = 0;
                for (int j = 0; j < R; ++j)
                    if ((diag[i].z >> pos[L + j]) & 1) zr |= 1u << j;
                return zr;
            };
            for (int c = 0; c < 3; ++c) {
                auto& v = cls[c];
                if (c != 1)
                    std::stable_sort(v.begin(), v.end(), [&](size_t u, size_t w) { return zreg_of(u) < zreg_of(w); });
                for (size_t j = 0; j < v.size(); ++j) {
                    const bool flush = c != 1 && (j + 1 == v.size() || zreg_of(v[j + 1]) != zreg_of(v[j]));
                    add(diag[v[j]], flush ? svk::PT_FLUSH : 0u);
                }
            }
            sw.n_dstat = (uint32_t)cls[0].size();
            sw.n_dglob = (uint32_t)cls[1].size();
            sw.n_dmix = (uint32_t)cls[2].size();
        }
        for (size_t i : mine) {
            add(off[i], 0u);
            used[i] = 1;
            --left;
        }
        sw.n_terms = (uint32_t)(out->terms.size() - sw.term_off);
        out->sweeps.push_back(sw);
        first = false;
    }
    return SV_OK;
}

// Run the sweeps; lam != nullptr also forms lam = O psi.  Leaves the expectation
// value (FP64) at red[0] on the device.
// Expectation-only complex64 sweeps run as kernels generated per sweep (svj::
// generate_pauli), memoised by the sweep's and its terms' bytes; SVGB_PAULI_JIT=0
// selects the generic sweep kernel.  Returns false when a sweep has no generated form.
static std::mutex g_pauli_mu;
static std::unordered_map<std::string, std::shared_ptr<svj::Built>> g_pauli_memo;

static bool pauli_jit(int n, int eb, const PauliPlan& pp, std::vector<std::shared_ptr<svj::Built>>* out,
                      sv_status* st) {
    *st = SV_OK;
    out->clear();
    const char* ev = getenv("SVGB_PAULI_JIT");
    if (eb != 8 || (ev && atoi(ev) == 0)) return false;
    std::vector<svj::Built*> fresh;
    for (const svk::PauliSweep& sw : pp.sweeps) {
        std::string key((const char*)&sw, sizeof(sw));
        key.append((const char*)(pp.terms.data() + sw.term_off), sw.n_terms * sizeof(svk::PauliTerm));
        std::shared_ptr<svj::Built> b;
        {
            std::lock_guard<std::mutex> lk(g_pauli_mu);
            auto it = g_pauli_memo.find(key);
            if (it != g_pauli_memo.end()) b = it->second;
        }
        if (!b) {
            b = std::make_shared<svj::Built>();
            if (!svj::generate_pauli(sw, pp.terms.data(), n, b.get()).empty()) return false;
            fresh.push_back(b.get());
            std::lock_guard<std::mutex> lk(g_pauli_mu);
            if (g_pauli_memo.size() > 1024) g_pauli_memo.clear();
            g_pauli_memo[key] = b;
        }
        out->push_back(b);
    }
    if (!fresh.empty()) {
        const std::string err = svj::compile(fresh);
        if (!err.empty()) {
            *st = fail(SV_ERR_CUDA, "run-time compilation of a Pauli sweep failed: " + err);
            return true;
        }
    }
    return true;
}

static sv_status run_pauli(sv_handle h, const PauliPlan& pp, void* lam) {
    const int n = (int)h->n;
    if (!lam) {
        std::vector<std::shared_ptr<svj::Built>> built;
        sv_status js = SV_OK;
        if (pauli_jit(n, h->eb, pp, &built, &js)) {
            if (js) return js;
            int nsm = 0, dev = 0;
            SV_CUDA(cudaGetDevice(&dev));
            SV_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
            uint64_t rows = 0;   // at most 32 CTAs per SM per sweep
            for (auto& b : built) rows += std::min<uint64_t>(b->ntiles, (uint64_t)nsm * 32);
            SV_CUDA(h->red.ensure((rows + 16) * sizeof(double)));
            double* part = (double*)h->red.p + 16;
            uint64_t off = 0;
            for (auto& b : built) {
                uint32_t grid = 0;
                cudaEvent_t t0 = tick(h);
                SV_CUDA(svj::launch(*b, h->psi, nullptr, part + off, nullptr, h->stream, &grid));
                tock(h, t0, TK_OBS);
                off += grid;
                h->info.reduction_sweeps += 1;
                h->info.kernel_launches += 1;
                h->info.hbm_bytes += (double)state_bytes(h);
            }
            SV_CUDA(svk::launch_reduce_rows(part, off, 1, (double*)h->red.p, h->stream));
            h->info.kernel_launches += 1;
            return SV_OK;
        }
    }
    const size_t szs = align16(pp.sweeps.size() * sizeof(svk::PauliSweep));
    const size_t szt = align16(std::max<size_t>(1, pp.terms.size()) * sizeof(svk::PauliTerm));
    SV_CUDA(h->aux.ensure(szs + szt));
    h->aux_host.assign(szs + szt, 0);
    std::memcpy(h->aux_host.data(), pp.sweeps.data(), pp.sweeps.size() * sizeof(svk::PauliSweep));
    std::memcpy(h->aux_host.data() + szs, pp.terms.data(), pp.terms.size() * sizeof(svk::PauliTerm));
    SV_CUDA(cudaMemcpyAsync(h->aux.p, h->aux_host.data(), szs + szt, cudaMemcpyHostToDevice, h->stream));
    uint64_t total_rows = 0;
    for (auto& sw : pp.sweeps) {
        const uint32_t g = svk::pauli_grid(h->eb, sw, 1ull << (n - (int)sw.T));
        if (!g) {
            const cudaError_t e = cudaGetLastError();
            SV_CUDA(e != cudaSuccess ? e : cudaErrorInvalidValue);
        }
        total_rows += g;
    }
    SV_CUDA(h->red.ensure((total_rows + 16) * sizeof(double)));
    double* part = (double*)h->red.p + 16;
    uint64_t off = 0;
    for (size_t i = 0; i < pp.sweeps.size(); ++i) {
        const svk::PauliSweep& sw = pp.sweeps[i];
        const uint64_t nt = 1ull << (n - (int)sw.T);
        uint32_t grid = 0;
        cudaEvent_t t0 = tick(h);
        SV_CUDA(svk::launch_pauli(h->eb, h->psi, lam, i > 0, sw, (const svk::PauliSweep*)h->aux.p + i,
                                  (const svk::PauliTerm*)((uint8_t*)h->aux.p + szs), part + off, nt, &grid,
                                  h->stream));
        tock(h, t0, TK_OBS);
        off += grid;
        h->info.reduction_sweeps += 1;
        h->info.kernel_launches += 1;
        h->info.hbm_bytes += (double)state_bytes(h) * (lam ? (i ? 3.0 : 2.0) : 1.0);
    }
    SV_CUDA(svk::launch_reduce_rows(part, off, 1, (double*)h->red.p, h->stream));
    h->info.kernel_launches += 1;
    return SV_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* sv_last_error(void) { return g_err.c_str(); }

sv_status sv_create(uint32_t n_qubits, sv_dtype dtype, void* dev_state, void* cuda_stream,
                    sv_handle* out) {
    if (!out) return fail(SV_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_qubits < 1 || n_qubits > 34) return fail(SV_ERR_ARG, "n_qubits must be in [1, 34]");
    if (dtype != SV_C64 && dtype != SV_C128) return fail(SV_ERR_ARG, "bad dtype");
    if (dev_state && ((uintptr_t)dev_state & 15)) return fail(SV_ERR_ARG, "state buffer must be 16-byte aligned");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(SV_ERR_CUDA, "no CUDA device");
    }
    sv_handle h = new (std::nothrow) sv_handle_s();
    if (!h) return fail(SV_ERR_OOM, "host allocation failed");
    h->n = n_qubits;
    h->dt = dtype;
    h->eb = dtype == SV_C64 ? 8 : 16;
    h->stream = (cudaStream_t)cuda_stream;
    if (dev_state) {
        h->psi = dev_state;
        h->owns = false;
    } else {
        cudaError_t e = cudaMalloc(&h->psi, state_bytes(h));
        if (e != cudaSuccess) {
            delete h;
            cudaGetLastError();
            return fail(SV_ERR_OOM, std::string("cudaMalloc state: ") + cudaGetErrorString(e));
        }
        h->owns = true;
        e = svk::launch_zero_state(h->eb, h->psi, 1ull << h->n, h->stream);
        if (e != cudaSuccess) {
            cudaFree(h->psi);
            delete h;
            return fail(SV_ERR_CUDA, cudaGetErrorString(e));
        }
    }
    *out = h;
    return SV_OK;
}

sv_status sv_timing_enable(sv_handle h, int enable) {
    if (check_handle(h)) return SV_ERR_ARG;
    h->timing = enable != 0;
    return SV_OK;
}

sv_status sv_timing_read(sv_handle h, sv_timing* out, int reset) {
    if (check_handle(h) || !out) return fail(SV_ERR_ARG, "null argument");
    SV_CUDA(cudaStreamSynchronize(h->stream));
    std::memset(out, 0, sizeof(*out));
    for (auto& r : h->recs) {
        float ms = 0.f;
        SV_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        switch (r.kind) {
            case TK_STAGE: out->stage_ms += ms; out->stage_launches++; break;
            case TK_BWD: out->backward_ms += ms; out->backward_launches++; break;
            case TK_PERM: out->permute_ms += ms; out->permute_launches++; break;
            default: out->observable_ms += ms; out->observable_launches++; break;
        }
    }
    if (reset) {
        h->recs.clear();
        h->ev_used = 0;
    }
    return SV_OK;
}

sv_status sv_destroy(sv_handle h) {
    if (!h) return SV_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    if (h->owns && h->psi) cudaFree(h->psi);
    h->scratch.release();
    h->fwd.buf.release();
    h->bwd.buf.release();
    h->partial.release();
    h->slot_sum.release();
    h->red.release();
    h->aux.release();
    h->gemm.release();
    h->status.release();
    h->jflag.release();
    delete h;
    return SV_OK;
}

sv_status sv_info(sv_handle h, uint32_t* n_qubits, sv_dtype* dtype, void** dev_state) {
    if (check_handle(h)) return SV_ERR_ARG;
    if (n_qubits) *n_qubits = h->n;
    if (dtype) *dtype = h->dt;
    if (dev_state) *dev_state = h->psi;
    return SV_OK;
}

sv_status sv_reset_zero(sv_handle h) {
    if (check_handle(h)) return SV_ERR_ARG;
    SV_CUDA(svk::launch_zero_state(h->eb, h->psi, 1ull << h->n, h->stream));
    return SV_OK;
}

sv_status sv_set_state(sv_handle h, const void* dev_src) {
    if (check_handle(h) || !dev_src) return fail(SV_ERR_ARG, "null argument");
    SV_CUDA(cudaMemcpyAsync(h->psi, dev_src, state_bytes(h), cudaMemcpyDeviceToDevice, h->stream));
    return SV_OK;
}
sv_status sv_get_state(sv_handle h, void* dev_dst) {
    if (check_handle(h) || !dev_dst) return fail(SV_ERR_ARG, "null argument");
    SV_CUDA(cudaMemcpyAsync(dev_dst, h->psi, state_bytes(h), cudaMemcpyDeviceToDevice, h->stream));
    return SV_OK;
}
sv_status sv_set_state_host(sv_handle h, const void* host_src) {
    if (check_handle(h) || !host_src) return fail(SV_ERR_ARG, "null argument");
    SV_CUDA(cudaMemcpyAsync(h->psi, host_src, state_bytes(h), cudaMemcpyHostToDevice, h->stream));
    return SV_OK;
}
sv_status sv_get_state_host(sv_handle h, void* host_dst) {
    if (check_handle(h) || !host_dst) return fail(SV_ERR_ARG, "null argument");
    SV_CUDA(cudaMemcpyAsync(host_dst, h->psi, state_bytes(h), cudaMemcpyDeviceToHost, h->stream));
    SV_CUDA(cudaStreamSynchronize(h->stream));
    return jflag_check(h);
}

sv_status sv_synchronize(sv_handle h) {
    if (check_handle(h)) return SV_ERR_ARG;
    SV_CUDA(cudaStreamSynchronize(h->stream));
    return jflag_check(h);
}

sv_status sv_last_run_info(sv_handle h, sv_run_info* out) {
    if (check_handle(h) || !out) return fail(SV_ERR_ARG, "null argument");
    *out = h->info;
    return SV_OK;
}

// ---------------- partitioning ----------------
static sv_status build_plan(const sv_circuit* c, uint32_t L, uint32_t n_fixed, sv_plan** out, bool strict = false) {
    if (!out) return fail(SV_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!c || (c->n_gates && !c->gates)) return fail(SV_ERR_ARG, "null circuit");
    if (c->n_qubits < 1 || c->n_qubits > (uint32_t)svk::kMaxQ) return fail(SV_ERR_ARG, "n_qubits out of range");
    if (L < 1 || L > (uint32_t)svk::kMaxT) return fail(SV_ERR_ARG, "L must be in [1, 14]");
    if (c->n_gates > 32768) return fail(SV_ERR_ARG, "more than 32768 gates");
    std::vector<svh::GateRec> gates;
    std::string gerr = svh::gates_from_circuit(c, &gates);
    if (!gerr.empty()) return fail(SV_ERR_ARG, gerr);
    sv_plan* p = new (std::nothrow) sv_plan();
    if (!p) return fail(SV_ERR_OOM, "host allocation failed");
    svh::Plan& P = p->plan;
    P.n = (int)c->n_qubits;
    P.n_params = (int)c->n_params;
    P.L = (int)L;
    P.gates = std::move(gates);
    svh::relabel(P.n, P.gates, &P.phys, &P.final_map);
    const int nf = (int)std::min<uint32_t>(n_fixed, std::min<uint32_t>(L, c->n_qubits));
    P.n_fixed = nf;
    const uint64_t fixed = nf ? ((1ull << nf) - 1) : 0;
    const uint64_t universe = (P.n >= 64) ? ~0ull : ((1ull << P.n) - 1);
    std::string err = svh::partition_core(P.n, P.phys, (int)L, fixed, universe, &P.top, &P.cc, strict);
    if (strict) P.gemm_k = (int)L;
    if (!err.empty()) {
        delete p;
        return fail(SV_ERR_PARTITION, err);
    }
    *out = p;
    return SV_OK;
}

sv_status sv_partition(const sv_circuit* circuit, uint32_t L, sv_plan** out) {
    // reserve the coalescing low bits, but always leave one free local qubit
    return build_plan(circuit, L, L > 1 ? std::min<uint32_t>(4, L - 1) : 0, out);
}
sv_status sv_partition_ex(const sv_circuit* circuit, uint32_t L, uint32_t n_fixed, sv_plan** out) {
    return build_plan(circuit, L, n_fixed, out);
}

sv_status sv_partition_gemm(const sv_circuit* circuit, uint32_t k, sv_plan** out) {
    if (k < 5 || k > 7) return fail(SV_ERR_ARG, "fusion width k must be 5, 6 or 7");
    return build_plan(circuit, k, 0, out, true);
}

sv_status sv_partition_hier(const sv_circuit* circuit, uint32_t k, sv_plan** out) {
    if (k != 5 && k != 6) return fail(SV_ERR_ARG, "sub-partition width k must be 5 or 6");
    if (!circuit || !out) return fail(SV_ERR_ARG, "null argument");
    if (circuit->n_qubits < k + 7) return fail(SV_ERR_UNSUPPORTED, "hierarchical stages need at least k + 7 qubits");
    sv_status s = build_plan(circuit, k + 7, 4, out, true);
    if (s) return s;
    (*out)->plan.gemm_k = 0;
    (*out)->plan.hier_k = (int)k;
    return SV_OK;
}

sv_status sv_hier_plan_info(const sv_plan* plan, const double* params, sv_prec prec, uint32_t* n_launches,
                            uint32_t* n_sub) {
    if (!plan) return fail(SV_ERR_ARG, "null argument");
    if (prec != SV_PREC_TF32X3 && prec != SV_PREC_BF16X3) return fail(SV_ERR_ARG, "bad precision");
    if (plan->plan.hier_k == 0) return fail(SV_ERR_UNSUPPORTED, "not a plan from sv_partition_hier");
    if (plan->plan.n_params > 0 && !params) return fail(SV_ERR_ARG, "params is NULL");
    svh::HierProgram hp;
    std::string err = svh::plan_hier(plan->plan, params, prec == SV_PREC_TF32X3 ? 1 : 2, &hp);
    if (!err.empty()) return fail(SV_ERR_UNSUPPORTED, err);
    if (n_launches) *n_launches = (uint32_t)hp.launches.size();
    if (n_sub) *n_sub = hp.n_sub;
    return SV_OK;
}

sv_status sv_gemm_plan_info(const sv_plan* plan, const double* params, sv_prec prec, uint32_t* n_stages,
                            uint32_t* keff, uint32_t* resident, uint32_t* nslot, uint8_t* lane_roles) {
    if (!plan || !n_stages) return fail(SV_ERR_ARG, "null argument");
    if (prec != SV_PREC_TF32X3 && prec != SV_PREC_BF16X3) return fail(SV_ERR_ARG, "bad precision");
    if (plan->plan.gemm_k == 0) return fail(SV_ERR_UNSUPPORTED, "tensor-core precision needs a plan from sv_partition_gemm");
    if (plan->plan.n_params > 0 && !params) return fail(SV_ERR_ARG, "params is NULL");
    svh::GemmProgram gp;
    std::string err = svh::plan_gemm(plan->plan, params, prec == SV_PREC_TF32X3 ? 1 : 2, &gp);
    if (!err.empty()) return fail(SV_ERR_UNSUPPORTED, err);
    if ((keff || resident || nslot || lane_roles) && *n_stages < gp.stages.size())
        return fail(SV_ERR_ARG, "arrays too small");
    *n_stages = (uint32_t)gp.stages.size();
    for (size_t i = 0; i < gp.stages.size(); ++i) {
        const svk::GemmStage& st = gp.stages[i];
        if (keff) keff[i] = st.keff;
        if (resident) resident[i] = st.resident;
        if (nslot) nslot[i] = st.nslot;
        if (lane_roles) {
            for (int l = 0; l < 5; ++l)   // producer lane bit l: chunk-varying bit pperm[l] (255: none)
                lane_roles[i * 6 + l] = (uint32_t)l + 1 < st.nvar ? st.var_role[st.pperm[l]] : (uint8_t)255;
            lane_roles[i * 6 + 5] = st.var_role[0];
        }
    }
    return SV_OK;
}

sv_status sv_plan_stages(const sv_plan* plan, uint32_t* n_stages, uint64_t* local_masks,
                         uint32_t* gate_counts) {
    if (!plan || !n_stages) return fail(SV_ERR_ARG, "null argument");
    const auto& top = plan->plan.top;
    if ((local_masks || gate_counts) && *n_stages < top.local.size())
        return fail(SV_ERR_ARG, "arrays too small");
    *n_stages = (uint32_t)top.local.size();
    for (size_t s = 0; s < top.local.size(); ++s) {
        if (local_masks) local_masks[s] = top.local[s];
        if (gate_counts) gate_counts[s] = (uint32_t)top.ids[s].size();
    }
    return SV_OK;
}

sv_status sv_plan_order(const sv_plan* plan, uint32_t* gate_order, uint32_t* final_map) {
    if (!plan) return fail(SV_ERR_ARG, "null plan");
    if (gate_order) {
        size_t k = 0;
        for (auto& ids : plan->plan.top.ids)
            for (uint32_t i : ids) gate_order[k++] = i;
    }
    if (final_map)
        for (int q = 0; q < plan->plan.n; ++q) final_map[q] = (uint32_t)plan->plan.final_map[q];
    return SV_OK;
}

sv_status sv_plan_centrality(const sv_plan* plan, uint32_t* reach, uint64_t* dist, uint32_t* level) {
    if (!plan) return fail(SV_ERR_ARG, "null plan");
    const auto& cc = plan->plan.cc;
    for (size_t i = 0; i < cc.reach.size(); ++i) {
        if (reach) reach[i] = cc.reach[i];
        if (dist) dist[i] = cc.dist[i];
        if (level) level[i] = cc.level[i];
    }
    return SV_OK;
}

sv_status sv_plan_destroy(sv_plan* plan) {
    delete plan;
    return SV_OK;
}

// ---------------- execution ----------------
// Register-group width (amplitudes per thread = 2^R); SVGB_RMAX_FWD / SVGB_RMAX_BWD
// override the defaults for tuning.
static int env_int(const char* name, int dflt, int lo, int hi) {
    const char* v = getenv(name);
    if (!v) return dflt;
    int x = atoi(v);
    return x < lo ? lo : (x > hi ? hi : x);
}
static int rmax_fwd(int eb) { return eb == 8 ? env_int("SVGB_RMAX_FWD", 4, 1, 5) : env_int("SVGB_RMAX_FWD", 4, 1, 4); }
static int rmax_bwd(int eb) { return eb == 8 ? env_int("SVGB_RMAX_BWD", 4, 1, 4) : env_int("SVGB_RMAX_BWD", 3, 1, 3); }

// ---------------- generated (run-time compiled) stage kernels ----------------
// complex64 stage sweeps run as kernels generated per stage (jit.h); SVGB_JIT=0 selects
// the generic interpreter kernel instead (both are GPU paths; there is no CPU path).
static bool jit_enabled(sv_handle h) { return h->eb == 8 && env_int("SVGB_JIT", 1, 0, 1) == 1; }
// generated forward sweeps: stages needing 4+ register groups at R = 4 may use R = 5
// (SVGB_RWIDE_FWD=5; off by default: measured slower on QFT30, 26.8 -> 28.9 ms)
static int rwide_fwd() { return env_int("SVGB_RWIDE_FWD", 0, 0, 5); }

// Generated stages are memoised by the exact bytes of their lowered program section
// (a pure function of those bytes), so repeated runs skip the generation; the memo is
// dropped when it grows large (kernels themselves stay cached by source).
static std::mutex g_jit_mu;
static std::unordered_map<std::string, std::shared_ptr<svj::Built>> g_jit_memo;

// dst_last: the last stage writes out of place through this bit map (StageView::dst)
static sv_status jit_prepare(uint32_t n, const svh::Packed& pk, int nv,
                             std::vector<std::shared_ptr<svj::Built>>* out, const int* dst_last = nullptr) {
    const uint8_t* blob = pk.blob.data();
    const auto* groups = (const svk::Group*)(blob + pk.group_off);
    const auto* ops = (const svk::DevOp<float>*)(blob + pk.op_off);
    const auto* terms = (const svk::DevTerm<float>*)(blob + pk.term_off);
    const auto* slots = (const svk::PhaseSlot<float>*)(blob + pk.slot_off);
    out->clear();
    std::vector<svj::Built*> fresh;
    for (const svk::Stage& st : pk.stages) {
        svj::StageView v{&st, groups + st.group_off, ops + st.op_off, terms, slots + st.phase_off, (int)n, nv};
        std::string key;
        if (dst_last && &st == &pk.stages.back()) {
            v.dst = dst_last;
            key.append("P");
            key.append((const char*)dst_last, n * sizeof(int));
        }
        key.append((const char*)&nv, sizeof(nv));
        key.append((const char*)&n, sizeof(n));
        key.append((const char*)&st, sizeof(st));
        key.append((const char*)v.groups, st.n_groups * sizeof(svk::Group));
        key.append((const char*)v.ops, st.n_ops * sizeof(svk::DevOp<float>));
        key.append((const char*)v.slots, st.n_phase * sizeof(svk::PhaseSlot<float>));
        for (uint32_t i = 0; i < st.n_ops; ++i)
            if (v.ops[i].flags & svk::F_TERMS)
                key.append((const char*)(terms + v.ops[i].term_off), v.ops[i].n_terms * sizeof(svk::DevTerm<float>));
        for (uint32_t p = 0; p < st.n_phase; ++p)
            key.append((const char*)(terms + v.slots[p].glob_off), v.slots[p].n_glob * sizeof(svk::DevTerm<float>));
        std::shared_ptr<svj::Built> b;
        {
            std::lock_guard<std::mutex> lk(g_jit_mu);
            auto it = g_jit_memo.find(key);
            if (it != g_jit_memo.end()) b = it->second;
        }
        if (!b) {
            b = std::make_shared<svj::Built>();
            std::string err = svj::generate(v, b.get());
            if (!err.empty()) return fail(SV_ERR_UNSUPPORTED, err);
            if (b->smem > 227 * 1024) return fail(SV_ERR_UNSUPPORTED, "a generated stage needs more shared memory than a CTA has");
            fresh.push_back(b.get());
            std::lock_guard<std::mutex> lk(g_jit_mu);
            if (g_jit_memo.size() > 4096) g_jit_memo.clear();
            g_jit_memo[key] = b;
        }
        out->push_back(b);
    }
    if (!fresh.empty()) {
        std::string err = svj::compile(fresh);
        if (!err.empty()) return fail(SV_ERR_CUDA, "run-time compilation of a stage kernel failed: " + err);
    }
    for (auto& b : *out)
        if (!b->kernel) return fail(SV_ERR_CUDA, "internal: stage kernel missing");
    return SV_OK;
}

static sv_status run_forward(sv_handle h, const sv_plan* plan, const double* params, bool permute_back) {
    const svh::Plan& P = plan->plan;
    svh::Program prog;
    const bool jit = jit_enabled(h);
    // generated kernels fuse the final permutation into the last stage's write-back
    const bool fuse = jit && permute_back && env_int("SVGB_FUSE_PERM", 1, 0, 1) == 1;
    std::string err = svh::lower(P, params, h->eb, rmax_fwd(h->eb), false, &prog, false, jit ? rwide_fwd() : 0, fuse);
    if (!err.empty()) return fail(SV_ERR_ARG, err);
    for (auto& st : prog.stages)
        if (((size_t)h->eb << st.T) > 227 * 1024) return fail(SV_ERR_UNSUPPORTED, "tile too wide for shared memory at this dtype (use L <= 13 for complex128)");
    std::vector<std::shared_ptr<svj::Built>> built;
    sv_status s = SV_OK;
    int* flag = nullptr;
    if (jit) {
        err = svh::pack(prog, (int)h->n, h->eb, &h->fwd.packed);
        if (!err.empty()) return fail(SV_ERR_ARG, err);
        s = jit_prepare(h->n, h->fwd.packed, 1, &built, prog.fused_perm ? prog.dst.data() : nullptr);
        if (!s) s = jflag_device(h, &flag);
        if (!s && prog.fused_perm && cudaSuccess != h->scratch.ensure(state_bytes(h)))
            return fail(SV_ERR_CUDA, "could not allocate the permuted stage's output buffer");
    } else {
        s = upload_program(h, prog, &h->fwd, false);
    }
    if (s) return s;
    const auto& stages = h->fwd.packed.stages;
    for (size_t i = 0; i < stages.size(); ++i) {
        cudaEvent_t t0 = tick(h);
        const bool outp = jit && prog.fused_perm && i + 1 == stages.size();
        if (jit)
            SV_CUDA(svj::launch(*built[i], h->psi, outp ? h->scratch.p : nullptr, nullptr, flag, h->stream, nullptr));
        else
            SV_CUDA(svk::launch_stage_fwd(h->eb, h->fwd.launch(i, h->psi, nullptr, nullptr), stages[i], h->stream));
        tock(h, t0, TK_STAGE);
        h->info.stage_sweeps += 1;
        h->info.kernel_launches += 1;
        h->info.hbm_bytes += 2.0 * (double)state_bytes(h);
    }
    if (prog.fused_perm) {
        // the permuted state is in the second buffer: a handle that owns its state takes
        // that buffer as the state, a caller's buffer receives a copy
        if (h->owns) {
            std::swap(h->psi, h->scratch.p);
        } else {
            SV_CUDA(cudaMemcpyAsync(h->psi, h->scratch.p, state_bytes(h), cudaMemcpyDeviceToDevice, h->stream));
            h->info.hbm_bytes += 2.0 * (double)state_bytes(h);
        }
    } else if (permute_back && !prog.identity_map) {
        std::vector<uint32_t> m(P.n);
        for (int q = 0; q < P.n; ++q) m[q] = (uint32_t)P.final_map[q];
        s = do_permute(h, m.data());
        if (s) return s;
    }
    return SV_OK;
}

// FP64 norm of the state into the handle's reduction slot `slot` (device double)
static sv_status norm_to(sv_handle h, int slot) {
    SV_CUDA(h->red.ensure((152 * 16 + 16) * sizeof(double)));
    double* part = (double*)h->red.p + 16;
    uint32_t nb = 0;
    cudaEvent_t t0 = tick(h);
    SV_CUDA(svk::launch_norm(h->eb, h->psi, 1ull << h->n, part, &nb, h->stream));
    tock(h, t0, TK_OBS);
    SV_CUDA(svk::launch_reduce_rows(part, nb, 1, (double*)h->red.p + slot, h->stream));
    h->info.kernel_launches += 2;
    h->info.hbm_bytes += (double)state_bytes(h);
    return SV_OK;
}

// After tensor-core stages: scale the state back to the norm it had before them (the
// accumulators' round-toward-zero shrinks every fused stage's output slightly; the
// stages are unitary, so the exact result has the input's norm)
static sv_status restore_norm(sv_handle h) {
    sv_status s = norm_to(h, 3);
    if (s) return s;
    const double* r = (const double*)h->red.p;
    SV_CUDA(svk::launch_scale_to_norm(h->eb, h->psi, 1ull << h->n, r + 2, r + 3, h->stream));
    h->info.kernel_launches += 1;
    h->info.hbm_bytes += 2.0 * (double)state_bytes(h);
    return SV_OK;
}

// hierarchical tensor-core stages: one launch per run of sub-partitions of a stage
static sv_status run_hier(sv_handle h, const sv_plan* plan, const double* params, int prec, bool renorm) {
    const svh::Plan& P = plan->plan;
    svh::HierProgram hp;
    std::string err = svh::plan_hier(P, params, prec, &hp);
    if (!err.empty()) return fail(SV_ERR_UNSUPPORTED, err);
    const size_t sb = hp.launches.size() * sizeof(svk::HierStage);
    const size_t aoff = (sb + 1023) & ~(size_t)1023;
    const size_t total = aoff + hp.ublob.size();
    SV_CUDA(h->gemm.ensure(total));
    SV_CUDA(h->status.ensure(sizeof(int)));
    h->gemm_host.assign(total, 0);
    std::memcpy(h->gemm_host.data(), hp.launches.data(), sb);
    std::memcpy(h->gemm_host.data() + aoff, hp.ublob.data(), hp.ublob.size());
    SV_CUDA(cudaMemcpyAsync(h->gemm.p, h->gemm_host.data(), total, cudaMemcpyHostToDevice, h->stream));
    SV_CUDA(cudaMemsetAsync(h->status.p, 0, sizeof(int), h->stream));
    if (renorm) {
        sv_status s0 = norm_to(h, 2);
        if (s0) return s0;
    }
    for (size_t i = 0; i < hp.launches.size(); ++i) {
        cudaEvent_t t0 = tick(h);
        SV_CUDA(svk::launch_hier_stage(prec, h->psi, (const svk::HierStage*)h->gemm.p + i, hp.launches[i],
                                       (const uint8_t*)h->gemm.p + aoff, (int*)h->status.p, h->stream));
        tock(h, t0, TK_STAGE);
        h->info.stage_sweeps += 1;
        h->info.kernel_launches += 1;
        h->info.hbm_bytes += 2.0 * (double)state_bytes(h);
    }
    if (!hp.identity_map) {
        std::vector<uint32_t> m(P.n);
        for (int q = 0; q < P.n; ++q) m[q] = (uint32_t)P.final_map[q];
        sv_status s = do_permute(h, m.data());
        if (s) return s;
    }
    if (renorm) {
        sv_status s = restore_norm(h);
        if (s) return s;
    }
    int st = 0;
    SV_CUDA(cudaMemcpyAsync(&st, h->status.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    SV_CUDA(cudaStreamSynchronize(h->stream));
    if (st) return fail(SV_ERR_TIMEOUT, "a hierarchical tensor-core stage gave up waiting for its copies or MMAs");
    return SV_OK;
}

static sv_status run_gemm(sv_handle h, const sv_plan* plan, const double* params, int prec, bool renorm) {
    const svh::Plan& P = plan->plan;
    svh::GemmProgram gp;
    std::string err = svh::plan_gemm(P, params, prec, &gp);
    if (!err.empty()) return fail(SV_ERR_UNSUPPORTED, err);
    const size_t sb = gp.stages.size() * sizeof(svk::GemmStage);
    const size_t aoff = align16(sb);
    const size_t total = aoff + gp.ublob.size();
    for (auto& st : gp.stages)
        if (svk::gemm_smem_bytes(st) > 227 * 1024) return fail(SV_ERR_UNSUPPORTED, "tensor-core stage too wide");
    SV_CUDA(h->gemm.ensure(total));
    SV_CUDA(h->status.ensure(sizeof(int)));
    h->gemm_host.assign(total, 0);
    std::memcpy(h->gemm_host.data(), gp.stages.data(), sb);
    std::memcpy(h->gemm_host.data() + aoff, gp.ublob.data(), gp.ublob.size());
    SV_CUDA(cudaMemcpyAsync(h->gemm.p, h->gemm_host.data(), total, cudaMemcpyHostToDevice, h->stream));
    SV_CUDA(cudaMemsetAsync(h->status.p, 0, sizeof(int), h->stream));
    if (renorm) {
        sv_status s0 = norm_to(h, 2);
        if (s0) return s0;
    }
    for (size_t i = 0; i < gp.stages.size(); ++i) {
        cudaEvent_t t0 = tick(h);
        SV_CUDA(svk::launch_gemm_stage(prec, h->psi, (const svk::GemmStage*)h->gemm.p + i, gp.stages[i],
                                       (const uint8_t*)h->gemm.p + aoff, (int*)h->status.p, h->stream));
        tock(h, t0, TK_STAGE);
        h->info.stage_sweeps += 1;
        h->info.kernel_launches += 1;
        h->info.hbm_bytes += 2.0 * (double)state_bytes(h);
    }
    if (!gp.identity_map) {
        std::vector<uint32_t> m(P.n);
        for (int q = 0; q < P.n; ++q) m[q] = (uint32_t)P.final_map[q];
        sv_status s = do_permute(h, m.data());
        if (s) return s;
    }
    if (renorm) {
        sv_status s = restore_norm(h);
        if (s) return s;
    }
    int st = 0;
    SV_CUDA(cudaMemcpyAsync(&st, h->status.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    SV_CUDA(cudaStreamSynchronize(h->stream));
    if (st) return fail(SV_ERR_TIMEOUT, "a tensor-core stage gave up waiting for its MMAs");
    return SV_OK;
}

sv_status sv_plan_compile(const sv_plan* plan, const double* params, uint32_t which, uint32_t* n_kernels) {
    if (!plan || which == 0 || which > 3) return fail(SV_ERR_ARG, "null plan or bad direction mask");
    const svh::Plan& P = plan->plan;
    if (P.n_params > 0 && !params) return fail(SV_ERR_ARG, "params is NULL");
    if (P.gemm_k) return fail(SV_ERR_UNSUPPORTED, "tensor-core plans run the tcgen05 stage kernel, nothing to compile");
    uint32_t count = 0;
    for (int d = 0; d < 2; ++d) {
        if (!((which >> d) & 1)) continue;
        svh::Program prog;
        const bool fuse = d == 0 && env_int("SVGB_FUSE_PERM", 1, 0, 1) == 1;   // as sv_run lowers it
        std::string err = svh::lower(P, params, 8, d ? rmax_bwd(8) : rmax_fwd(8), d == 1, &prog, false, d ? 0 : rwide_fwd(), fuse);
        if (!err.empty()) return fail(err.find("not supported") != std::string::npos ? SV_ERR_UNSUPPORTED : SV_ERR_ARG, err);
        svh::Packed pk;
        err = svh::pack(prog, P.n, 8, &pk);
        if (!err.empty()) return fail(SV_ERR_ARG, err);
        std::vector<std::shared_ptr<svj::Built>> built;
        sv_status s = jit_prepare((uint32_t)P.n, pk, d + 1, &built, prog.fused_perm ? prog.dst.data() : nullptr);
        if (s) return s;
        count += (uint32_t)built.size();
    }
    if (n_kernels) *n_kernels = count;
    return SV_OK;
}

sv_status sv_pauli_compile(uint32_t n_qubits, sv_dtype dtype, const sv_observable* obs, uint32_t* n_kernels) {
    if (n_qubits < 1 || n_qubits > 40 || (dtype != SV_C64 && dtype != SV_C128)) return fail(SV_ERR_ARG, "bad width or dtype");
    std::vector<int> ident(n_qubits);
    for (uint32_t q = 0; q < n_qubits; ++q) ident[q] = (int)q;
    PauliPlan pp;
    sv_status s = plan_pauli((int)n_qubits, dtype == SV_C64 ? 8 : 16, obs, ident, &pp);
    if (s) return s;
    std::vector<std::shared_ptr<svj::Built>> built;
    sv_status js = SV_OK;
    const bool gen = pauli_jit((int)n_qubits, dtype == SV_C64 ? 8 : 16, pp, &built, &js);
    if (js) return js;
    if (n_kernels) *n_kernels = gen ? (uint32_t)built.size() : 0u;
    return SV_OK;
}

sv_status sv_jit_stats(uint64_t* compiles, uint64_t* cache_hits, double* compile_ms) {
    svj::stats(compiles, cache_hits, compile_ms);
    return SV_OK;
}

sv_status sv_run(sv_handle h, const sv_plan* plan, const double* params, sv_prec prec) {
    if (check_handle(h) || !plan) return fail(SV_ERR_ARG, "null argument");
    if (plan->plan.n != (int)h->n) return fail(SV_ERR_ARG, "plan width differs from the state");
    if (plan->plan.n_params > 0 && !params) return fail(SV_ERR_ARG, "params is NULL");
    h->info = sv_run_info{};
    const int mode = (int)prec & ~(int)SV_PREC_NO_RENORM;
    const bool renorm = ((int)prec & (int)SV_PREC_NO_RENORM) == 0;
    if (mode == SV_PREC_TF32X3 || mode == SV_PREC_BF16X3) {
        if (plan->plan.gemm_k == 0 && plan->plan.hier_k == 0)
            return fail(SV_ERR_UNSUPPORTED, "tensor-core precision needs a plan from sv_partition_gemm or sv_partition_hier");
        if (h->dt != SV_C64) return fail(SV_ERR_UNSUPPORTED, "tensor-core stages operate on complex64 states");
        if (plan->plan.hier_k) return run_hier(h, plan, params, mode == SV_PREC_TF32X3 ? 1 : 2, renorm);
        return run_gemm(h, plan, params, mode == SV_PREC_TF32X3 ? 1 : 2, renorm);
    }
    if (prec != SV_PREC_CUDACORE) return fail(SV_ERR_ARG, "bad precision");
    return run_forward(h, plan, params, true);
}

sv_status sv_permute(sv_handle h, const uint32_t* phys_of_qubit) {
    if (check_handle(h) || !phys_of_qubit) return fail(SV_ERR_ARG, "null argument");
    return do_permute(h, phys_of_qubit);
}

sv_status sv_norm(sv_handle h, double* out) {
    if (check_handle(h) || !out) return fail(SV_ERR_ARG, "null argument");
    SV_CUDA(h->red.ensure((152 * 16 + 16) * sizeof(double)));
    double* part = (double*)h->red.p + 16;
    uint32_t nb = 0;
    cudaEvent_t t0 = tick(h);
    SV_CUDA(svk::launch_norm(h->eb, h->psi, 1ull << h->n, part, &nb, h->stream));
    tock(h, t0, TK_OBS);
    h->info.kernel_launches += 2;
    SV_CUDA(svk::launch_reduce_rows(part, nb, 1, (double*)h->red.p, h->stream));
    SV_CUDA(cudaMemcpyAsync(out, h->red.p, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    SV_CUDA(cudaStreamSynchronize(h->stream));
    return jflag_check(h);
}

sv_status sv_expval(sv_handle h, const sv_observable* obs, double* out) {
    if (check_handle(h) || !out) return fail(SV_ERR_ARG, "null argument");
    std::vector<int> ident(h->n);
    for (uint32_t q = 0; q < h->n; ++q) ident[q] = (int)q;
    PauliPlan pp;
    sv_status s = plan_pauli((int)h->n, h->eb, obs, ident, &pp);
    if (s) return s;
    s = run_pauli(h, pp, nullptr);
    if (s) return s;
    SV_CUDA(cudaMemcpyAsync(out, h->red.p, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    SV_CUDA(cudaStreamSynchronize(h->stream));
    return jflag_check(h);
}

sv_status sv_permute_plan_info(uint32_t n_qubits, sv_dtype dtype, const uint32_t* phys_of_qubit, uint32_t* tile_bits,
                               uint64_t* tile_mask, uint32_t* in_run, uint32_t* out_run) {
    if (!phys_of_qubit || !tile_bits || !tile_mask || !in_run || !out_run) return fail(SV_ERR_ARG, "null argument");
    if (n_qubits < 1 || n_qubits > (uint32_t)svk::kMaxQ) return fail(SV_ERR_ARG, "n_qubits out of range");
    if (dtype != SV_C64 && dtype != SV_C128) return fail(SV_ERR_ARG, "bad dtype");
    const int n = (int)n_qubits;
    int dst[64];
    if (!perm_dst(n, phys_of_qubit, dst)) return fail(SV_ERR_ARG, "not a permutation");
    int T = 0;
    const uint64_t B = perm_tile(n, dtype == SV_C64 ? 8 : 16, phys_of_qubit, dst, &T);
    uint32_t ri = 0, ro = 0;
    while ((int)ri < n && ((B >> ri) & 1)) ++ri;
    while ((int)ro < n && ((B >> phys_of_qubit[ro]) & 1)) ++ro;
    *tile_bits = (uint32_t)T;
    *tile_mask = B;
    *in_run = ri;
    *out_run = ro;
    return SV_OK;
}

sv_status sv_pauli_plan_info(uint32_t n_qubits, sv_dtype dtype, const sv_observable* obs, uint32_t* n_sweeps,
                             uint64_t* tile_masks, uint64_t* reg_masks, uint32_t* n_terms) {
    if (!obs || !n_sweeps) return fail(SV_ERR_ARG, "null argument");
    if (n_qubits < 1 || n_qubits > 34) return fail(SV_ERR_ARG, "n_qubits must be in [1, 34]");
    if (dtype != SV_C64 && dtype != SV_C128) return fail(SV_ERR_ARG, "bad dtype");
    std::vector<int> ident(n_qubits);
    for (uint32_t q = 0; q < n_qubits; ++q) ident[q] = (int)q;
    PauliPlan pp;
    sv_status s = plan_pauli((int)n_qubits, dtype == SV_C64 ? 8 : 16, obs, ident, &pp);
    if (s) return s;
    if ((tile_masks || reg_masks || n_terms) && *n_sweeps < pp.sweeps.size())
        return fail(SV_ERR_ARG, "arrays too small");
    *n_sweeps = (uint32_t)pp.sweeps.size();
    for (size_t i = 0; i < pp.sweeps.size(); ++i) {
        const svk::PauliSweep& sw = pp.sweeps[i];
        uint64_t t = 0, r = 0;
        for (uint32_t b = 0; b < sw.T; ++b) t |= sw.ptile[b];
        for (uint32_t b = sw.L; b < sw.L + sw.R; ++b) r |= sw.ptile[b];
        if (tile_masks) tile_masks[i] = t;
        if (reg_masks) reg_masks[i] = r;
        if (n_terms) n_terms[i] = sw.n_terms;
    }
    return SV_OK;
}

sv_status sv_grad(sv_handle h, const sv_plan* plan, const double* params, const sv_observable* obs,
                  double* expval_out, double* grad_out) {
    if (check_handle(h) || !plan || !obs) return fail(SV_ERR_ARG, "null argument");
    const svh::Plan& P = plan->plan;
    if (P.n != (int)h->n) return fail(SV_ERR_ARG, "plan width differs from the state");
    if (P.n_params > 0 && (!params || !grad_out)) return fail(SV_ERR_ARG, "params / grad_out is NULL");
    h->info = sv_run_info{};
    // lower the backward program first so unsupported parameters fail before any work
    svh::Program bprog;
    std::string err = svh::lower(P, params, h->eb, rmax_bwd(h->eb), true, &bprog);
    if (!err.empty()) return fail(err.find("not supported") != std::string::npos ? SV_ERR_UNSUPPORTED : SV_ERR_ARG, err);
    for (auto& st : bprog.stages)
        if (((size_t)h->eb << (st.T + 1)) > 200 * 1024 || (st.T - st.R) > 9)
            return fail(SV_ERR_UNSUPPORTED, "tile too wide for the adjoint sweep (psi and lambda tiles must fit shared memory)");
    sv_status s = run_forward(h, plan, params, false);
    if (s) return s;
    // lambda = O psi in the forward program's final physical layout
    PauliPlan pp;
    s = plan_pauli((int)h->n, h->eb, obs, P.final_map, &pp);
    if (s) return s;
    SV_CUDA(h->scratch.ensure(state_bytes(h)));
    s = run_pauli(h, pp, h->scratch.p);
    if (s) return s;
    double E = 0.0;
    SV_CUDA(cudaMemcpyAsync(&E, h->red.p, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    const bool jit = jit_enabled(h);
    std::vector<std::shared_ptr<svj::Built>> built;
    int* flag = nullptr;
    if (jit) {
        err = svh::pack(bprog, (int)h->n, h->eb, &h->bwd.packed);
        if (!err.empty()) return fail(SV_ERR_ARG, err);
        s = jit_prepare(h->n, h->bwd.packed, 2, &built);
        if (!s) s = jflag_device(h, &flag);
    } else {
        s = upload_program(h, bprog, &h->bwd, true);
    }
    if (s) return s;
    const size_t nslots_total = bprog.slot_param.size();
    const auto& bst = h->bwd.packed.stages;
    size_t maxpart = 1;
    for (auto& st : bst)
        maxpart = std::max(maxpart, (size_t)st.n_slots << (h->n - st.T));
    SV_CUDA(h->partial.ensure(maxpart * sizeof(double)));
    SV_CUDA(h->slot_sum.ensure(std::max<size_t>(1, nslots_total) * sizeof(double)));
    for (size_t i = 0; i < bst.size(); ++i) {
        const svk::Stage& st = bst[i];
        const uint64_t ntiles = 1ull << (h->n - st.T);
        cudaEvent_t t0 = tick(h);
        uint32_t grid = 0;
        if (jit)
            SV_CUDA(svj::launch(*built[i], h->psi, h->scratch.p, (double*)h->partial.p, flag, h->stream, &grid));
        else
            SV_CUDA(svk::launch_stage_bwd(h->eb, h->bwd.launch(i, h->psi, h->scratch.p, (double*)h->partial.p),
                                          st, h->stream, &grid));
        tock(h, t0, TK_BWD);
        h->info.backward_sweeps += 1;
        h->info.kernel_launches += 1;
        h->info.hbm_bytes += 4.0 * (double)state_bytes(h);
        (void)ntiles;
        if (st.n_slots) {
            SV_CUDA(svk::launch_reduce_rows((double*)h->partial.p, grid, st.n_slots,
                                            (double*)h->slot_sum.p + st.slot_off, h->stream));
            h->info.kernel_launches += 1;
        }
    }
    std::vector<double> slots(nslots_total);
    if (nslots_total)
        SV_CUDA(cudaMemcpyAsync(slots.data(), h->slot_sum.p, nslots_total * sizeof(double),
                                cudaMemcpyDeviceToHost, h->stream));
    SV_CUDA(cudaStreamSynchronize(h->stream));
    s = jflag_check(h);
    if (s) return s;
    if (expval_out) *expval_out = E;
    if (grad_out) {
        for (int k = 0; k < P.n_params; ++k) grad_out[k] = 0.0;
        for (size_t i = 0; i < nslots_total; ++i) grad_out[bprog.slot_param[i]] += slots[i];
    }
    return SV_OK;
}

}  // extern "C"
