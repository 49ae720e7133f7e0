// lower.cpp — turn a partition into the device program of one direction.
//
// For each partition (stage) the tile bits are its local set (Sec. 4.3: the state
// tensor is split on the partition's global dimensions, each tile packed into
// shared memory).  Inside a stage the partitioner is invoked again with the
// register budget R (the next memory level, Sec. 4.2: "the algorithm can be invoked
// for each of the newly determined partitions"), giving register groups.
//
// Gates become micro-ops on the amplitudes a thread holds.  Diagonal gates (Z, S,
// T, P, RZ, CZ, CP) are kept as phase terms and applied just before the next dense
// gate on one of their qubits, or at the end of the circuit: they commute with
// every gate in between, so the product is unchanged (only rounding differs).  A
// term on the dense gate's target and a non-register bit becomes a twiddle of that
// gate (the linear phase a butterfly needs); a term on two register bits is applied
// directly.  SWAP is a relabel and emits nothing.
//
// Backward (adjoint) programs visit the stages and their gates in reverse with every
// gate conjugate-transposed, and emit, for each parametric rotation
// U = exp(-i theta G / 2) (G = X, Y, Z), an op accumulating Im <lambda|G|psi> at the
// gate's position, which equals dE/dtheta = 2 Re <lambda| dU/dtheta psi>.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>

#include "planner.h"

namespace svh {

namespace {

struct Pend {
    double angle = 0.0;
    std::vector<int> params;   // RZ parameters whose gradient is evaluated at emission
};

class Lowerer {
  public:
    Lowerer(const Plan& p, const double* params, int eb, int rmax, bool bwd, bool bind, Program* out, int rwide,
            bool fuse_perm)
        : P_(p), params_(params), eb_(eb), rmax_(rmax), rwide_(rwide), bwd_(bwd), bind_(bind), fuse_perm_(fuse_perm),
          out_(out) {}

    std::string run();

  private:
    uint64_t output_tile(int s, uint64_t tile) const;
    const Plan& P_;
    const double* params_;
    int eb_, rmax_, rwide_;
    bool bwd_, bind_, fuse_perm_;
    Program* out_;
    std::map<uint64_t, Pend> pending_;
    double gphase_ = 0.0;
    int regidx_[64];
    svk::Group* grp_ = nullptr;
    int grp_R_ = 0;   // register bits of the current group
    uint32_t stage_slots_ = 0;
    uint32_t slot_base_ = 0;

    double theta(const GateRec& g, int i = 0) const {
        if (g.param >= 0) return params_ ? params_[g.param] : 0.0;   // bind mode: formed on the device
        return g.angle[i];
    }
    svk::Op& new_op(uint8_t type, int j) {
        out_->ops.emplace_back();
        svk::Op& o = out_->ops.back();
        std::memset(&o, 0, sizeof(o));
        o.type = type;
        o.j = (uint8_t)j;
        grp_->n_ops++;
        return o;
    }
    int new_slot(int param) {
        out_->slot_param.push_back(param);
        return (int)(stage_slots_++);
    }
    void add_term(uint64_t mask, double angle, int param) {
        Pend& p = pending_[mask];
        p.angle += angle;
        if (param >= 0) p.params.push_back(param);
    }
    void emit_grad_z(int bit, int param);
    // Apply the pending terms on bit t before a dense gate on t.  Terms on t and a
    // register partner become PHASE2 ops; the rest (a constant and single-bit terms on
    // non-register bits) is either emitted as a PHASE1 op or, when fuse is set,
    // returned for the dense op to apply as its twiddle.
    void flush_bit(int t, bool fuse, double* cangle_out, std::vector<svk::Term>* terms_out,
                   std::map<int, double>* pairs_out = nullptr);
    void flush_all();
    std::string gate(const GateRec& g, const PGate& pg);
    std::string stage(int s);
};

void Lowerer::emit_grad_z(int bit, int param) {
    int r = regidx_[bit];
    svk::Op& o = new_op(svk::OP_GRAD_Z, r >= 0 ? r : 0);
    o.u = r >= 0 ? 0 : 1;
    o.ctrl_fix = r >= 0 ? 0 : (1ull << bit);
    o.slot = (uint32_t)new_slot(param);
}

// Apply every pending term that involves physical bit t (a register bit of the
// current group) — right before a dense gate on t.
void Lowerer::flush_bit(int t, bool fuse, double* cangle_out, std::vector<svk::Term>* terms_out,
                        std::map<int, double>* pairs_out) {
    const uint64_t tb = 1ull << t;
    const int jt = regidx_[t];
    double cangle = 0.0;
    bool any1 = false;
    std::vector<svk::Term> terms;
    std::map<int, double> pair;
    for (auto it = pending_.begin(); it != pending_.end();) {
        if (!(it->first & tb)) {
            ++it;
            continue;
        }
        if (bwd_)
            for (int prm : it->second.params) emit_grad_z(t, prm);
        uint64_t other = it->first & ~tb;
        if (other == 0) {
            cangle += it->second.angle;
            any1 = true;
        } else {
            int u = __builtin_ctzll(other);
            if (regidx_[u] >= 0) {
                pair[regidx_[u]] += it->second.angle;
            } else {
                terms.push_back(svk::Term{other, it->second.angle});
                any1 = true;
            }
        }
        it = pending_.erase(it);
    }
    if (pairs_out) {   // the dense op applies them (register bit -> angle)
        *pairs_out = pair;
        pair.clear();
    }
    for (auto& kv : pair) {   // diagonal: order among the phases is free
        int a = jt, b = kv.first;
        if (a > b) std::swap(a, b);
        svk::Op& o = new_op(svk::OP_PHASE2, a);
        o.u = (uint8_t)b;
        o.m[0] = std::cos(kv.second);
        o.m[1] = std::sin(kv.second);
    }
    *cangle_out = 0.0;
    terms_out->clear();
    if (!any1) return;
    if (fuse) {
        *cangle_out = cangle;
        *terms_out = terms;
        return;
    }
    svk::Op& o = new_op(svk::OP_PHASE1, jt);
    o.m[0] = std::cos(cangle);
    o.m[1] = std::sin(cangle);
    o.term_off = (uint32_t)out_->terms.size();
    o.n_terms = (uint32_t)terms.size();
    for (auto& x : terms) out_->terms.push_back(x);
}

// End of the program: apply every remaining term and the global phase.
void Lowerer::flush_all() {
    if (bwd_) {
        for (auto& kv : pending_)
            for (int prm : kv.second.params) emit_grad_z(__builtin_ctzll(kv.first), prm);
    }
    std::vector<svk::Term> t0;
    std::map<int, std::pair<double, std::vector<svk::Term>>> t1;
    std::map<std::pair<int, int>, double> t2;
    for (auto& kv : pending_) {
        uint64_t m = kv.first;
        int regs[2], nreg = 0;
        uint64_t rest = 0;
        for (uint64_t x = m; x; x &= x - 1) {
            int b = __builtin_ctzll(x);
            if (regidx_[b] >= 0) regs[nreg++] = regidx_[b];
            else rest |= 1ull << b;
        }
        if (nreg == 0) {
            t0.push_back(svk::Term{m, kv.second.angle});
        } else if (nreg == 1) {
            auto& e = t1[regs[0]];
            if (rest == 0) e.first += kv.second.angle;
            else e.second.push_back(svk::Term{rest, kv.second.angle});
        } else {
            t2[{std::min(regs[0], regs[1]), std::max(regs[0], regs[1])}] += kv.second.angle;
        }
    }
    pending_.clear();
    {
        svk::Op& o = new_op(svk::OP_PHASE0, 0);
        o.m[0] = std::cos(gphase_);
        o.m[1] = std::sin(gphase_);
        o.term_off = (uint32_t)out_->terms.size();
        o.n_terms = (uint32_t)t0.size();
        for (auto& x : t0) out_->terms.push_back(x);
    }
    for (auto& kv : t1) {
        svk::Op& o = new_op(svk::OP_PHASE1, kv.first);
        o.m[0] = std::cos(kv.second.first);
        o.m[1] = std::sin(kv.second.first);
        o.term_off = (uint32_t)out_->terms.size();
        o.n_terms = (uint32_t)kv.second.second.size();
        for (auto& x : kv.second.second) out_->terms.push_back(x);
    }
    for (auto& kv : t2) {
        svk::Op& o = new_op(svk::OP_PHASE2, kv.first.first);
        o.u = (uint8_t)kv.first.second;
        o.m[0] = std::cos(kv.second);
        o.m[1] = std::sin(kv.second);
    }
}

// 2x2 matrices (row-major re,im pairs).  Backward uses the conjugate transpose.
static void set_m(double* m, double a, double b, double c, double d, double e, double f, double g,
                  double h) {
    m[0] = a; m[1] = b; m[2] = c; m[3] = d; m[4] = e; m[5] = f; m[6] = g; m[7] = h;
}
static void dagger(double* m) {
    double r[8];
    // (U^dagger)_{ij} = conj(U_{ji})
    r[0] = m[0]; r[1] = -m[1];
    r[2] = m[4]; r[3] = -m[5];
    r[4] = m[2]; r[5] = -m[3];
    r[6] = m[6]; r[7] = -m[7];
    std::memcpy(m, r, sizeof(r));
}

std::string Lowerer::gate(const GateRec& g, const PGate& pg) {
    const double s = bwd_ ? -1.0 : 1.0;   // angle sign for diagonal terms
    switch (g.kind) {
        case K_SWAP:
            return "";
        case K_Z: add_term(1ull << pg.p[0], s * M_PI, -1); return "";
        case K_S: add_term(1ull << pg.p[0], s * M_PI / 2, -1); return "";
        case K_SDG: add_term(1ull << pg.p[0], -s * M_PI / 2, -1); return "";
        case K_T: add_term(1ull << pg.p[0], s * M_PI / 4, -1); return "";
        case K_TDG: add_term(1ull << pg.p[0], -s * M_PI / 4, -1); return "";
        case K_P:
            if (bind_ && g.param >= 0) return "a parametric P gate cannot be bound on the device";
            if (bwd_ && g.param >= 0) return "gradient of a P parameter is not supported";
            add_term(1ull << pg.p[0], s * theta(g), -1);
            return "";
        case K_RZ: {
            if (bind_ && g.param >= 0) break;   // dense op with a device-formed matrix
            double t = theta(g);
            gphase_ += -s * t / 2;
            add_term(1ull << pg.p[0], s * t, bwd_ ? g.param : -1);
            return "";
        }
        case K_CZ: add_term((1ull << pg.p[0]) | (1ull << pg.p[1]), s * M_PI, -1); return "";
        case K_CP:
            if (bind_ && g.param >= 0) return "a parametric CP gate cannot be bound on the device";
            if (bwd_ && g.param >= 0) return "gradient of a CP parameter is not supported";
            add_term((1ull << pg.p[0]) | (1ull << pg.p[1]), s * theta(g), -1);
            return "";
        default: break;
    }
    // dense gate on target t (controlled gates: q[1]); t is a register bit
    const int t = kind_is_controlled(g.kind) ? pg.p[1] : pg.p[0];
    const int jt = regidx_[t];
    if (jt < 0) return "internal: dense gate target is not a register bit";
    // The pending phase on t becomes the dense op's twiddle, except for a controlled
    // gate (the phase applies whatever the control is) and for a parametric gate of
    // the adjoint program (its gradient op must see the phase un-applied first).
    // A bound op's matrix is replaced on the device, so it takes no twiddle either.
    const bool fuse = !kind_is_controlled(g.kind) && !((bwd_ || bind_) && g.param >= 0);
    double tw_angle = 0.0;
    std::vector<svk::Term> tw_terms;
    // a real 2x2 (H, RY) also takes the pair phases on its target and another register
    // bit, when its group's other register bits fit the op's three spare slots
    const bool real_op = g.kind == K_H || g.kind == K_RY;
    const bool pair_fuse = fuse && real_op && grp_R_ <= 4 && !bwd_;   // forward programs only
    std::map<int, double> pairs;
    flush_bit(t, fuse, &tw_angle, &tw_terms, pair_fuse ? &pairs : nullptr);
    double m[8];
    uint8_t type = svk::OP_U;
    switch (g.kind) {
        case K_H: {
            double r = 1.0 / std::sqrt(2.0);
            set_m(m, r, 0, r, 0, r, 0, -r, 0);
            type = svk::OP_UR;
            break;
        }
        case K_X: case K_CX: set_m(m, 0, 0, 1, 0, 1, 0, 0, 0); type = svk::OP_X; break;
        case K_Y: case K_CY: set_m(m, 0, 0, 0, -1, 0, 1, 0, 0); break;
        case K_RX: {
            double c = std::cos(theta(g) / 2), sn = std::sin(theta(g) / 2);
            set_m(m, c, 0, 0, -sn, 0, -sn, c, 0);
            break;
        }
        case K_RY: {
            double c = std::cos(theta(g) / 2), sn = std::sin(theta(g) / 2);
            set_m(m, c, 0, -sn, 0, sn, 0, c, 0);
            type = svk::OP_UR;
            break;
        }
        case K_RZ: {   // bind mode only: diag(exp(-i t/2), exp(i t/2))
            double c = std::cos(theta(g) / 2), sn = std::sin(theta(g) / 2);
            set_m(m, c, -sn, 0, 0, 0, 0, c, sn);
            break;
        }
        case K_U3: {
            double th = g.angle[0], ph = g.angle[1], la = g.angle[2];
            double c = std::cos(th / 2), sn = std::sin(th / 2);
            set_m(m, c, 0, -std::cos(la) * sn, -std::sin(la) * sn, std::cos(ph) * sn, std::sin(ph) * sn,
                  std::cos(ph + la) * c, std::sin(ph + la) * c);
            break;
        }
        default: return "internal: unknown gate kind";
    }
    if (bwd_) {
        dagger(m);
        if (g.param >= 0) {
            if (g.kind != K_RX && g.kind != K_RY && g.kind != K_RZ)
                return "gradient of this parameter kind is not supported";
            svk::Op& go = new_op(g.kind == K_RX ? svk::OP_GRAD_X : g.kind == K_RY ? svk::OP_GRAD_Y : svk::OP_GRAD_Z, jt);
            go.slot = (uint32_t)new_slot(g.param);
        }
    }
    svk::Op& o = new_op(type, jt);
    std::memcpy(o.m, m, sizeof(m));
    if (!pairs.empty()) {
        if (type != svk::OP_UR) return "internal: pair phases on a complex dense op";
        o.has_pairs = 1;
        for (auto& kv : pairs) {
            const int idx = kv.first < jt ? kv.first : kv.first - 1;   // rank among the other bits
            o.pair_ang[idx] += kv.second;
        }
    }
    if (bind_ && g.param >= 0) {
        o.bparam1 = (uint32_t)g.param + 1;
        o.bkind = (uint8_t)((g.kind == K_RX ? svk::BK_RX : g.kind == K_RY ? svk::BK_RY : svk::BK_RZ) |
                            (bwd_ ? svk::BK_DAGGER : 0));
    }
    if (tw_angle != 0.0 || !tw_terms.empty()) {
        o.has_tw = 1;
        o.tw_angle = tw_angle;
        o.term_off = (uint32_t)out_->terms.size();
        o.n_terms = (uint32_t)tw_terms.size();
        for (auto& x : tw_terms) out_->terms.push_back(x);
    }
    if (kind_is_controlled(g.kind)) {
        int c = pg.p[0];
        if (regidx_[c] >= 0) o.ctrl_reg = 1u << regidx_[c];
        else o.ctrl_fix = 1ull << c;
    }
    return "";
}

// The last forward stage of a plan whose final map is not the identity writes its tile
// out of place through that map (the data reshaping of Sec. 4.3 fused into the stage's
// write-back).  Destination addresses are contiguous over the tile bits whose
// destinations are the lowest qubits, so local bits that no gate of the stage touches
// (the partitioner's fill, Sec. 4.2) are traded for the physical bits that land on
// qubits 0, 1, 2, ...: more local bits never make a stage wrong.
uint64_t Lowerer::output_tile(int s, uint64_t tile) const {
    const int n = P_.n;
    uint64_t keep = (eb_ == 8 ? 1ull : 0ull);
    for (int b = 0; b < P_.n_fixed && b < n; ++b) keep |= 1ull << b;
    for (uint32_t i : P_.top.ids[s]) {
        const GateRec& g = P_.gates[i];
        if (g.kind == K_SWAP) continue;   // a relabel: no op
        for (int k = 0; k < P_.phys[i].nq; ++k) keep |= 1ull << P_.phys[i].p[k];
    }
    uint64_t freeb = tile & ~keep;
    for (int q = 0; q < n && freeb; ++q) {
        const uint64_t want = 1ull << P_.final_map[q];   // physical bit that becomes qubit q
        if (tile & want) continue;
        const uint64_t drop = freeb & (~freeb + 1);      // lowest free bit
        tile = (tile & ~drop) | want;
        freeb &= ~drop;
    }
    return tile;
}

std::string Lowerer::stage(int s) {
    // complex64 tiles are staged in 16-byte chunks of two amplitudes, so the tile
    // always holds physical bit 0 (a plan without reserved low bits may not)
    uint64_t tile = P_.top.local[s] | (eb_ == 8 ? 1ull : 0ull);
    const int n = P_.n;
    if (fuse_perm_ && s == (int)P_.top.local.size() - 1) tile = output_tile(s, tile);
    svk::Stage st;
    std::memset(&st, 0, sizeof(st));
    int T = 0;
    for (int b = 0; b < n; ++b)
        if ((tile >> b) & 1) st.tile_pos[T++] = (uint8_t)b;
    if (T > svk::kMaxT) return "tile wider than 14 qubits";
    int ng = 0;
    for (int b = 0; b < n; ++b)
        if (!((tile >> b) & 1)) st.glob_pos[ng++] = (uint8_t)b;
    int R = std::min(rmax_, T);
    // at most 2^9 threads per tile: a 14-qubit complex64 forward tile takes 5 register bits
    if (T - R > 9 && eb_ == 8 && !bwd_) R = std::min(5, T);
    st.T = (uint32_t)T;
    st.n_glob = (uint32_t)ng;
    for (int b = 0; b < T; ++b) {
        st.ptile[b] = 1ull << st.tile_pos[b];
        st.swbit[b] = svk::swizzle(1u << b, eb_);
    }
    int tidx[64];
    for (int b = 0; b < 64; ++b) tidx[b] = -1;
    for (int b = 0; b < T; ++b) tidx[st.tile_pos[b]] = b;

    // stage gates in direction order, then the register-level partition
    std::vector<uint32_t> ids = P_.top.ids[s];
    if (bwd_) std::reverse(ids.begin(), ids.end());
    std::vector<PGate> sub;
    sub.reserve(ids.size());
    for (uint32_t i : ids) sub.push_back(P_.phys[i]);
    Partition groups;
    std::string err = partition_core(n, sub, R, 0, tile, &groups, nullptr);
    if (!err.empty()) return "register partition: " + err;
    // deep stages: a wider register level (more amplitudes per thread) when it needs
    // fewer register groups, i.e. fewer shared-memory exchanges per tile
    if (rwide_ > R && groups.local.size() >= 4 && std::min(rwide_, T) > R) {
        Partition wide;
        const int R2 = std::min(rwide_, T);
        if (partition_core(n, sub, R2, 0, tile, &wide, nullptr).empty() && wide.local.size() < groups.local.size()) {
            groups = wide;
            R = R2;
        }
    }
    st.R = (uint32_t)R;

    st.group_off = (uint32_t)out_->groups.size();
    st.n_groups = (uint32_t)groups.local.size();
    st.slot_off = slot_base_;
    stage_slots_ = 0;
    for (size_t gi = 0; gi < groups.local.size(); ++gi) {
        out_->groups.emplace_back();
        svk::Group& G = out_->groups.back();
        std::memset(&G, 0, sizeof(G));
        G.op_off = (uint32_t)out_->ops.size();
        grp_ = &G;
        grp_R_ = R;
        for (int b = 0; b < 64; ++b) regidx_[b] = -1;
        int nr = 0, nt = 0;
        for (int b = 0; b < T; ++b) {
            if ((groups.local[gi] >> st.tile_pos[b]) & 1) {
                G.reg_pos[nr] = (uint8_t)b;
                regidx_[st.tile_pos[b]] = nr;
                ++nr;
            } else {
                G.thr_pos[nt++] = (uint8_t)b;
            }
        }
        if (nr != R) return "internal: register group width mismatch";
        G.pairs = (eb_ == 8 && G.reg_pos[0] == 0) ? 1 : 0;
        for (int j = 0; j < R; ++j) G.sreg[j] = svk::swizzle(1u << G.reg_pos[j], eb_);
        for (int i = 0; i < nt; ++i) {
            G.sthr[i] = svk::swizzle(1u << G.thr_pos[i], eb_);
            G.pthr[i] = 1ull << st.tile_pos[G.thr_pos[i]];
        }
        for (uint32_t sid : groups.ids[gi]) {
            uint32_t gid = ids[sid];
            err = gate(P_.gates[gid], P_.phys[gid]);
            if (!err.empty()) return err;
        }
        if (s == (bwd_ ? 0 : (int)P_.top.local.size() - 1) && gi + 1 == groups.local.size())
            flush_all();
        grp_ = nullptr;
    }
    (void)tidx;
    st.n_slots = stage_slots_;
    slot_base_ += stage_slots_;
    out_->stages.push_back(st);
    return "";
}

std::string Lowerer::run() {
    out_->stages.clear();
    out_->groups.clear();
    out_->ops.clear();
    out_->terms.clear();
    out_->slot_param.clear();
    out_->groups.reserve(4096);
    const int S = (int)P_.top.local.size();
    // S == 0: an empty circuit, whose program has no stages (the identity)
    for (int k = 0; k < S; ++k) {
        int s = bwd_ ? S - 1 - k : k;
        std::string err = stage(s);
        if (!err.empty()) return err;
    }
    out_->identity_map = true;
    for (int q = 0; q < P_.n; ++q)
        if (P_.final_map[q] != q) out_->identity_map = false;
    out_->fused_perm = false;
    out_->dst.clear();
    if (fuse_perm_ && !out_->identity_map) {
        out_->fused_perm = true;
        out_->dst.assign(P_.n, 0);
        for (int q = 0; q < P_.n; ++q) out_->dst[P_.final_map[q]] = q;
    }
    return "";
}

}  // namespace

// radians -> device angle (turns for complex64, radians for complex128)
template <typename Real> static typename svk::AngT<Real>::type dev_angle(double rad);
template <> uint32_t dev_angle<float>(double rad) {
    double t = rad / (2.0 * M_PI);
    t -= std::floor(t);
    return (uint32_t)((uint64_t)std::llround(t * 4294967296.0) & 0xffffffffull);
}
template <> double dev_angle<double>(double rad) { return rad; }

template <typename Real>
static void pack_real(const Program& p, int n, Packed* out) {
    using DOp = svk::DevOp<Real>;
    using DTerm = svk::DevTerm<Real>;
    std::vector<svk::Stage> stages = p.stages;
    std::vector<svk::Group> groups = p.groups;
    std::vector<DOp> ops;
    std::vector<DTerm> terms;
    std::vector<svk::PhaseSlot<Real>> slots;
    ops.reserve(p.ops.size());
    for (auto& st : stages) {
        const uint32_t first_group = st.group_off;
        uint32_t first_op = first_group < groups.size() ? p.groups[first_group].op_off : (uint32_t)p.ops.size();
        uint32_t last_op = first_op;
        for (uint32_t gi = 0; gi < st.n_groups; ++gi) {
            const svk::Group& G0 = p.groups[first_group + gi];
            last_op = G0.op_off + G0.n_ops;
        }
        st.op_off = (uint32_t)ops.size();
        st.n_ops = last_op - first_op;
        st.phase_off = (uint32_t)slots.size();
        st.n_phase = 0;
        st.thr_off = 0;
        const int TR = (int)st.T - (int)st.R;
        uint64_t tile_mask = 0;
        for (uint32_t b = 0; b < st.T; ++b) tile_mask |= 1ull << st.tile_pos[b];
        for (uint32_t gi = 0; gi < st.n_groups; ++gi) {
            svk::Group& G = groups[first_group + gi];
            const svk::Group& G0 = p.groups[first_group + gi];
            G.op_off = G0.op_off - first_op;
            for (uint32_t oi = 0; oi < G0.n_ops; ++oi) {
                const svk::Op& o = p.ops[G0.op_off + oi];
                DOp d;
                std::memset(&d, 0, sizeof(d));
                d.type = o.type;
                d.j = o.j;
                d.u = o.u;
                d.ctrl_reg = o.ctrl_reg;
                d.ctrl_fix = o.ctrl_fix;
                d.slot = o.slot;
                for (int i = 0; i < 8; ++i) d.m[i] = (Real)o.m[i];
                if (o.has_pairs) {   // angles in the imaginary slots OP_UR ignores
                    d.flags |= svk::F_PAIRS;
                    for (int i = 0; i < 3; ++i) {
                        const typename svk::AngT<Real>::type a = dev_angle<Real>(o.pair_ang[i]);
                        static_assert(sizeof(a) == sizeof(Real), "angle slot size");
                        std::memcpy(&d.m[1 + 2 * i], &a, sizeof(a));
                    }
                }
                if (o.bparam1) {
                    d.flags |= svk::F_BIND;
                    d.term_off = o.bparam1 - 1;
                    d.u = o.bkind;
                }
                const bool dense_tw = o.type <= svk::OP_X && o.has_tw;
                const bool phase = ((o.type == svk::OP_PHASE0 || o.type == svk::OP_PHASE1) && o.n_terms > 0) || dense_tw;
                if (dense_tw) d.flags |= svk::F_TW;
                const double cang = dense_tw ? o.tw_angle : std::atan2(o.m[1], o.m[0]);
                if (phase) {
                    bool single = true;
                    for (uint32_t ti = 0; ti < o.n_terms; ++ti)
                        if (__builtin_popcountll(p.terms[o.term_off + ti].mask) != 1) single = false;
                    if (!single) {
                        d.flags |= svk::F_TERMS;
                        d.term_off = (uint32_t)terms.size();
                        d.n_terms = o.n_terms;
                        if (dense_tw) {   // the constant as an always-true (mask 0) term
                            DTerm t0;
                            t0.mask = 0;
                            t0.angle = dev_angle<Real>(o.tw_angle);
                            t0.pad = 0;
                            terms.push_back(t0);
                            d.n_terms++;
                        }
                        for (uint32_t ti = 0; ti < o.n_terms; ++ti) {
                            DTerm t;
                            t.mask = p.terms[o.term_off + ti].mask;
                            t.angle = dev_angle<Real>(p.terms[o.term_off + ti].angle);
                            t.pad = 0;
                            terms.push_back(t);
                        }
                    } else {
                        // split: global-bit terms per tile, thread-bit terms per thread
                        d.flags |= svk::F_SLOT;
                        d.slot = st.n_phase++;
                        svk::PhaseSlot<Real> ps;
                        std::memset(&ps, 0, sizeof(ps));
                        ps.cangle = dev_angle<Real>(cang);
                        ps.glob_off = (uint32_t)terms.size();
                        for (uint32_t ti = 0; ti < o.n_terms; ++ti) {
                            const svk::Term& t = p.terms[o.term_off + ti];
                            if (t.mask & tile_mask) {
                                for (int i = 0; i < TR; ++i)
                                    if (t.mask == G.pthr[i]) {
                                        ps.J[i] += dev_angle<Real>(t.angle);   // wraps mod 2 pi in turns
                                        ps.has_thr = 1;
                                    }
                            } else {
                                DTerm dt;
                                dt.mask = t.mask;
                                dt.angle = dev_angle<Real>(t.angle);
                                dt.pad = 0;
                                terms.push_back(dt);
                                ps.n_glob++;
                            }
                        }
                        slots.push_back(ps);
                    }
                }
                // flat dispatch code
                switch (o.type) {
                    case svk::OP_U: case svk::OP_UR: case svk::OP_X: {
                        const uint32_t ctrl = (o.ctrl_reg != 0) ? 1u : 0u;
                        d.code = svk::C_DENSE + ((uint32_t)o.type * 2 + ctrl) * 5 + o.j;
                        if (o.has_pairs) d.code = svk::C_URP + o.j;   // uncontrolled OP_UR only
                        break;
                    }
                    case svk::OP_PHASE1: d.code = svk::C_PHASE1 + o.j; break;
                    case svk::OP_PHASE2: d.code = svk::C_PHASE2 + svk::pair_index(o.j, o.u); break;
                    case svk::OP_PHASE0: d.code = svk::C_PHASE0; break;
                    case svk::OP_GRAD_X: d.code = svk::C_GRAD + 0 * 5 + o.j; break;
                    case svk::OP_GRAD_Y: d.code = svk::C_GRAD + 1 * 5 + o.j; break;
                    default: d.code = o.u ? svk::C_GRADZ_FIX : svk::C_GRAD + 2 * 5 + o.j; break;
                }
                if (d.code < svk::C_DENSE + 10) st.has_complex = 1;   // OP_U codes
                ops.push_back(d);
            }
        }
    }
    auto put = [&](const void* src, size_t bytes) -> size_t {
        size_t off = (out->blob.size() + 127) & ~(size_t)127;
        out->blob.resize(off + bytes + 16, 0);
        if (bytes) std::memcpy(out->blob.data() + off, src, bytes);
        return off;
    };
    out->blob.clear();
    out->stage_off = put(stages.data(), stages.size() * sizeof(svk::Stage));
    out->group_off = put(groups.data(), groups.size() * sizeof(svk::Group));
    out->op_off = put(ops.data(), ops.size() * sizeof(DOp));
    out->term_off = put(terms.data(), terms.size() * sizeof(DTerm));
    out->slot_off = put(slots.data(), slots.size() * sizeof(svk::PhaseSlot<Real>));
    out->wthr_off = out->slot_off;
    out->n_groups = groups.size();
    out->n_ops = ops.size();
    out->n_terms = terms.size();
    out->n_slots = slots.size();
    out->stages = stages;
}

std::string pack(const Program& p, int n, int elem_bytes, Packed* out) {
    if (elem_bytes == 8) pack_real<float>(p, n, out);
    else pack_real<double>(p, n, out);
    return "";
}

std::string lower(const Plan& plan, const double* params, int elem_bytes, int rmax, bool backward,
                  Program* out, bool bind, int rwide, bool fuse_perm) {
    if (plan.n_params > 0 && params == nullptr && !bind) return "circuit has parameters but params is NULL";
    if (fuse_perm && backward) return "internal: a fused output permutation needs a forward program";
    Lowerer L(plan, params, elem_bytes, rmax, backward, bind, out, rwide, fuse_perm);
    return L.run();
}

}  // namespace svh
