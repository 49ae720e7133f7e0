// planner.h — host-side partitioner and program lowering (internal).
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "program.h"

namespace svh {

enum Kind {
    K_H = 1, K_X, K_Y, K_Z, K_S, K_SDG, K_T, K_TDG, K_RX, K_RY, K_RZ, K_P, K_U3, K_CX,
    K_CY, K_CZ, K_CP, K_SWAP, K_LAST = K_SWAP
};

inline bool kind_is_diagonal(int k) {
    return k == K_Z || k == K_S || k == K_SDG || k == K_T || k == K_TDG || k == K_RZ || k == K_P ||
           k == K_CZ || k == K_CP;
}
inline bool kind_is_controlled(int k) { return k == K_CX || k == K_CY; }
inline int kind_nq(int k) { return (k >= K_CX) ? 2 : 1; }

struct GateRec {
    int kind;
    int nq;
    int q[2];       // circuit qubits (wires)
    int param;      // -1 = fixed angles
    double angle[3];
};

// A gate as the partitioner sees it: physical bit positions after SWAP relabels.
struct PGate {
    int kind;
    int nq;
    int p[2];
    bool bound = false;   // parametric RZ lowered as a dense op (bind mode): needs its qubit
};

struct Partition {
    std::vector<uint64_t> local;                 // physical-bit mask per stage
    std::vector<std::vector<uint32_t>> ids;      // indices into the gate list, execution order
};

struct Centrality {
    std::vector<uint32_t> reach;   // |RN(v)|
    std::vector<uint64_t> dist;    // sum over RN(v) of (l_x - l_v)
    std::vector<uint32_t> level;   // critical-path length l_v
};

// Closeness-centrality partitioner (Sec. 4.1-4.2) over gates given in physical bits.
// L: local-bit budget; fixed: bits local in every partition; universe: bits that may
// be used to fill a partition's local set up to min(L, |universe|) after the cut.
// Returns "" on success or an error message (status SV_ERR_PARTITION).
// strict: no exemptions (every qubit of a gate must be local; SWAP stays a relabel).
std::string partition_core(int nbits, const std::vector<PGate>& gates, int L, uint64_t fixed,
                           uint64_t universe, Partition* out, Centrality* cc, bool strict = false);

// Physical positions of every gate after replaying the SWAP relabels in circuit
// order, and the final map wire -> physical bit.
void relabel(int n, const std::vector<GateRec>& gates, std::vector<PGate>* phys,
             std::vector<int>* final_map);

struct Plan {
    int n = 0;
    int n_params = 0;
    int L = 0;
    int n_fixed = 0;
    int gemm_k = 0;             // > 0: partitioned without exemptions for tensor-core stages
    int hier_k = 0;             // > 0: hierarchical tensor-core stages (tiles of hier_k + 7 qubits)
    std::vector<GateRec> gates;
    std::vector<PGate> phys;
    std::vector<int> final_map;
    Partition top;
    Centrality cc;
};

// Lowered program of one direction, ready to upload.
struct Program {
    std::vector<svk::Stage> stages;
    std::vector<svk::Group> groups;
    std::vector<svk::Op> ops;
    std::vector<svk::Term> terms;
    std::vector<int> slot_param;   // backward: global gradient slot -> parameter
    bool identity_map = true;
    // fuse_perm: the last stage writes out of place through the final map;
    // dst[physical bit] = the qubit it becomes
    bool fused_perm = false;
    std::vector<int> dst;
};

// Device blob of a lowered program for one precision: Stage[] | Group[] |
// DevOp<Real>[] | DevTerm<Real>[] | PhaseSlot[] | wthr (complex Real) at the offsets.
struct Packed {
    std::vector<uint8_t> blob;
    size_t stage_off = 0, group_off = 0, op_off = 0, term_off = 0, slot_off = 0, wthr_off = 0;
    size_t n_groups = 0, n_ops = 0, n_terms = 0, n_slots = 0;   // element counts of the sections
    std::vector<svk::Stage> stages;   // with op/phase offsets filled in
};
std::string pack(const Program& p, int n, int elem_bytes, Packed* out);

// Lower a plan with bound parameters.  rmax: register bits per thread.
// backward: un-apply the stages in reverse (conjugate-transposed gates) and emit
// gradient ops for parametric RX / RY / RZ gates.  Returns "" or an error.
// bind: parametric RX / RY / RZ become dense ops flagged F_BIND (no twiddle fused, RZ
// kept on a register bit, which the plan's partition must guarantee via
// PGate::bound), so the program's structure does not depend on the parameters;
// params may then be NULL (the kernel forms those matrices).  Parametric P / CP are
// rejected in this mode.
// rwide > rmax: a stage that needs 4 or more register groups at rmax is lowered with
// rwide register bits instead when that needs fewer groups (0: never).
// fuse_perm (forward only): when the final map is not the identity, the last stage's
// tile trades its untouched fill bits for the bits that become the lowest qubits, and
// the program is marked for an out-of-place write-back through the map (Program::dst).
std::string lower(const Plan& plan, const double* params, int elem_bytes, int rmax, bool backward,
                  Program* out, bool bind = false, int rwide = 0, bool fuse_perm = false);

}  // namespace svh
