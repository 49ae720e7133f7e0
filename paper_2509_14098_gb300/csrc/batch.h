// batch.h — batched execution of many small circuits in one persistent launch
// (device format shared by the host builder and the kernel; internal).
//
// Each distinct circuit structure (qubit count, gate list, fixed angles, parameter
// slots) is partitioned and lowered once, in bind mode: its parametric RX / RY / RZ
// gates are dense ops whose matrices the kernel forms from the circuit's own
// parameters when it stages the ops in shared memory.  Circuits therefore share
// programs and a replay needs nothing but the new parameters.
//
// One CTA runs one circuit start to finish (forward stages, <O> and lambda = O psi
// for a diagonal observable O, adjoint stages with gradient ops), taking circuits from
// a queue ordered largest first.  A circuit whose tile covers all its qubits lives
// in shared memory for its whole run (psi and lambda, no HBM traffic); larger ones
// sweep their tiles through a per-circuit HBM workspace.  The last forward stage, the
// observable and the first adjoint stage are fused into one tile visit (they share
// the tile bits), the first forward stage starts from |0...0> without a load and
// the last adjoint stage stores nothing.
#pragma once
#include <stdint.h>

#include "program.h"

namespace svk {

struct BatchProg {
    uint32_t n, Rf, Rb, pad;
    uint32_t f_stage, n_f, b_stage, n_b;      // into the Stage array
    uint32_t f_group, f_op, f_term, f_slot;   // bases of the forward program's arrays
    uint32_t b_group, b_op, b_term, b_slot;   // bases of the adjoint program's arrays
    uint32_t slot_param;                       // adjoint: base of the slot -> parameter table
    uint32_t pad2[3];
};

struct BatchCirc {
    uint32_t prog;        // BatchProg index
    uint32_t param_off;   // first parameter (and gradient entry) of this circuit
    uint32_t obs_off, n_obs;
    uint32_t out;         // expectation-value index (the caller's circuit index)
    uint32_t pad;
    uint64_t ws;          // amplitude offset of psi in the workspace; lambda follows at ws + 2^n
};

struct ObsTerm {          // coeff * prod_{b in zmask} Z_b   (physical bits)
    uint64_t zmask;
    double coeff;
};

// Shared-memory layout of one launch (byte offsets; the host sizes every region
// for the largest stage of the batch).
struct BatchSmem {
    uint32_t tiles;                            // tile region bytes (at offset 0)
    uint32_t st[2];                            // Stage copies (forward, adjoint)
    uint32_t grp[2], ops[2], slots[2], ang[2]; // staged stage programs (forward, adjoint)
    uint32_t gsm, gacc, red;                   // gradient partials, FP64 slot sums, reduction
    uint32_t total;
    uint32_t max_slots;                        // gradient slots of the largest adjoint stage
};

struct BatchArgs {
    const BatchCirc* circs;
    uint32_t n_circ;
    uint32_t pad;
    const BatchProg* progs;
    const Stage* stages;
    const Group* groups;
    const DevOp<float>* ops;
    const DevTerm<float>* terms;
    const PhaseSlot<float>* slots;
    const int32_t* slot_param;
    const ObsTerm* obs;
    const double* params;
    void* ws;              // complex64 workspace
    double* expval;
    double* grad;          // same layout as params; zeroed before the launch
    uint32_t* queue;       // next circuit (zeroed before the launch)
    BatchSmem sm;
};

}  // namespace svk
