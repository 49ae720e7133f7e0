// program.h — device program format shared by the host planner and the kernels.
//
// A plan is lowered into a flat program per direction (forward / backward):
//   Stage[]  one per partition (one HBM sweep each): tile geometry
//   Group[]  register groups inside a stage (the partitioner re-run with the
//            register budget, i.e. the paper's next memory level, Sec. 4.2)
//   Op[]     micro-ops applied to the amplitudes a thread holds in registers
//   Term[]   phase terms that depend on bits outside the registers
//
// Index spaces
//   physical bit  p in [0, n): bit of the amplitude index in HBM
//   tile bit      b in [0, T): position inside a shared-memory tile; tile bit b
//                 is physical bit tile_pos[b] (ascending)
//   register bit  j in [0, R): bit of the per-thread register index k; register
//                 bit j is tile bit reg_pos[j] (ascending)
//   thread bit    i in [0, T-R): bit of threadIdx.x; tile bit thr_pos[i]
// A thread's "fixed index" is the physical index of its amplitudes with every
// register bit zero (tile base | thread bits); phase terms and controls on
// non-register bits are evaluated on it.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define SVK_HD __host__ __device__ __forceinline__
#else
#define SVK_HD inline
#endif

namespace svk {

constexpr int kMaxT = 14;      // widest tile (2^14 amplitudes)
constexpr int kMaxR = 5;       // widest register group (32 amplitudes per thread)
constexpr int kMaxQ = 40;      // widest state the planner accepts

enum OpType : uint8_t {
    OP_U = 0,       // dense complex 2x2 on register bit j (optionally controlled)
    OP_UR = 1,      // dense real 2x2 on register bit j
    OP_X = 2,       // swap the pair on register bit j (X / CX target)
    OP_PHASE0 = 3,  // every amplitude *= c * exp(i * sum of terms on the fixed index)
    OP_PHASE1 = 4,  // amplitudes with register bit j set *= c * exp(i * sum of terms)
    OP_PHASE2 = 5,  // amplitudes with register bits j and u set *= c
    OP_GRAD_X = 6,  // gradient slot += Im <lam| X_j |psi>  (backward only)
    OP_GRAD_Y = 7,  // gradient slot += Im <lam| Y_j |psi>
    OP_GRAD_Z = 8,  // gradient slot += Im <lam| Z_b |psi>, b register bit j (u=0) or
                    // the physical bit in ctrl_fix (u=1)
};

// Host-side op produced by the lowering (FP64 matrix, generic phase terms).
struct Op {
    uint8_t type;
    uint8_t j;              // register bit (target)
    uint8_t u;              // second register bit (PHASE2) / flag (GRAD_Z)
    uint8_t has_tw;         // dense op: phase exp(i (tw_angle + terms)) on the bit-j amplitude first
    uint32_t ctrl_reg;      // controls on register bits (mask over k)
    uint64_t ctrl_fix;      // controls on non-register bits (mask over the fixed index)
    uint32_t term_off;      // first Term of this op
    uint32_t n_terms;
    uint32_t slot;          // gradient slot (GRAD ops): index into the stage's slot list
    uint32_t bparam1;       // bound dense op: parameter index + 1 (0 = matrix fixed at lowering)
    double m[8];            // row-major 2x2 (re, im) pairs; PHASE ops use m[0], m[1]
    double tw_angle;        // dense op twiddle constant (has_tw)
    uint8_t bkind;          // bound dense op: BK_RX / BK_RY / BK_RZ, | BK_DAGGER for the adjoint
    uint8_t has_pairs;      // real dense op: pair phases folded in (pair_ang)
    double pair_ang[3];     // phase on the target's |1> half when the i-th other register bit
                            // (ascending, skipping j) is set; 0 for bits without a phase
};

struct Term {               // phase angle added when every bit of mask is set
    uint64_t mask;
    double angle;
};

enum OpFlag : uint8_t {
    F_SLOT = 1,             // PHASE op whose angle comes from phase slot `slot`
    F_TERMS = 2,            // PHASE op evaluated from its DevTerm list on the fixed index
    F_TW = 4,               // dense op preceded by a phase on its target bit (F_SLOT / F_TERMS
                            // give the angle; a dense op's constant is a mask-0 term)
    F_BIND = 8,             // dense op whose matrix the kernel forms from a parameter:
                            // term_off = parameter index, u = BK_* kind (| BK_DAGGER)
    F_PAIRS = 32,           // real dense op (OP_UR) preceded by phases on its target's |1> half
                            // that depend on the other register bits: the angles (device angle
                            // type) sit in m[1], m[3], m[5], the imaginary slots OP_UR ignores
};

// Parametric rotations whose matrix is formed on the device (batched programs are
// lowered once and replayed with new parameters).
enum BindKind : uint8_t { BK_RX = 1, BK_RY = 2, BK_RZ = 3, BK_DAGGER = 4 };

// Device op: 64 bytes (complex64 kernels) / 96 bytes (complex128 kernels).  The
// kernels stage a stage's ops in shared memory once per CTA.
template <typename Real>
struct alignas(16) DevOp {
    uint8_t type;
    uint8_t j;
    uint8_t u;
    uint8_t flags;
    uint32_t ctrl_reg;
    uint64_t ctrl_fix;
    uint32_t slot;          // phase slot (F_SLOT) or gradient slot (GRAD ops)
    uint32_t term_off;      // F_TERMS: DevTerm range
    uint32_t n_terms;
    uint32_t code;          // flat dispatch code (op_code())
    Real m[8];
};

// Flat dispatch codes: one switch selects the op kind, its control form and its
// compile-time register bit(s).
enum : uint32_t {
    C_DENSE = 0,            // + ((type * 2 + controlled) * 5 + j), type in {U, UR, X}: 0..29
    C_PHASE1 = 30,          // + j
    C_PHASE2 = 35,          // + pair index of (j < u): 0..9
    C_PHASE0 = 45,
    C_GRAD = 46,            // + (kind * 5 + j), kind 0 = X, 1 = Y, 2 = Z on a register bit
    C_GRADZ_FIX = 61,       // Z on a non-register bit
    C_URP = 62,             // + j: real dense op with folded pair phases (F_PAIRS, uncontrolled)
};
SVK_HD uint32_t pair_index(int j, int u) {   // j < u < 5: (0,1..4) -> 0..3, (1,2..4) -> 4..6, (2,3..4) -> 7..8, (3,4) -> 9
    return (uint32_t)(j == 0 ? u - 1 : j == 1 ? u + 2 : j == 2 ? u + 4 : 9);
}

// Phase angles on the device: complex64 kernels use 32-bit fixed-point turns
// (angle = 2 pi k / 2^32), whose sums are exact modulo 2 pi (the QFT's dyadic angles
// are represented exactly); complex128 kernels use FP64 radians.
template <typename Real> struct AngT;
template <> struct AngT<float> { using type = uint32_t; };
template <> struct AngT<double> { using type = double; };

template <typename Real>
struct DevTerm {
    uint64_t mask;
    typename AngT<Real>::type angle;
    Real pad;
};

// Phase slot of a PHASE op whose terms are all single bits: the angle is
// cangle + sum of global-bit terms (evaluated once per tile) + sum over the thread
// bits i of the op's group of J[i] * bit i of threadIdx.x.
template <typename Real>
struct alignas(16) PhaseSlot {
    typename AngT<Real>::type cangle;
    uint32_t glob_off, n_glob;   // DevTerm range (single global bits)
    uint32_t has_thr;            // any J[i] != 0
    typename AngT<Real>::type J[kMaxT];
};

struct alignas(16) Group {
    uint32_t op_off, n_ops;       // relative to the stage's first op
    uint8_t reg_pos[kMaxR];
    uint8_t thr_pos[kMaxT];
    uint8_t pairs;          // tile bit 0 is register bit 0: load amplitude pairs as 16 B
    uint8_t pad[4];
    uint32_t sreg[kMaxR];   // swizzled shared-memory element offset of each register bit
    uint32_t sthr[kMaxT];   // swizzled shared-memory element offset of each thread bit
    uint64_t pthr[kMaxT];   // physical index value of each thread bit (1 << phys)
};

struct Stage {
    uint32_t T, R;          // tile bits, register bits
    uint32_t n_glob;        // n - T
    uint32_t group_off, n_groups;
    uint32_t n_slots;       // gradient slots of this stage (backward)
    uint32_t slot_off;      // first global slot
    uint32_t op_off, n_ops; // this stage's ops (groups index relative to op_off)
    uint32_t phase_off, n_phase;  // phase slots of this stage
    uint32_t thr_off;       // unused
    uint32_t has_complex;   // any complex dense op (OP_U) in this stage
    uint8_t glob_pos[kMaxQ];  // physical positions of the global bits (ascending)
    uint8_t tile_pos[kMaxT];  // physical positions of the tile bits (ascending)
    uint8_t pad2[2];
    uint64_t ptile[kMaxT];    // 1 << tile_pos[b]
    uint32_t swbit[kMaxT];    // swizzled element offset of tile bit b
};

// Shared-memory swizzle (element index inside a tile -> storage index).  XOR-linear,
// so sw(a ^ b) = sw(a) ^ sw(b).  complex64 (8 B): XOR bits 1..4 with a fold of the
// bits above 5 (bit 0 untouched so 16-byte chunks stay whole); complex128 (16 B):
// XOR bits 0..2 with a fold of the bits above 3.  Spreads strided lanes over banks.
SVK_HD uint32_t swizzle8(uint32_t t) {
    uint32_t y = t >> 5;
    uint32_t f = (y ^ (y >> 5)) & 15u;
    return t ^ (f << 1);
}
SVK_HD uint32_t swizzle16(uint32_t t) {
    uint32_t y = t >> 3;
    uint32_t f = (y ^ (y >> 3) ^ (y >> 6) ^ (y >> 9)) & 7u;
    return t ^ f;
}
SVK_HD uint32_t swizzle(uint32_t t, int elem_bytes) {
    return elem_bytes == 8 ? swizzle8(t) : swizzle16(t);
}

}  // namespace svk
