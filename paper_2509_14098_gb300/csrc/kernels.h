// kernels.h — host-callable launchers of the CUDA kernels (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "program.h"

namespace svk {

// Device pointers of one stage launch (blob sections + state buffers).
struct StageLaunch {
    void* psi;
    void* lam;                 // backward only
    const Stage* stage;        // this stage's descriptor (device)
    const Group* groups;
    const void* ops;           // DevOp<Real>[]
    const void* terms;         // DevTerm<Real>[]
    const void* slots;         // PhaseSlot<Real>[]
    double* partial;           // backward: per-tile gradient partials
};
// hst: host copy of the same stage (launch geometry).
cudaError_t launch_stage_fwd(int elem_bytes, const StageLaunch& L, const Stage& hst, cudaStream_t s);
// grid_out: CTAs launched (rows of per-CTA gradient partials written to L.partial)
cudaError_t launch_stage_bwd(int elem_bytes, const StageLaunch& L, const Stage& hst, cudaStream_t s,
                             uint32_t* grid_out);
size_t stage_smem_bytes(int elem_bytes, const Stage& st, bool backward);

// Bit-permutation sweep descriptor: out[pi(x)] = in[x], pi moves physical bit p to dst[p].
struct PermDesc {
    uint32_t T, n_glob;
    uint8_t glob_pos[kMaxQ];      // input global bits
    uint8_t tile_pos[16];         // input tile bits (ascending)
    uint64_t ptile[16];           // 1 << tile_pos[b]
    uint32_t swbit[16];           // swizzled element offset of tile bit b
    uint64_t gout[kMaxQ];         // output value of input global bit i (1 << dst[glob_pos[i]])
    uint64_t pout[16];            // output value of output-tile bit c (ascending output positions)
    uint32_t sig[16];             // swizzled input element offset of output-tile bit c
};
// d is passed by value (kernel parameter space); ntiles = 2^(n - d.T)
cudaError_t launch_permute(int elem_bytes, const void* in, void* out, const PermDesc& d, uint64_t ntiles,
                           cudaStream_t s);

// Pauli-sum sweep.  A tile fixes the global bits; its T bits are laid out as
//   tile bits [0, L)       the L lowest physical bits    (thread bits 0..L-1)
//   tile bits [L, L + R)   register bits                 (element k of a thread)
//   tile bits [L + R, T)   the remaining tile bits       (thread bits L..)
// so a thread holds 2^R elements and, for each of them, the lanes of a warp cover
// 2^L-amplitude runs of consecutive addresses.  Terms act on the tile of their sweep;
// diagonal terms (no X / Y) are evaluated once, in sweep 0, ordered: Z on tile bits
// only (n_dstat, folded into a per-thread table once per CTA), Z on global bits only
// (n_dglob, one constant per tile), Z on both (n_dmix); then the X / Y terms.
struct PauliSweep {
    uint32_t T, R, L, n_glob;
    uint32_t n_terms, term_off, n_dstat, n_dglob;
    uint32_t n_dmix, pad0, pad1, pad2;
    uint64_t ptile[16];           // physical value of tile bit b
    uint8_t glob_pos[kMaxQ];      // physical positions of the global bits (ascending)
};
enum : uint32_t {
    PT_SMEM = 1,    // partner outside the thread's registers: read from the staged tile
    PT_FLUSH = 2,   // diagonal: last term of a run with the same zreg
    PT_REAL = 4,    // fim == 0
    PT_NOZ = 8,     // no Z / Y outside the register bits: no per-thread sign
};
struct PauliTerm {         // 48 bytes, read as three 16-byte words
    uint64_t zmask;        // physical bits carrying Z or Y
    uint32_t xtile;        // bits carrying X or Y as a tile-index mask (0: diagonal)
    uint32_t flags;        // PT_*
    uint16_t xreg;         // X / Y register bits, as a mask of the element index k
    uint16_t zreg;         // Z / Y register bits, as a mask of k
    uint32_t smask;        // bit k: parity of (k & zreg)
    float fre32, fim32;    // the coefficient rounded to FP32 (complex64 sweeps)
    double fre, fim;       // coeff * i^{#Y} * (-1)^{|xmask & zmask|}
};
// lam == nullptr: expectation value only.  accumulate: lam += O_sweep psi, else lam =.
// Persistent: *grid_out CTAs each walk a fixed set of tiles and write one partial
// partial[cta] = sum over its tiles of Re(conj(psi) * (O_sweep psi)).
cudaError_t launch_pauli(int elem_bytes, const void* psi, void* lam, bool accumulate,
                         const PauliSweep& hsw, const PauliSweep* d_sweep, const PauliTerm* d_terms,
                         double* partial, uint64_t ntiles, uint32_t* grid_out, cudaStream_t s);
// CTAs launch_pauli uses for a sweep (the rows of partials it writes); 0 on error
uint32_t pauli_grid(int elem_bytes, const PauliSweep& sw, uint64_t ntiles);

// sum |psi|^2 per block into partial[]; returns the number of blocks used.
cudaError_t launch_norm(int elem_bytes, const void* psi, uint64_t n_amp, double* partial,
                        uint32_t* nblocks, cudaStream_t s);
// out[r] = sum_{i < n} in[i * stride + r] for r < rows, fixed order (one block per row).
cudaError_t launch_reduce_rows(const double* in, uint64_t n, uint32_t rows, double* out,
                               cudaStream_t s);
// psi *= sqrt(*norm_before / *norm_after) (device doubles; unchanged if either is 0)
cudaError_t launch_scale_to_norm(int elem_bytes, void* psi, uint64_t n_amp, const double* norm_before,
                                 const double* norm_after, cudaStream_t s);
// state set to |0...0>
cudaError_t launch_zero_state(int elem_bytes, void* psi, uint64_t n_amp, cudaStream_t s);

struct GemmStage;
size_t gemm_smem_bytes(const GemmStage& st);
// prec 1 = TF32x3, 2 = BF16x3; d_status receives 1 if a bounded wait gave up
cudaError_t launch_gemm_stage(int prec, void* psi, const GemmStage* d_stage, const GemmStage& hst,
                              const uint8_t* d_ablob, int* d_status, cudaStream_t s);

// hierarchical tensor-core stage (hier.h): prec 1 = TF32x3 (k = 5), 2 = BF16x3 (k = 5, 6);
// d_status receives 1 if a bounded wait gave up
struct HierStage;
cudaError_t launch_hier_stage(int prec, void* psi, const HierStage* d_st, const HierStage& hst, const uint8_t* d_ublob,
                              int* d_status, cudaStream_t s);

// batched circuits (batch.h): one persistent launch of `grid` CTAs
struct BatchArgs;
cudaError_t launch_batch(const BatchArgs& a, int grid, cudaStream_t s);
// CTAs of the batch kernel that fit on one SM with `smem` bytes of dynamic shared memory
cudaError_t batch_occupancy(size_t smem, int* per_sm);
int batch_threads();
// wide circuits of a batch (batch_kernels.cu): lambda = h psi with E partials; gradient
// slot sums over tiles; per-circuit E and gradient gather
struct ObsTerm;
cudaError_t launch_bgs_obs(const void* psi, void* lam, int n, uint32_t ncirc, const ObsTerm* obs,
                           const uint32_t* obs_off, double* epart, uint32_t nblk, cudaStream_t s);
cudaError_t launch_bgs_slotsum(const double* partial, uint32_t ncirc, uint32_t ntiles, uint32_t nsl, uint32_t slot_off,
                               uint32_t nst, double* slotsum, cudaStream_t s);
cudaError_t launch_bgs_finish(const double* epart, uint32_t nblk, const double* slotsum, uint32_t nst,
                              const uint32_t* pidx, const uint32_t* plist, uint32_t np, const uint32_t* pofs,
                              const uint32_t* outidx, uint32_t ncirc, double* expval, double* grad, cudaStream_t s);

}  // namespace svk
