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
cudaError_t launch_permute(int elem_bytes, const void* in, void* out, const PermDesc* d_desc, int T,
                           uint64_t ntiles, cudaStream_t s);

// Pauli-sum sweep.  Terms act on the tile of the sweep; diagonal terms (xmask 0) are
// evaluated once, in sweep 0.
struct PauliTerm {
    uint64_t zmask;        // physical bits carrying Z or Y
    uint64_t xmask;        // physical bits carrying X or Y
    uint32_t xtile;        // xmask as a tile-element mask
    uint32_t zreg;         // zmask restricted to the register bits (tile bits 0..R-1) as a k mask
    double fre, fim;       // coeff * i^{#Y}
};
struct PauliSweep {
    uint32_t T, n_glob, n_terms, term_off;
    uint8_t glob_pos[kMaxQ];
    uint8_t tile_pos[16];
    uint64_t ptile[16];
    uint32_t swbit[16];
};
// lam == nullptr: expectation value only.  accumulate: lam += O_sweep psi, else lam =.
// partial[blockIdx] = sum over the tile of Re(conj(psi) * (O_sweep psi)).
cudaError_t launch_pauli(int elem_bytes, int R, const void* psi, void* lam, bool accumulate,
                         const PauliSweep* d_sweep, const PauliTerm* d_terms, double* partial, int T,
                         uint64_t ntiles, cudaStream_t s);

// sum |psi|^2 per block into partial[]; returns the number of blocks used.
cudaError_t launch_norm(int elem_bytes, const void* psi, uint64_t n_amp, double* partial,
                        uint32_t* nblocks, cudaStream_t s);
// out[r] = sum_{i < n} in[i * stride + r] for r < rows, fixed order (one block per row).
cudaError_t launch_reduce_rows(const double* in, uint64_t n, uint32_t rows, double* out,
                               cudaStream_t s);
// state set to |0...0>
cudaError_t launch_zero_state(int elem_bytes, void* psi, uint64_t n_amp, cudaStream_t s);

struct GemmStage;
size_t gemm_smem_bytes(const GemmStage& st);
// prec 1 = TF32x3, 2 = BF16x3; d_status receives 1 if a bounded wait gave up
cudaError_t launch_gemm_stage(int prec, void* psi, const GemmStage* d_stage, const GemmStage& hst,
                              const uint8_t* d_ablob, int* d_status, cudaStream_t s);

// batched circuits (batch.h): one persistent launch of `grid` CTAs
struct BatchArgs;
cudaError_t launch_batch(const BatchArgs& a, int grid, cudaStream_t s);
// CTAs of the batch kernel that fit on one SM with `smem` bytes of dynamic shared memory
cudaError_t batch_occupancy(size_t smem, int* per_sm);
int batch_threads();

}  // namespace svk
