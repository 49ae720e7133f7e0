// gemm.h — split-precision tensor-core stage (fused dense unitaries as GEMMs).
#pragma once
#include <stdint.h>

#include <complex>

#include <string>
#include <vector>

#include "program.h"

namespace svk {

// One fused stage applied as D = X * Ut^T per tile:
//   X  (the MMA's A operand, M = 128): 128 state columns of the tile, one per row; a
//      column is the 2^keff amplitudes whose local bits vary, i.e. K = 2^(keff+1)
//      interleaved (re, im) floats;
//   Ut (the B operand, N = 2^(keff+1) rows): the real embedding of the stage's fused
//      unitary, row n = output float n of a column;
//   D  (M x N FP32 in tensor memory): the updated columns.
// A tile fixes the global bits; its columns are indexed by the 7 column bits (the
// lowest non-local bits).  K is processed in chunks of 128 bytes per row (32 TF32 or
// 64 BF16 elements = 2^camp_bits amplitudes): chunk c fixes the local bits above
// camp_bits to c.  Both operands use the 128-byte-swizzled K-major layout (rows of
// 128 bytes, 8-row groups of 1024 bytes, 16-byte units XORed with the row index).
struct GemmStage {
    uint32_t keff;          // local qubits (6 or 7)
    uint32_t N;             // 2^(keff+1)
    uint32_t nchunk;        // K chunks
    uint32_t camp_bits;     // log2 amplitudes per K chunk (4 TF32, 5 BF16)
    uint32_t n_glob;        // tile-index bits
    uint32_t resident;      // 1: every B chunk stays in shared memory for the whole launch
    uint32_t b_chunk_bytes; // one B chunk: hi block then lo block (N x 128 bytes each)
    uint32_t nvar;          // camp_bits + ncol_bits chunk-varying bits
    uint32_t ncol_bits;     // log2 columns per tile: 7, fewer only for states with n < keff + 7
                            // (the MMA rows beyond the columns are zero and never stored)
    uint32_t nslot;         // operand ring depth (A slots, with their B chunks when streamed)
    uint64_t b_off;         // byte offset of this stage's B chunks in the blob
    uint8_t glob_pos[kMaxQ];
    uint8_t local_pos[8];   // physical positions of the local bits, ascending
    uint8_t col_pos[8];     // physical positions of the column bits, ascending
    uint8_t var_role[12];   // chunk-varying bits in ascending physical order: 0..4 = bit of
                            // the amplitude index inside the chunk, 8 + c = column bit c
    uint8_t var_pos[12];    // their physical positions
    uint8_t pperm[12];      // producer bit i (thread bits 0..8, then round bits) -> chunk-varying bit
                            // 1..nvar-1 (bit 0 is the 16-byte pair); the lane bits are chosen so a
                            // warp's operand stores fall on distinct shared-memory banks
};

}  // namespace svk

namespace svh {
struct Plan;
struct GemmProgram {
    std::vector<svk::GemmStage> stages;
    std::vector<uint8_t> ublob;   // B chunks of every stage (1024-byte aligned)
    bool identity_map = true;
};
// prec: 1 = TF32x3, 2 = BF16x3.  Returns "" or an error.
std::string plan_gemm(const Plan& plan, const double* params, int prec, GemmProgram* out);

// The fused unitary of the gates ids (plan gate indices, in order) over the physical
// bits lp[0..k-1] (index bit j <-> lp[j]), formed in FP64, column-major
// (U[col * 2^k + row]).  Returns "" or an error (a gate outside those bits).
std::string fuse_unitary(const Plan& P, const std::vector<uint32_t>& ids, const int* lp, int k, const double* params,
                         std::vector<std::complex<double>>* U);
// The B operand of U: its real embedding (N = 2^(k+1) rows), split into rounded hi / lo
// halves, per K chunk of 128 bytes per row (32 TF32 / 64 BF16 elements) one hi block of
// N x 128 bytes then one lo block, 128-byte-swizzled K-major; (2^(k+1) / chunk elements)
// x 2 N x 128 bytes written at dst.
void emit_b(const std::vector<std::complex<double>>& U, int k, bool tf32, uint8_t* dst);
}  // namespace svh
