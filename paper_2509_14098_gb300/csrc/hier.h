// hier.h — the hierarchical tensor-core stage (Sec. 4.2: the partitioner invoked again
// inside each partition for the next memory level; Sec. 5.2: fusion at several levels).
//
// The circuit is partitioned (without exemptions) into stages of T = k + 7 local qubits,
// the tile of one CTA in shared memory; each stage's gates are partitioned again with
// budget k into sub-partitions, each a fused 2^k x 2^k unitary.  A CTA loads a tile from
// HBM once, applies every sub-partition of the stage to it as a split-precision GEMM on
// the tensor cores (the tile's 2^T amplitudes viewed as 128 columns of 2^k amplitudes
// over the sub-partition's qubits), and writes the tile back once: one HBM pass per
// stage instead of one per fused unitary.
#pragma once
#include <stdint.h>

#include <complex>
#include <string>
#include <vector>

#include "program.h"

namespace svk {

constexpr int kHierMaxSub = 24;   // sub-partitions one launch applies (longer stages: more launches)

// Operand layouts.  Layout s < n_sub is sub-partition s's A operand: per K chunk c (128
// bytes per row: 32 BF16 / 16 TF32 amplitudes) a hi block of 128 rows x 128 bytes at
// c * 32768 and the lo block 16384 bytes above it, rows 128-byte swizzled (K-major).
// Element (row m, amplitude j) lies at an offset XOR-linear in the tile bits of its
// amplitude; ao[s][b] is tile bit b's term.  Layout n_sub is the FP32 output tile
// (element x at 8 (x ^ (((x >> 4) ^ (x >> 8)) & 14)), pairs 2i, 2i + 1 adjacent).
struct HierStage {
    uint32_t T;             // tile qubits, k + 7
    uint32_t k;             // sub-partition width (5 or 6)
    uint32_t N;             // 2^(k+1): output floats per column
    uint32_t nchunk;        // K chunks per column
    uint32_t n_sub;         // sub-partitions of this launch
    uint32_t n_glob;        // tile-index bits
    uint32_t b_bytes;       // B operand of one sub-partition: nchunk x (hi, lo) blocks of N x 128 bytes
    uint32_t a_bytes;       // A operand region (nchunk x 32768), also holds the FP32 output tile
    uint32_t b_slots;       // B operand buffers in shared memory (1 or 2)
    uint32_t reserved;
    uint64_t b_off;         // byte offset of sub-partition 0's B operand in the blob
    uint8_t tile_pos[16];   // physical position of tile bit b, ascending (bits 0..3 first)
    uint8_t ld_bits[16];    // load / store: bit i of a thread's 16-byte pair index (thread bits 0..6,
                            // then round bits) is tile bit ld_bits[i] (tile bits 1..3 first)
    uint8_t glob_pos[kMaxQ];
    uint8_t amp_bits[kHierMaxSub][8];   // sub-partition s: tile bit of amplitude-index bit i
    uint8_t col_bits[kHierMaxSub][8];   // tile bit of row bit i (7 bits)
    uint32_t ao[kHierMaxSub + 1][16];   // byte-offset term of tile bit b in layout s
};

}  // namespace svk

namespace svh {
struct Plan;
struct HierProgram {
    std::vector<svk::HierStage> launches;   // one per run of at most kHierMaxSub sub-partitions
    std::vector<uint8_t> ublob;              // B operands (1024-byte aligned per launch)
    uint32_t n_sub = 0;                      // sub-partitions in all
    bool identity_map = true;
};
// prec: 1 = TF32x3, 2 = BF16x3.  The plan must come from a strict partition with
// L = k + 7 and qubits 0..3 fixed.  Returns "" or an error.
std::string plan_hier(const Plan& plan, const double* params, int prec, HierProgram* out);
// shared-memory bytes of a launch (dynamic part)
size_t hier_smem_bytes(const svk::HierStage& st);
}  // namespace svh
