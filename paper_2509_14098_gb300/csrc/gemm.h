// gemm.h — split-precision tensor-core stage (fused dense unitaries as GEMMs).
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "program.h"

namespace svk {

// One fused stage.  A tile = 2^ncol_bits columns (fixed global bits); a column = the
// 2^keff amplitudes whose local bits vary, i.e. 2^(keff+1) interleaved floats (the K
// dimension).  K is streamed in chunks of 32 floats = 16 amplitudes: chunk c fixes
// the local bits 4..keff-1 to c; inside a chunk the 4 lowest local bits and the column
// bits vary ("var" bits, ascending physical position).
struct GemmStage {
    uint32_t keff;          // local qubits (6 or 7)
    uint32_t nacc;          // 128-row accumulators = 2^(keff+1) / 128
    uint32_t nchunk;        // K chunks = 2^(keff+1) / 32
    uint32_t ncol_bits;     // log2(columns per tile), 4..7
    uint32_t n_glob;        // tile-index bits
    uint32_t nvar;          // 4 + ncol_bits
    uint32_t a_chunk_bytes; // bytes of one A chunk (hi then lo)
    uint32_t pad;
    uint64_t a_off;         // byte offset of this stage's A chunks in the A blob
    uint8_t glob_pos[kMaxQ];
    uint8_t var_role[12];   // 0..3: bit j of the chunk's amplitude index; 8 + c: column bit c
    uint64_t var_phys[12];  // 1 << physical position
    uint64_t hi_local[4];   // physical value of local bits 4..keff-1 (chunk index bits)
};

}  // namespace svk

namespace svh {
struct Plan;
struct GemmProgram {
    std::vector<svk::GemmStage> stages;
    std::vector<uint8_t> ablob;
    bool identity_map = true;
};
// prec: 1 = TF32x3, 2 = BF16x3.  Returns "" or an error.
std::string plan_gemm(const Plan& plan, const double* params, int prec, GemmProgram* out);
}  // namespace svh
