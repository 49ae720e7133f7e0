// jit.h — per-stage specialised sweep kernels, generated and compiled at run time.
//
// The paper turns each partition into generated code (Sec. 4.3, "From Partitions to
// Code"); here each stage of a lowered complex64 program becomes one CUDA kernel whose
// tile geometry, register groups and op sequence are compiled in, so the op dispatch,
// descriptor loads and runtime bit loops of the generic interpreter disappear.  The
// kernel source depends only on the stage's structure (bit positions inside the tile,
// op kinds and register bits); every numeric value (gate matrices, phase angles,
// physical bit positions, control masks) travels in the launch's argument block, so
// a kernel is reused across parameter values and across stages of the same shape.
//
// Kernels are compiled with NVRTC for sm_103a and cached per process by source text.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "program.h"

namespace svk {
struct PauliSweep;
struct PauliTerm;
}  // namespace svk

namespace svj {

// One stage of a packed complex64 program (host copies of its blob sections).
struct StageView {
    const svk::Stage* st;
    const svk::Group* groups;            // this stage's groups
    const svk::DevOp<float>* ops;        // this stage's ops (group op_off is relative)
    const svk::DevTerm<float>* terms;    // the program's whole term array
    const svk::PhaseSlot<float>* slots;  // this stage's phase slots
    int n;                               // state width
    int nv;                              // 1: forward (psi); 2: adjoint (psi and lambda)
    // batched mode: one launch sweeps the stage of many circuits of the same structure,
    // circuit c's state at v0 + c 2^n (lambda at v1 + c 2^n); bound ops (F_BIND) take
    // their angle from params[pofs[c] + index]; gradient partials per circuit segment
    int batched = 0;
    int zero_init = 0;                   // batched forward stage 0: tiles start as |0...0>
    // forward, not batched: write the tile out of place (to v1) through a bit map,
    // dst[physical bit] = destination bit (the final qubit order); nullptr = in place
    const int* dst = nullptr;
};

struct Kernel;

// A generated stage: kernel source (structure only) and its argument block (values).
struct Built {
    std::string src;
    std::string name;
    std::vector<uint8_t> args;   // pointers at offsets 0 (v0), 8 (v1), 16 (partial) patched at launch
    uint32_t nthr = 0, smem = 0, n_slots = 0;
    uint64_t ntiles = 0;
    // TMA tile staging (tma): the state seen as a 5-D tensor of 8-byte elements whose
    // dimensions are runs of consecutive physical bits; the tile is one box
    bool tma = false;
    uint64_t gdim[5] = {1, 1, 1, 1, 1};
    uint64_t gstride[4] = {0, 0, 0, 0};   // bytes, dimensions 1..4
    uint32_t box[5] = {1, 1, 1, 1, 1};
    Kernel* kernel = nullptr;    // set by compile()
};

// Generate the kernel of one stage.  Returns "" or an error (an op the generator does
// not handle: the caller then reports it; there is no fallback path).
std::string generate(const StageView& v, Built* out);

// Compile every kernel not yet in the cache (in parallel host threads).
std::string compile(std::vector<Built*>& kernels);

// Launch a built stage: persistent grid of min(tiles, CTAs per SM x SMs) CTAs.
// grid_out: CTAs launched (rows of gradient partials for the adjoint).  flag: device
// int set to 1 if a bounded wait of the kernel gave up (the caller reports it).
cudaError_t launch(const Built& b, void* v0, void* v1, double* partial, int* flag, cudaStream_t s,
                   uint32_t* grid_out);

// Batched launch (StageView::batched): ncirc circuits; params / pofs as above.
// Gradient partials: partial[(c 2^(n-T) + t) * n_slots + s] for the first tile t of each
// run of tiles a CTA processes for circuit c (other rows untouched: zero them first).
cudaError_t launch_batched(const Built& b, void* v0, void* v1, double* partial, int* flag, const double* params,
                           const uint32_t* pofs, uint32_t ncirc, cudaStream_t s);

// Load a compiled kernel and set its launch attributes (before a stream capture).
cudaError_t preload(const Built& b);

// A Pauli-sum expectation sweep (complex64, expectation only): the terms of one sweep of
// the host's Pauli plan (diagonal classes, then X / Y terms; kernels.h) compiled into one
// kernel.  Launch with launch(b, psi, nullptr, partial, nullptr, s, &grid): every CTA
// writes partial[blockIdx] = its tiles' sum of Re(conj(psi) (O_sweep psi)) in FP64.
// Returns "" or an error (a sweep shape the generator does not handle: the caller then
// runs the generic sweep kernel).
std::string generate_pauli(const svk::PauliSweep& sw, const svk::PauliTerm* terms, int n, Built* out);

// NVRTC compiles and cache hits since load (diagnostics).
void stats(uint64_t* compiles, uint64_t* hits, double* compile_ms);

}  // namespace svj
