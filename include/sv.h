/*
 * sv.h — C ABI of the GB300 state-vector engine for closeness-centrality
 * partitioned quantum circuits.
 *
 * What it computes.  A circuit is a flat gate list applied to an n-qubit state
 * psi (2^n complex amplitudes; qubit q is bit q of the amplitude index).  The
 * exact result is psi = U_G ... U_1 psi_0 with the gates in their original order
 * (Sec. 3.2; Sec. 4.1: gates are neither permuted nor replaced).  The host builds
 * the gate-dependency graph and partitions it by closeness centrality (Sec. 4.2);
 * the GPU then executes each partition as one sweep over the state held in HBM:
 * a partition's local qubits become the bits of a shared-memory tile, its other
 * qubits index the tiles (Sec. 4.3, "Partitioning the Input/Output Tensors" and
 * the single-device pack/unpack into shared memory).
 *
 * Conventions shared by every call
 *  - Every call returns sv_status; SV_OK (0) on success.  Nothing throws across
 *    the ABI.  sv_last_error() returns a message for the calling thread's most
 *    recent failure (valid until that thread's next call).
 *  - Device pointers are CUDA global-memory pointers on the handle's device;
 *    host pointers are ordinary CPU memory.  "Borrowed" means the caller owns the
 *    memory and must keep it alive (and unmodified by other streams) while the
 *    handle may use it; "library-owned" objects are freed by the matching
 *    destroy call.
 *  - Work is enqueued on the handle's CUDA stream and is asynchronous unless the
 *    call returns host values (sv_expval, sv_norm, sv_grad, sv_get_state_host),
 *    which synchronise that stream.
 *  - There is no CPU fallback: every state operation runs in the library's CUDA
 *    kernels.  Without a usable GPU, state calls return SV_ERR_CUDA.  The host
 *    partitioning calls (sv_partition*, sv_plan_*) need no GPU.
 *  - Amplitude layout: complex64 = {float re, float im}, complex128 =
 *    {double re, double im}, contiguous, index = sum_q bit_q * 2^q.  Between
 *    calls the state is always in this canonical layout.
 */
#ifndef SV_GB300_H
#define SV_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SV_OK = 0,
    SV_ERR_ARG = 1,          /* invalid argument (null pointer, bad size, bad gate)         */
    SV_ERR_OOM = 2,          /* device or host allocation failed                            */
    SV_ERR_CUDA = 3,         /* a CUDA runtime call or kernel launch failed / no GPU        */
    SV_ERR_PARTITION = 4,    /* a gate needs more local qubits than the budget L allows     */
    SV_ERR_UNSUPPORTED = 5,  /* valid request this build does not implement                 */
    SV_ERR_TIMEOUT = 6       /* a bounded device-side wait gave up (error flag, no hang)     */
} sv_status;

typedef enum { SV_C64 = 0, SV_C128 = 1 } sv_dtype;

/* Arithmetic used for stage sweeps.  SV_PREC_CUDACORE: complex FP32 (complex64
 * states) or FP64 (complex128 states) on the CUDA cores.  The split-precision
 * tensor-core modes apply stages fused into dense 2^k x 2^k unitaries as GEMMs.
 * The tensor cores' FP32 accumulation rounds toward zero, so every fused stage
 * shrinks the state by about 1e-6 of its norm (nearly all of the split-precision
 * error is this shrink); every stage is unitary, so a tensor-core run restores the
 * input's norm at its end (an FP64 norm before and after, one scaling sweep).
 * SV_PREC_NO_RENORM, OR-ed into a tensor-core mode, skips that step (to measure the
 * raw split-precision error). */
typedef enum { SV_PREC_CUDACORE = 0, SV_PREC_TF32X3 = 1, SV_PREC_BF16X3 = 2, SV_PREC_NO_RENORM = 0x100 } sv_prec;

/* Gate kinds.  Matrices (Sec. 3.1): H, Pauli X/Y/Z, S = P(pi/2), SDG = P(-pi/2),
 * T = P(pi/4), TDG = P(-pi/4), RX/RY/RZ(t) = exp(-i t {X,Y,Z} / 2),
 * P(a) = diag(1, e^{ia}) (the paper prints e^{-ja}; this library uses the usual
 * +i sign), U3(t,p,l) = [[cos t/2, -e^{il} sin t/2], [e^{ip} sin t/2, e^{i(p+l)} cos t/2]],
 * CX/CY/CZ controlled Paulis, CP(a) = diag(1,1,1,e^{ia}), SWAP. */
enum {
    SV_GATE_H = 1, SV_GATE_X, SV_GATE_Y, SV_GATE_Z, SV_GATE_S, SV_GATE_SDG, SV_GATE_T,
    SV_GATE_TDG, SV_GATE_RX, SV_GATE_RY, SV_GATE_RZ, SV_GATE_P, SV_GATE_U3, SV_GATE_CX,
    SV_GATE_CY, SV_GATE_CZ, SV_GATE_CP, SV_GATE_SWAP
};

/* One gate, 40 bytes, no implicit padding.  q[0] is the control of CX/CY/CP/CZ,
 * q[1] the target.  param >= 0 makes the gate's single angle params[param]
 * (RX, RY, RZ, P, CP only); param = -1 uses angle[] (U3 uses all three). */
typedef struct {
    uint16_t kind;
    uint8_t  nq;
    uint8_t  q[3];
    uint16_t reserved;
    int32_t  param;
    double   angle[3];
} sv_gate;

/* A circuit (borrowed for the duration of the call that receives it). */
typedef struct {
    uint32_t n_qubits;
    uint32_t n_gates;
    uint32_t n_params;
    const sv_gate* gates;
} sv_circuit;

/* Sum of Pauli strings.  pauli[t * n_qubits + q] in {0=I, 1=X, 2=Y, 3=Z} is the
 * factor on qubit q of term t; coeff[t] its real coefficient.  Borrowed. */
typedef struct {
    uint32_t n_terms;
    uint32_t n_qubits;
    const uint8_t* pauli;
    const double* coeff;
} sv_observable;

typedef struct sv_handle_s* sv_handle;
typedef struct sv_plan_s sv_plan;

/* Work counters of the last sv_run / sv_grad on a handle. */
typedef struct {
    uint32_t stage_sweeps;       /* read+write passes over psi by stage kernels          */
    uint32_t permutation_sweeps; /* bit-permutation passes                              */
    uint32_t reduction_sweeps;   /* read-only / observable passes                       */
    uint32_t backward_sweeps;    /* adjoint passes (psi and lambda together)             */
    uint32_t kernel_launches;    /* kernels this library launched in the call           */
    double   hbm_bytes;          /* algorithmic bytes moved (reads + writes)            */
} sv_run_info;

/* ---------------------------------------------------------------------------
 * Errors
 * ------------------------------------------------------------------------- */
/* Message of the calling thread's last failure ("" if none).  Library-owned. */
const char* sv_last_error(void);

/* ---------------------------------------------------------------------------
 * Handles (state vectors)
 * ------------------------------------------------------------------------- */
/* Create a handle for an n_qubits state (1 <= n_qubits <= 34) of the given dtype.
 * dev_state: borrowed device buffer of 2^n amplitudes (16-byte aligned), or NULL
 * to let the library allocate (and own) one initialised to |0...0>.
 * cuda_stream: a cudaStream_t to enqueue on (NULL = the legacy default stream).
 * Errors: SV_ERR_ARG (bad n, dtype, null out, misaligned buffer), SV_ERR_OOM,
 * SV_ERR_CUDA (no device). */
sv_status sv_create(uint32_t n_qubits, sv_dtype dtype, void* dev_state, void* cuda_stream,
                    sv_handle* out);

/* Free the handle and every library-owned buffer (not a borrowed state). */
sv_status sv_destroy(sv_handle h);

/* Number of qubits, dtype and the device pointer of the state.  A borrowed buffer
 * never changes; a library-owned state may move to the handle's second state-sized
 * buffer after sv_run (see there), so read the pointer again after a run. */
sv_status sv_info(sv_handle h, uint32_t* n_qubits, sv_dtype* dtype, void** dev_state);

/* Set psi to |0...0>.  Async. */
sv_status sv_reset_zero(sv_handle h);

/* Copy 2^n amplitudes from / to device memory (async, stream-ordered). */
sv_status sv_set_state(sv_handle h, const void* dev_src);
sv_status sv_get_state(sv_handle h, void* dev_dst);

/* Copy 2^n amplitudes from / to host memory.  Pinned host memory gives full
 * transfer speed; set is async with respect to the host only for pinned memory,
 * get synchronises the stream. */
sv_status sv_set_state_host(sv_handle h, const void* host_src);
sv_status sv_get_state_host(sv_handle h, void* host_dst);

/* Wait for all work queued on the handle's stream. */
sv_status sv_synchronize(sv_handle h);

/* Counters of the last sv_run / sv_grad. */
sv_status sv_last_run_info(sv_handle h, sv_run_info* out);

/* Per-kernel device time, accumulated while timing is enabled on a handle. */
typedef struct {
    double   stage_ms;          /* forward stage sweeps        */
    double   backward_ms;       /* adjoint stage sweeps        */
    double   permute_ms;        /* bit-permutation sweeps      */
    double   observable_ms;     /* Pauli / norm sweeps         */
    uint32_t stage_launches;
    uint32_t backward_launches;
    uint32_t permute_launches;
    uint32_t observable_launches;
} sv_timing;

/* enable != 0: record a CUDA event pair on the handle's stream around every
 * sweep kernel the handle launches (negligible overhead); 0 stops recording. */
sv_status sv_timing_enable(sv_handle h, int enable);

/* Sum the recorded event pairs into *out (synchronises the stream); reset != 0
 * clears the record afterwards. */
sv_status sv_timing_read(sv_handle h, sv_timing* out, int reset);

/* ---------------------------------------------------------------------------
 * Partitioning (host only; Sec. 4.1-4.2)
 * ------------------------------------------------------------------------- */
/* Build the contraction DAG (each gate a node, edges = qubit dimensions, critical
 * path level l_g = 1 + max over predecessors), compute exact closeness centrality
 * CC(v) = |RN(v)|^2 / (N * dist(v)) with RN the reachable set and
 * dist(v) = sum_{x in RN(v)} (l_x - l_v) (Sec. 4.2 equations; the overlap
 * threshold heuristic is unnecessary because the distance sum is exact), and cut
 * the circuit into partitions whose required qubits fit L local qubits with the
 * forward frontier pass of Sec. 4.2 (highest CC first, ties by gate index;
 * diagonal gates and non-local controls exempt; SWAP executed as a relabel).
 * L is the width of the shared-memory tile in qubits.  sv_partition reserves the
 * min(4, L - 1, n) lowest physical qubits in every partition: a tile must contain them
 * so that each HBM access is a contiguous run of >= 128 bytes.  The plan is
 * deterministic, library-owned, independent of any handle and of the dtype.  A
 * circuit with no gates has no partitions (running it leaves the state unchanged).
 * Errors: SV_ERR_ARG (bad circuit: qubit out of range, unknown kind, bad param
 * slot; L < 1 or > 14), SV_ERR_PARTITION (a gate's qubits cannot be made local). */
sv_status sv_partition(const sv_circuit* circuit, uint32_t L, sv_plan** out);

/* As sv_partition with an explicit number of reserved low qubits (0 gives the
 * paper's unconstrained partitioner, e.g. for its worked examples). */
sv_status sv_partition_ex(const sv_circuit* circuit, uint32_t L, uint32_t n_fixed, sv_plan** out);

/* Partition for the split-precision tensor-core stages: the same DAG, closeness and
 * frontier pass, but without the two exemptions (every qubit of every gate must be
 * local; SWAP stays a relabel), so each partition is one fixed dense unitary on its k
 * local qubits, fused in FP64 and applied as a GEMM over all 2^(n-k) columns
 * (sv_run with SV_PREC_TF32X3 or SV_PREC_BF16X3; complex64 states, n >= k + 4).
 * k in {5, 6, 7} (k = 5 stages run as k = 6 with an identity qubit).  Such a plan can
 * also run on the CUDA cores (SV_PREC_CUDACORE).  Errors as sv_partition. */
sv_status sv_partition_gemm(const sv_circuit* circuit, uint32_t k, sv_plan** out);

/* Layout of a tensor-core plan's stages for prec (SV_PREC_TF32X3 / SV_PREC_BF16X3),
 * computed on the host (no GPU; an introspection call with no counterpart in the paper,
 * whose partitions are the fused stages of Sec. 4.2 run without exemptions): keff[s] = local qubits of stage s's fused unitary (6
 * or 7), resident[s] = 1 when its B operand stays in shared memory for the launch,
 * nslot[s] = depth of its operand ring, lane_roles[6 s + i] = what producer lane bit i
 * (i < 5) and the 16-byte pair bit (i = 5) select: 0..4 = a bit of the amplitude index
 * inside a K chunk, 8 + c = column bit c (the operand row), 255 = none.  params as for
 * sv_run (NULL when the circuit has none).  Arrays may be NULL; each holds *n_stages
 * entries (lane_roles 6 *n_stages); query *n_stages first.  Errors: SV_ERR_ARG,
 * SV_ERR_UNSUPPORTED (not a tensor-core plan, or a stage the kernel cannot hold). */
sv_status sv_gemm_plan_info(const sv_plan* plan, const double* params, sv_prec prec, uint32_t* n_stages,
                            uint32_t* keff, uint32_t* resident, uint32_t* nslot, uint8_t* lane_roles);

/* Partition for the hierarchical tensor-core stages (Sec. 4.2: the partitioner invoked
 * again inside each partition, for the next memory level; Sec. 5.2's multi-level
 * fusion).  Level 1: the same DAG, closeness and frontier pass without exemptions, with
 * L = k + 7 local qubits and qubits 0..3 reserved, one tile of a CTA in shared memory;
 * level 2 (formed at sv_run): each stage's gates partitioned again with budget k inside
 * its tile, each sub-partition one fused 2^k x 2^k unitary applied by the tensor cores
 * to the tile's 128 columns, so a stage is one HBM pass however many sub-partitions it
 * holds.  Run with sv_run and SV_PREC_BF16X3 (k = 5 or 6) or SV_PREC_TF32X3 (k = 5);
 * complex64 states of at least k + 7 qubits.  Such a plan also runs on the CUDA cores.
 * Errors: SV_ERR_ARG (k not 5 or 6, null argument), SV_ERR_UNSUPPORTED (fewer than
 * k + 7 qubits), SV_ERR_PARTITION. */
sv_status sv_partition_hier(const sv_circuit* circuit, uint32_t k, sv_plan** out);

/* Shape of a hierarchical plan for prec, computed on the host (no GPU; introspection
 * with no counterpart in the paper): *n_launches = stage launches (a stage of more than
 * 24 sub-partitions takes several), *n_sub = sub-partitions (GEMMs per tile) in all.
 * Either pointer may be NULL.  params as for sv_run.  Errors: SV_ERR_ARG,
 * SV_ERR_UNSUPPORTED (not a hierarchical plan, or a combination the kernel lacks). */
sv_status sv_hier_plan_info(const sv_plan* plan, const double* params, sv_prec prec, uint32_t* n_launches,
                            uint32_t* n_sub);

/* Partition summary.  local_masks[s] = physical-bit mask of stage s's local set
 * (after SWAP relabelling); gate_counts[s] = gates in stage s.  Either array may be
 * NULL; each must hold n_stages entries (query n_stages first with both NULL). */
sv_status sv_plan_stages(const sv_plan* plan, uint32_t* n_stages, uint64_t* local_masks,
                         uint32_t* gate_counts);

/* Gate ids in execution order (n_gates entries) and the final map circuit qubit ->
 * physical bit (n_qubits entries).  Either may be NULL. */
sv_status sv_plan_order(const sv_plan* plan, uint32_t* gate_order, uint32_t* final_map);

/* Exact closeness of every gate as the integers |RN(v)| and dist(v), and the
 * critical-path level l_v (arrays of n_gates; any may be NULL). */
sv_status sv_plan_centrality(const sv_plan* plan, uint32_t* reach, uint64_t* dist, uint32_t* level);

/* Free a plan. */
sv_status sv_plan_destroy(sv_plan* plan);

/* Read an OpenQASM 2.0 program into a flat gate list (Sec. 4.1: the circuit enters
 * as a QASM file; Step A then builds the dependency graph from the gate list).
 * Accepted: the OPENQASM header, include lines, qreg / creg declarations (several
 * quantum registers are numbered one after another), gate calls on single qubits or
 * element-wise on whole registers, parameter expressions (numbers, pi, + - * / ^,
 * unary minus, parentheses, sin cos tan exp ln sqrt), and the gates id u u1 u2 u3 U p
 * x y z h s sdg t tdg rx ry rz cx CX cy cz cp cu1 swap rzz (rzz(t) a,b becomes
 * CX(a,b) RZ(t)(b) CX(a,b), the same unitary); measure and barrier emit nothing.
 * Gate definitions, opaque gates, reset and conditionals are rejected.
 * text: NUL-terminated.  gates: caller-owned array of capacity entries, or NULL to
 * only count.  On success *n_qubits and *n_gates hold the circuit's sizes (also when
 * gates is NULL).  Errors: SV_ERR_ARG with the line and reason in sv_last_error
 * (syntax, unknown register or gate, index out of range, capacity too small, more
 * than 255 qubits).  Host only. */
sv_status sv_qasm_parse(const char* text, sv_gate* gates, uint32_t capacity, uint32_t* n_qubits,
                        uint32_t* n_gates);

/* Generate and compile ahead of time the complex64 stage kernels of a plan (Sec. 4.3,
 * "From Partitions to Code": each partition becomes one generated kernel with its
 * tile geometry, register groups and gate sequence compiled in; here compiled at run
 * time with NVRTC for sm_103a).  sv_run / sv_grad on complex64 states generate and
 * compile the same kernels on first use; this call lets a caller pay that cost before
 * a timed or latency-critical loop.  Kernels are cached for the life of the process
 * by source text; their source depends on the partition's structure only (gate kinds
 * and bit positions), not on angle values, so one compile serves every parameter
 * value.  which: bit 0 = forward sweeps (sv_run), bit 1 = adjoint sweeps (sv_grad).
 * params: host array of n_params angles (NULL if n_params == 0).  n_kernels
 * (nullable): stage kernels of the plan (cache hits included).  Host only: needs no
 * GPU.  Errors: SV_ERR_ARG, SV_ERR_UNSUPPORTED (tensor-core plan, unsupported
 * parameter kind), SV_ERR_CUDA (the compiler failed; sv_last_error has its log). */
sv_status sv_plan_compile(const sv_plan* plan, const double* params, uint32_t which, uint32_t* n_kernels);

/* Counters of the run-time compiled stage kernels since the library was loaded: NVRTC
 * compilations, cache hits, and the compile wall time in milliseconds (any pointer may
 * be NULL).  Host only. */
sv_status sv_jit_stats(uint64_t* compiles, uint64_t* cache_hits, double* compile_ms);

/* Generate and compile ahead of time (host only, no GPU) the kernels sv_expval uses for
 * this observable (Sec. 4.2's Pauli-sum observable; code generation as in Sec. 4.3) on a
 * complex64 state of n_qubits: one expectation-only kernel per
 * Pauli sweep with the sweep's terms compiled in (sv_expval generates them on first use
 * otherwise; they are cached by source for the process).  *n_kernels (may be NULL) =
 * kernels made ready; 0 for complex128, whose sweeps run the generic sweep kernel.
 * Errors: SV_ERR_ARG (bad width, dtype or observable), SV_ERR_UNSUPPORTED (a term wider
 * than a sweep's tile), SV_ERR_CUDA (run-time compilation failed). */
sv_status sv_pauli_compile(uint32_t n_qubits, sv_dtype dtype, const sv_observable* obs, uint32_t* n_kernels);

/* ---------------------------------------------------------------------------
 * Execution
 * ------------------------------------------------------------------------- */
/* Apply the planned circuit to the handle's state: one stage-sweep kernel per
 * partition.  If the SWAP relabels leave a non-identity qubit map, the complex64
 * path writes the last stage's tiles out of place through that map (the data
 * reshaping of Sec. 4.3 fused into the last stage's write-back; no permutation
 * sweep) into the handle's second state-sized buffer, which then becomes the state
 * of a library-owned handle or is copied back into a borrowed one; complex128
 * stages run in place and then one bit-permutation sweep.  params: host array of the circuit's n_params angles
 * (NULL if n_params == 0).  prec: SV_PREC_CUDACORE, or a tensor-core mode (needs a
 * plan from sv_partition_gemm or sv_partition_hier; one tcgen05 GEMM kernel per
 * partition, then the input's norm restored unless SV_PREC_NO_RENORM is set, then the
 * call synchronises to check the kernels' bounded waits, SV_ERR_TIMEOUT if one gave
 * up).  Async for SV_PREC_CUDACORE.
 * Errors: SV_ERR_ARG (width mismatch, null params), SV_ERR_UNSUPPORTED
 * (precision / dtype / plan combination), SV_ERR_CUDA. */
sv_status sv_run(sv_handle h, const sv_plan* plan, const double* params, sv_prec prec);

/* Bit-permutation sweep: new[y] = old[x] where bit phys_of_qubit[q] of x equals
 * bit q of y (Sec. 4.3 data reshaping; on one GPU the exchange is a relabel plus
 * this sweep).  phys_of_qubit: host array of n entries, a permutation. */
sv_status sv_permute(sv_handle h, const uint32_t* phys_of_qubit);

/* The tile sv_permute uses for phys_of_qubit on an n_qubits state of dtype, computed on
 * the host (no GPU, no handle; an introspection call with no counterpart in the paper):
 * *tile_bits = the tile's width T (12 for complex64, 11 for complex128, n if smaller),
 * *tile_mask = its input physical bits (the lowest 4, the inputs of output bits 0..3,
 * then alternately widening the contiguous input and output runs), *in_run = the number
 * of lowest input bits it holds contiguously (a read is a run of 2^in_run amplitudes),
 * *out_run = the same for the output bits.  Errors: SV_ERR_ARG (null pointer, bad width
 * or dtype, not a permutation). */
sv_status sv_permute_plan_info(uint32_t n_qubits, sv_dtype dtype, const uint32_t* phys_of_qubit, uint32_t* tile_bits,
                               uint64_t* tile_mask, uint32_t* in_run, uint32_t* out_run);

/* <psi|O|psi> for a Pauli sum (Sec. 4.2's observable, evaluated by Pauli sweeps:
 * one read of psi per group of X/Y-carrying terms whose X/Y qubits fit one tile of 13
 * (complex64) or 12 (complex128) qubits together with qubits 0..3; the diagonal terms
 * join the first sweep).  Each term's X/Y factors must fit such a tile: for wider states
 * at most 9 (complex64) or 8 (complex128) X/Y factors outside qubits 0..3 (physical
 * positions), else SV_ERR_UNSUPPORTED.  Reduction: complex64 states sum in FP32 over
 * one thread's 16 amplitudes per tile, compensated FP32 across its tiles, FP64 across
 * threads and CTAs in a fixed order; complex128 states sum in FP64.  Result written
 * to *out (host); synchronises.  Errors: SV_ERR_ARG (width mismatch, null or invalid
 * Pauli codes), SV_ERR_UNSUPPORTED, SV_ERR_CUDA. */
sv_status sv_expval(sv_handle h, const sv_observable* obs, double* out);

/* The Pauli-sweep grouping sv_expval uses for obs on an n_qubits state of dtype, computed
 * on the host (no GPU, no handle; an introspection call with no counterpart in the
 * paper): *n_sweeps sweeps; tile_masks[i] = the qubits held in
 * sweep i's shared-memory tile, reg_masks[i] = those of them held in registers (each
 * thread's element index), n_terms[i] = the terms evaluated in sweep i (every diagonal
 * term in sweep 0).  The arrays may be NULL (query *n_sweeps first); each must hold
 * *n_sweeps entries.  Errors: SV_ERR_ARG, SV_ERR_UNSUPPORTED (a term's X/Y factors do
 * not fit one tile). */
sv_status sv_pauli_plan_info(uint32_t n_qubits, sv_dtype dtype, const sv_observable* obs, uint32_t* n_sweeps,
                             uint64_t* tile_masks, uint64_t* reg_masks, uint32_t* n_terms);

/* ||psi||^2 in FP64; synchronises. */
sv_status sv_norm(sv_handle h, double* out);

/* ||psi||^2 in FP64 without allocating anything (the paper has no counterpart).
 * For callers that cannot call cudaMalloc: their device memory already belongs to
 * their own allocator, or an allocation's implicit device synchronisation is not
 * acceptable where they call.  No handle is needed and nothing is allocated: the
 * caller passes the state (dev_state: 2^n_qubits amplitudes of dtype, 16-byte
 * aligned, on the current device) and dev_out (one device double, written with the
 * result); the per-block partial sums use a file-scope static device array of
 * 2^14 doubles (128 KiB, held by every GPU that loads the library until exit), one
 * partial per 2^18 amplitudes, so n_qubits is limited to [1, 32]; larger states are
 * rejected with SV_ERR_ARG.  The first call on a device looks the array's device
 * address up (with that device current); make that first call before any stream
 * capture.  Work is enqueued on cuda_stream (NULL = legacy default stream) and the
 * call returns without synchronising.  Every call shares the one array: calls that
 * overlap on the GPU (different streams, or different host threads) race on it and
 * must be serialised by the caller.  Errors: SV_ERR_ARG, SV_ERR_CUDA. */
sv_status sv_norm_noalloc(const void* dev_state, uint32_t n_qubits, sv_dtype dtype, void* cuda_stream,
                          double* dev_out);

/* Adjoint differentiation of E(theta) = <psi(theta)|O|psi(theta)>: runs the
 * forward circuit from the current state, forms lambda = O psi, then un-applies
 * the partitions in reverse to psi and lambda together while accumulating
 * dE/dtheta_p = 2 Re <lambda| dU_p/dtheta psi> for every parameter (RX, RY, RZ
 * parameters supported).  On return the handle holds the backward pass's
 * reconstruction of the input state (the circuit un-applied: the input up to
 * rounding).  expval_out (host, may be NULL) receives E; grad_out (host, n_params)
 * the gradient.  Synchronises.  Errors: SV_ERR_UNSUPPORTED for parameters on other
 * gate kinds, and for partitions whose psi and lambda tiles together exceed shared
 * memory (L = 14 for complex64, L >= 13 for complex128). */
sv_status sv_grad(sv_handle h, const sv_plan* plan, const double* params, const sv_observable* obs,
                  double* expval_out, double* grad_out);

/* ---------------------------------------------------------------------------
 * Batched circuits (many small circuits, one persistent launch)
 *
 * The paper partitions one circuit at a time; this form runs many independent
 * circuits of uneven width together.  Each circuit is partitioned by closeness
 * centrality exactly as sv_partition does (budget L = its tile width), except that
 * parametric RZ gates need their qubit (they are lowered as dense ops so that the
 * program's structure does not depend on the angles).  Circuits with the same
 * structure share one lowered program; the kernel forms every RX / RY / RZ matrix
 * from the circuit's own parameters.  One CTA runs one circuit (forward stages, E =
 * <psi|O|psi>, lambda = O psi, adjoint stages with gradient accumulation, Sec. 4.2
 * partitions as in sv_grad), taking circuits largest first from a device queue.  A
 * circuit whose tile holds all its qubits never leaves shared memory.  The whole
 * evaluation (parameter upload, queue reset, the launch, result download) is one
 * CUDA graph, captured when the batch is built.
 * ------------------------------------------------------------------------- */
typedef struct sv_batch_s sv_batch;

/* Per-width tuning table: for circuits of n qubits, L[n] = tile width (qubits held
 * in shared memory per tile, 7..13; a circuit with n <= L[n] is held whole) and
 * k[n] = register-group width (qubits whose gates one thread applies from registers
 * between shared-memory passes, 2..4, at most L[n] - 5; the fusion width of this
 * form).  0 = default (L = min(n, 13), k = 4). */
typedef struct {
    uint8_t L[41];
    uint8_t k[41];
} sv_tune;

typedef struct {
    uint32_t n_circuits;
    uint32_t n_programs;         /* distinct lowered structures                          */
    uint32_t n_resident;         /* circuits held whole in shared memory                 */
    uint32_t total_params;
    uint64_t workspace_bytes;    /* HBM workspace (psi and lambda of multi-stage circuits) */
    uint32_t smem_bytes;         /* dynamic shared memory per CTA                        */
    uint32_t grid;               /* CTAs of the persistent launch                        */
    uint32_t graph;              /* 1: the evaluation is a captured CUDA graph           */
    uint32_t pad;
    double   last_ms;            /* device time of the last sv_run_batch (graph launch)  */
} sv_batch_info;

/* Build a batch.  circuits[i] (n_qubits in [7, 30]) and observables[i] (a sum of
 * Z strings: every Pauli factor I or Z; n_qubits must match) describe circuit i;
 * its parameters are params[param_off_i ...] with param_off_i the sum of the
 * n_params of the circuits before it, and the gradient uses the same layout.
 * Parametric gates: RX, RY, RZ only.  tune: NULL = defaults.  cuda_stream as for
 * sv_create.  Everything is copied; the inputs may be freed on return.
 * Errors: SV_ERR_ARG, SV_ERR_UNSUPPORTED (X / Y observable factors, parametric
 * P / CP, shared memory above the per-CTA limit), SV_ERR_PARTITION, SV_ERR_OOM,
 * SV_ERR_CUDA. */
sv_status sv_batch_create(const sv_circuit* circuits, const sv_observable* observables, uint32_t n_circuits,
                          const sv_tune* tune, void* cuda_stream, sv_batch** out);

/* Evaluate every circuit at params (host, total_params): expval_out[i] (host,
 * n_circuits) = <psi_i|O_i|psi_i> reduced in FP64, grad_out (host, total_params,
 * may be NULL) = dE_i/dtheta by the adjoint method.  Replays the captured graph and
 * synchronises.  Errors: SV_ERR_ARG, SV_ERR_CUDA. */
sv_status sv_run_batch(sv_batch* b, const double* params, double* expval_out, double* grad_out);

/* Autotuner: for every distinct width n in the batch, time the candidate
 * (L, k) pairs on up to one wave (one circuit per SM) of the batch's own circuits of
 * that width (CUDA events, one warm-up then one timed run; candidates: L = n with
 * k in {2, 3, 4} for n <= 13, L in {11, 12, 13} with k in {3, 4} for wider circuits),
 * keep the fastest, rebuild the batch with the chosen table and re-capture its
 * graph.  params: as for sv_run_batch (the timing runs use them).  table_out (may be
 * NULL) receives the table.  Errors: as sv_batch_create. */
sv_status sv_autotune(sv_batch* b, const double* params, sv_tune* table_out);

sv_status sv_batch_info_get(const sv_batch* b, sv_batch_info* out);
sv_status sv_batch_destroy(sv_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* SV_GB300_H */
