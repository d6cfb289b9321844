/*
 * tn.h - C ABI of libtnq: GB300 (sm_103a) contraction of quantum-circuit tensor networks.
 *
 * The problem follows "Tensor Networks for Simulating Quantum Circuits on FPGAs"
 * (arXiv 2108.06831):
 *   - a register of N qubits evolves by gates applied in sequence, each a unitary
 *     acting as psi' = U psi, multi-qubit operators being Kronecker products (Sec. 2.1);
 *   - the circuit is a tensor network whose open legs are the state's indices
 *     (Sec. 2.2.2, Eq. 2.3); closing those legs with a final basis state gives one
 *     amplitude (Sec. 2.2.3);
 *   - contracting a pair of tensors is a sum over their shared indices, i.e. a
 *     (batched) matrix product once the legs are grouped (Sec. 2.2.1, Eq. 2.2), and
 *     the contraction order is a free choice planned ahead (Sec. 2.2.3, Sec. 3).
 *
 * Conventions used by every entry point:
 *   - qubit q of an N-qubit register is bit (N-1-q) of a basis index (most significant
 *     first: |00>,|01>,|10>,|11> are |0>..|3>, Sec. 2.1); bitstrings are uint64 with the
 *     same mapping (N <= 63);
 *   - states and amplitudes are complex64, interleaved (re, im) float pairs; a batch of B
 *     states is B consecutive vectors of 2^N entries;
 *   - a two-qubit gate on (a, b) has a 4x4 matrix indexed 2*bit(a) + bit(b);
 *   - parameters are float64, laid out [batch][n_params]; gradients likewise.
 *
 * Ownership and errors:
 *   - the caller owns every device buffer and the stream; the library owns the opaque
 *     handles (circuit, plan, observable) and their device-side tables, which it
 *     allocates when a plan or observable is built and frees in tn_free_*;
 *   - calls that take a stream only enqueue work on it (asynchronous); none allocates
 *     device memory; none throws across the ABI;
 *   - argument checks return a status at once and leave the stream untouched; the text
 *     of the last error on the calling thread is in tn_last_error();
 *   - a device-side failure (a bounded wait that ran out, a non-finite result) is
 *     recorded in a per-device status word and reported by tn_sync_status().
 */
#ifndef TNQ_TN_H
#define TNQ_TN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream (cudaStream_t); NULL means the legacy default stream. */
typedef struct CUstream_st *tn_stream_t;

typedef enum {
  TN_OK = 0,
  TN_ERR_INVALID_ARG = 1, /* a pointer, size, qubit index or option is out of range */
  TN_ERR_UNSUPPORTED = 2, /* valid request this build does not implement (message says which) */
  TN_ERR_OOM = 3,         /* a plan/observable table could not be allocated */
  TN_ERR_CUDA = 4,        /* a CUDA runtime call failed (message holds cudaGetErrorString) */
  TN_ERR_TIMEOUT = 5,     /* a device-side bounded wait ran out (from tn_sync_status) */
  TN_ERR_NUMERIC = 6      /* a device-side non-finite value was detected (from tn_sync_status) */
} tn_status;

/* Gate kinds.  Matrices (Sec. 2.1 leaves them implicit; these are the textbook ones):
 * H = [[1,1],[1,-1]]/sqrt2; X, Y, Z Pauli; S = diag(1,i); SDG = S^dagger; T = diag(1,e^{i pi/4});
 * TDG = T^dagger; SX = RX(pi/2); SY = RY(pi/2); SW = exp(-i pi/4 (X+Y)/sqrt2);
 * RX/RY/RZ(t) = exp(-i t P/2); U3(t,p,l) = [[cos t/2, -e^{il} sin t/2], [e^{ip} sin t/2, e^{i(p+l)} cos t/2]];
 * CZ = diag(1,1,1,-1); CNOT(control = q[0], target = q[1]); CP(p) = diag(1,1,1,e^{ip}); SWAP;
 * MAT1 / MAT2: a caller-supplied 2x2 / 4x4 matrix (row-major complex128, copied at build time). */
typedef enum {
  TN_GATE_H = 0, TN_GATE_X = 1, TN_GATE_Y = 2, TN_GATE_Z = 3,
  TN_GATE_S = 4, TN_GATE_SDG = 5, TN_GATE_T = 6, TN_GATE_TDG = 7,
  TN_GATE_SX = 8, TN_GATE_SY = 9, TN_GATE_SW = 10,
  TN_GATE_RX = 11, TN_GATE_RY = 12, TN_GATE_RZ = 13, TN_GATE_U3 = 14,
  TN_GATE_CZ = 15, TN_GATE_CNOT = 16, TN_GATE_CP = 17, TN_GATE_SWAP = 18,
  TN_GATE_MAT1 = 19, TN_GATE_MAT2 = 20,
  TN_GATE_KIND_COUNT = 21
} tn_gate_kind;

/* One gate of a circuit (host memory, read during tn_build_from_circuit only).
 *   kind       tn_gate_kind
 *   q          qubit indices; q[1] ignored for one-qubit kinds
 *   param_idx  -1: angles are taken from angle[]; >= 0: the gate reads its angles
 *              from params[param_idx .. param_idx + arity - 1] at contraction time
 *              (arity 3 for U3, 1 for RX/RY/RZ/CP; invalid for fixed kinds)
 *   angle      fixed angles (U3: theta, phi, lambda)
 *   mat        MAT1/MAT2 only: row-major complex128 (re, im pairs), 2x2 or 4x4 */
typedef struct {
  int32_t kind;
  int32_t q[2];
  int32_t param_idx;
  double angle[3];
  const double *mat;
} tn_gate;

typedef struct tn_circuit tn_circuit;       /* opaque, library-owned, host only */
typedef struct tn_plan tn_plan;             /* opaque, library-owned, holds device tables */
typedef struct tn_observable tn_observable; /* opaque, library-owned, holds device tables */

typedef enum { TN_TARGET_STATE = 0, TN_TARGET_AMPLITUDES = 1, TN_TARGET_EXPECTATION = 2 } tn_target;

/* Arithmetic of dense pairwise merges (batched complex GEMM):
 *   FP32        CUDA-core FFMA, FP32 accumulate (the plain reference);
 *   3XTF32      tcgen05 kind::tf32, a = hi + lo split, hi*hi + hi*lo + lo*hi, FP32 accumulate in TMEM;
 *   SPLIT_BF16  tcgen05 kind::f16 (bf16), a = a0 + a1 + a2 split, the 6 products with i + j <= 2,
 *               FP32 accumulate in TMEM. */
typedef enum { TN_PREC_FP32 = 0, TN_PREC_3XTF32 = 1, TN_PREC_SPLIT_BF16 = 2 } tn_precision;

#define TN_PLAN_HOST_ONLY 1 /* plan without touching the GPU: only tn_plan_get_stats may use it */
#define TN_PLAN_NETWORK 4 /* TN_TARGET_AMPLITUDES by contracting the circuit's tensor network pairwise
                            * (batched complex GEMMs in opts->precision) instead of contracting the
                            * state; allows up to 63 qubits.  opts->amp_batch (a power of two) is the
                            * number of bitstrings per call the plan is sized for.  When no order found
                            * keeps every intermediate within 2^max_intermediate_log2 entries, the
                            * bitstrings are contracted in smaller passes and/or indices are sliced
                            * (each fixed to 0 and 1 in turn, the slices' amplitudes summed in FP64),
                            * whichever costs less, at most 2^16 slices; beyond that
                            * TN_ERR_UNSUPPORTED. */
#define TN_PLAN_Q428 8 /* a fixed-point plan for tn_contract_state_q428 (Sec. 3: the FPGA datapath's
                         * complex arithmetic in 32-bit fixed point, 28 fractional bits); fixed-angle
                         * circuits, batch 1, target TN_TARGET_STATE, at most 34 qubits */
#define TN_PLAN_NO_FUSION 16 /* apply the gates of the forward passes one by one: no precontraction of
                              * runs of gates on two qubits into dense 4x4 blocks (by default a run whose
                              * gates cost the pass kernels more than one dense 4x4 is precontracted,
                              * per call, in FP64 -- Sec. 3's precomputed small contractions) */
#define TN_PLAN_BLOCKS 32 /* TN_TARGET_STATE by uniform square blocks (Sec. 3: the contraction deployed as
                           * square matrices of one size): the circuit is cut into blocks of gates on
                           * opts->block_qubits = k qubits (6 or 7; windows of k qubits at alternating
                           * offsets, each taking its light cone), every block is precontracted per
                           * call into one 2^k x 2^k unitary (FP64, from the parameters), and applied
                           * to the state viewed as [2^(N-k)] x [2^k] by the batched complex GEMM in
                           * opts->precision (FP32 on the CUDA cores, 3XTF32 or SPLIT_BF16 on the
                           * tensor cores).  Needs k + 7 <= n_qubits (and n_qubits <= k + 23 on the
                           * tensor cores) and a power-of-two batch. */
#define TN_PLAN_NO_SPECIALIZE 2 /* run the interpreting gate-apply kernel instead of plan-specialised
                                 * kernels (those are generated as CUDA C++ and compiled with NVRTC
                                 * when the plan is built; compiled code is cached on disk) */

typedef struct {
  int32_t target;                /* tn_target: what the plan will be used for */
  int32_t precision;             /* tn_precision of dense merges */
  int32_t batch;                 /* parameter sets (states) per call, >= 1 */
  int32_t tile_qubits;           /* 0 = automatic; qubits held on chip per tile of the fused gate-apply kernel */
  int32_t max_intermediate_log2; /* 0 = 28; largest intermediate tensor (complex64 entries) a plan may create */
  int32_t flags;                 /* TN_PLAN_* bits */
  uint64_t seed;                 /* planner tie-break seed */
  int64_t amp_batch;             /* TN_PLAN_NETWORK: bitstrings per call (power of two), else 0 */
  int64_t order_trials;          /* TN_PLAN_NETWORK: contraction orders tried per search: 0 = 256 (randomised
                                  * greedy, qubit-sweep and fold-first trials); 1 = the deterministic greedy
                                  * alone; otherwise 4..4096 */
  int64_t order_search;          /* TN_PLAN_NETWORK: 0 = the fixed mix of trials above; 1 = adaptive search
                                  * (a cross-entropy hyper-optimiser over the trial kind, noise temperature and
                                  * bitstring-index weight, refitted each round to the best quarter so far) */
  int64_t block_qubits;          /* TN_PLAN_BLOCKS: qubits per block k (6 or 7); 0 = 6 */
  int64_t reserved[2];           /* must be zero */
} tn_plan_opts;

/* Plan summary (for measurement and tests). */
typedef struct {
  int32_t n_qubits;
  int32_t n_params;
  int64_t n_gates;
  int32_t n_passes;     /* launches of the fused gate-apply kernel per contraction */
  int32_t n_phases;     /* register remappings summed over passes */
  int64_t n_ops;        /* register-level gate operations over all phases */
  int32_t tile_qubits;  /* qubits per on-chip tile */
  int32_t reg_qubits;   /* qubits held in registers per thread during a phase */
  double hbm_bytes;     /* algorithmic HBM bytes of one tn_contract_state call (per batch element) */
  double flops;         /* algorithmic FP32 flops of one tn_contract_state call (per batch element) */
  int32_t n_bwd_passes; /* passes of the adjoint sweep */
  int32_t specialized;  /* 1 if the forward passes run plan-specialised kernels */
  int32_t net_merges;   /* TN_PLAN_NETWORK: merges launched per call (one batched GEMM each) */
  int32_t net_max_log2; /* TN_PLAN_NETWORK: log2 entries of the largest intermediate */
  int32_t net_tensor_merges; /* TN_PLAN_NETWORK: launched merges whose GEMM runs on the tensor cores */
  int32_t net_folded_merges; /* TN_PLAN_NETWORK: bitstring-independent merges evaluated at plan time (FP64) */
  double bwd_flops;     /* TN_TARGET_EXPECTATION: algorithmic FP32 flops of the adjoint sweep per batch element
                           (every op on psi and lambda, derivative products and dots) */
  int32_t net_sliced;   /* TN_PLAN_NETWORK: sliced indices (each pass contracts 2^net_sliced slices and sums
                           them in FP64); 0 when an order within max_intermediate_log2 exists */
  int32_t net_batch_log2; /* TN_PLAN_NETWORK: log2 bitstrings contracted together; a call of up to amp_batch
                             bitstrings runs in passes of 2^net_batch_log2 (fewer than amp_batch when that
                             is the cheaper way to keep intermediates within max_intermediate_log2) */
  double net_cost;      /* TN_PLAN_NETWORK: the planner's cost of one call of amp_batch bitstrings, in bytes:
                           sum over launched merges (all slices and passes) of a fixed 2e7 per launch plus
                           max(bytes read and written, complex flops / 32) */
  double net_bytes;     /* TN_PLAN_NETWORK: algorithmic HBM bytes of one call of amp_batch bitstrings: every
                           launched merge's operands read and result written once (complex64) */
  int32_t n_fused;      /* dense 4x4 blocks (precontracted runs of gates on two qubits) in the forward passes;
                           TN_PLAN_BLOCKS: the 2^k x 2^k blocks (n_passes = GEMM launches = blocks - 1) */
  int32_t reserved_stats;
} tn_plan_stats;

/* Pauli sum H = sum_t coef[t] * P_t (host memory, read during tn_build_observable only).
 *   paulis[t * n_qubits + q] in {0 = I, 1 = X, 2 = Y, 3 = Z} is the factor on qubit q. */
typedef struct {
  int32_t n_terms;
  const double *coef;
  const uint8_t *paulis;
} tn_pauli_sum;

/* ---------------------------------------------------------------------------------------
 * Network construction and planning (host; not hot).
 * ------------------------------------------------------------------------------------- */

/* Build the network of an n_qubits circuit (Sec. 2.2.2: gate tensors joined to the
 * register's input legs |init_basis>).  gates[0..n_gates) in time order, host memory.
 * Returns TN_ERR_INVALID_ARG for n_qubits outside [1, 63] (plans other than TN_PLAN_NETWORK
 * accept at most 34), a bad kind or qubit, equal
 * qubits of a two-qubit gate, a parameter index on a fixed kind, init_basis >= 2^n. */
tn_status tn_build_from_circuit(int32_t n_qubits, const tn_gate *gates, int64_t n_gates,
                                uint64_t init_basis, tn_circuit **out);
/* Number of float64 parameters per batch element the circuit reads (max param_idx + arity). */
tn_status tn_circuit_num_params(const tn_circuit *c, int32_t *n_params);
void tn_free_circuit(tn_circuit *c);

/* Plan the contraction (Sec. 2.2.3 / Sec. 3: the order is chosen ahead of evaluation):
 * groups the gates into passes of the fused gate-apply kernel, and within a pass into
 * register phases, honouring every gate's dependencies; also plans the adjoint sweep.
 * Allocates and uploads the plan's device tables on the current CUDA device unless
 * opts->flags has TN_PLAN_HOST_ONLY.  opts may be NULL (defaults). */
tn_status tn_plan_contraction(const tn_circuit *c, const tn_plan_opts *opts, tn_plan **out);
/* Tile autotuner of one plan (the paper fixes the contraction order before evaluation, Sec.
 * 2.2.3; the tile size -- qubits per on-chip tile, which decides passes, phases and the generated
 * kernels -- is left to the implementation and chosen here by measurement).  Plans the circuit
 * with opts at every candidate tile size (tune->candidates, 0-terminated, each in [6, 13]; all
 * zero = {10, 11, 12, 13}; opts->tile_qubits must be 0; not for network, Q4.28, block or host-only
 * plans), times each plan's tn_contract_state on s (one warm-up call, the fastest of tune->reps
 * calls, 0 = 3; CUDA events; all parameters zero) and returns the fastest plan in *out (the others
 * are freed) and its tile size in *tile_out (optional).  Blocking: allocates and frees its own
 * scratch device memory (a state, a workspace, zero parameters), synchronises s.  tune may be
 * NULL; tune->flags and reserved must be zero. */
typedef struct tn_tune_opts tn_tune_opts;
tn_status tn_plan_contraction_tuned(const tn_circuit *c, const tn_plan_opts *opts, const tn_tune_opts *tune,
                                   tn_stream_t s, tn_plan **out, int32_t *tile_out);
/* Device workspace (bytes) that every contraction call of this plan needs. */
tn_status tn_plan_workspace_bytes(const tn_plan *p, size_t *bytes);
tn_status tn_plan_get_stats(const tn_plan *p, tn_plan_stats *stats);
void tn_free_plan(tn_plan *p);

/* Prepare a Pauli-sum observable on n_qubits (uploads its reduction tables). */
tn_status tn_build_observable(int32_t n_qubits, const tn_pauli_sum *H, tn_observable **out);
void tn_free_observable(tn_observable *o);

/* ---------------------------------------------------------------------------------------
 * Contraction (device; asynchronous on stream s).
 * ------------------------------------------------------------------------------------- */

/* Full state: state_dev[b] = U_G(theta_b) ... U_1(theta_b) |init_basis>, b < batch
 * (Sec. 2.2.2, Eq. 2.3: every output leg left open).
 *   params_dev     float64 [batch][n_params] device, or NULL when n_params == 0
 *   state_dev      complex64 [batch][2^N] device, written (no input contents needed)
 *   workspace_dev  >= tn_plan_workspace_bytes device bytes, or NULL when that is 0 */
tn_status tn_contract_state(const tn_plan *p, const double *params_dev, void *state_dev,
                            void *workspace_dev, tn_stream_t s);

/* Fixed-point emulation of the paper's datapath (Sec. 3: complex arithmetic in 32-bit fixed point
 * with 28 bits behind the binary point).  p: a plan built with TN_PLAN_Q428.  state_dev: int32
 * [2^N][2] (re, im), device memory owned by the caller; on return (stream-ordered) it holds the
 * circuit applied to |init_basis>, every value q meaning q / 2^28.  Arithmetic: each gate matrix
 * is quantised once, Uq = floor(U 2^28 + 1/2) (FP64, then saturated to int32); each gate is applied
 * once, every output component being the exact integer sum of Uq[i][k] psi[k] (64-bit) rounded
 * half up to Q4.28 ((acc + 2^27) >> 28) and saturated to int32.  Exact for unitary gates on states
 * of norm <= 1 (every sum below 2^60).  Returns TN_ERR_INVALID_ARG for a NULL pointer or a plan
 * not built with TN_PLAN_Q428; needs no workspace. */
tn_status tn_contract_state_q428(const tn_plan *p, int32_t *state_dev, tn_stream_t s);

/* Single amplitudes <x_i| C |init_basis> (Sec. 2.2.3: output legs closed by basis states).
 *   bitstrings_dev uint64 [n_bitstrings] device (bit N-1-q = qubit q), each < 2^N
 *   amps_dev       complex64 [batch][n_bitstrings] device, written
 * The batch of parameter sets and the batch of bitstrings are independent. */
tn_status tn_contract_amplitudes(const tn_plan *p, const double *params_dev,
                                 const uint64_t *bitstrings_dev, int64_t n_bitstrings,
                                 void *amps_dev, void *workspace_dev, tn_stream_t s);

/* Expectation values out_dev[b] = <psi_b| H |psi_b> (float64 [batch], device), where
 * psi_b is the contracted state; the final reduction accumulates in FP64. */
tn_status tn_expectation(const tn_plan *p, const tn_observable *H, const double *params_dev,
                         double *out_dev, void *workspace_dev, tn_stream_t s);

/* Adjoint gradient: grad_params_dev[b][k] = grad_out_dev[b] * d<H>_b / d theta_{b,k}
 * (float64, device; overwritten).  Recomputes the forward state, forms lambda = H psi and
 * sweeps the gates in reverse (psi <- U^dagger psi, g += 2 Re <lambda| dU |psi>,
 * lambda <- U^dagger lambda).  grad_out_dev may be NULL (treated as all ones). */
tn_status tn_expectation_backward(const tn_plan *p, const tn_observable *H, const double *params_dev,
                                  const double *grad_out_dev, double *grad_params_dev,
                                  void *workspace_dev, tn_stream_t s);

/* Value and gradient in one sweep: out_dev[b] = <psi_b| H |psi_b> and grad_params_dev[b][k] =
 * d<H>_b / d theta_{b,k} (float64, device; both overwritten).  The same work as tn_expectation
 * followed by tn_expectation_backward with grad_out = 1, but the forward state is contracted once,
 * and the energy is summed as Re <psi|lambda> while lambda = H psi is formed (its last pass),
 * before the reverse sweep un-computes psi in place.  A circuit without parameters takes the
 * plain reduction of tn_expectation. */
tn_status tn_expectation_value_and_grad(const tn_plan *p, const tn_observable *H, const double *params_dev,
                                        double *out_dev, double *grad_params_dev, void *workspace_dev,
                                        tn_stream_t s);

/* ---------------------------------------------------------------------------------------
 * Kernels exposed on their own (composable; used for measurement).
 * ------------------------------------------------------------------------------------- */

/* <psi_b| H |psi_b> for given states (complex64 [batch][2^N] device) into out_dev
 * (float64 [batch] device).  Partial sums go to workspace_dev, which must hold
 * tn_state_expectation_workspace_bytes(...) bytes. */
tn_status tn_state_expectation_workspace_bytes(const tn_observable *H, int32_t batch, size_t *bytes);
tn_status tn_state_expectation(const tn_observable *H, int32_t batch, const void *state_dev,
                               double *out_dev, void *workspace_dev, size_t workspace_bytes,
                               tn_stream_t s);

/* The reduction of tn_state_expectation for callers that cannot provide a workspace (the
 * paper has no counterpart; this is a deployment variant).  Such callers either have all of
 * their device memory owned by another allocator with a fixed budget, or run where a
 * cudaMalloc would implicitly synchronise the device.  The partial sums go to a 1 MiB array
 * compiled into the library (held on every GPU that loads it until the process exits):
 *   - requests needing more than 131072 partial sums (batch x reduction passes x 512) fail
 *     with TN_ERR_INVALID_ARG, and nothing is enqueued;
 *   - all calls on a device share the array; each clears the slots it uses, but calls that
 *     overlap on the GPU (unordered streams) race on it;
 *   - every call looks up the array's address on the current device (cudaGetSymbolAddress;
 *     nothing is cached across calls, so it stays valid after cudaDeviceReset); the first
 *     lookup on a device loads the library's module there, so make the first call on each
 *     device before any stream capture begins.
 * Allocates no device memory.  Other arguments and results as tn_state_expectation. */
tn_status tn_state_expectation_noalloc(const tn_observable *H, int32_t batch, const void *state_dev,
                                       double *out_dev, tn_stream_t s);

/* Index permutation over binary legs (Sec. 3: operands regrouped into matrices before a
 * merge): for a tensor of n_legs legs of size 2 (leg 0 most significant), out has legs
 * ordered perm[0..n_legs): out leg j is in leg perm[j].  complex64, batch independent
 * tensors back to back; in_dev and out_dev must not overlap; 1 <= n_legs <= 34. */
tn_status tn_permute(int32_t n_legs, const int32_t *perm, int64_t batch, const void *in_dev,
                     void *out_dev, tn_stream_t s);

/* Batched complex GEMM (Sec. 2.2.1, Eq. 2.2: a pairwise merge as a sum over shared indices):
 *   C[b][m][n] = sum_k A[b][m][k] * B[b][n][k]   (both operands K-contiguous)
 * complex64 interleaved, row-major; precision is a tn_precision.  workspace_dev must hold
 * tn_cgemm_workspace_bytes(...) bytes (split operand copies; may be 0). */
tn_status tn_cgemm_workspace_bytes(int32_t precision, int64_t batch, int64_t M, int64_t N, int64_t K,
                                   size_t *bytes);
tn_status tn_cgemm_batched(int32_t precision, int64_t batch, int64_t M, int64_t N, int64_t K,
                           const void *A_dev, const void *B_dev, void *C_dev, void *workspace_dev,
                           size_t workspace_bytes, tn_stream_t s);

/* ---------------------------------------------------------------------------------------
 * Batched execution: the contractions of many circuits of uneven size in one persistent
 * launch (work items = (circuit, pass, tile), claimed in pass-major order; a tile waits,
 * bounded, until the previous pass of its circuit is complete).  Sec. 2.2.3 / Sec. 3: each
 * circuit's contraction order is its plan; the batch only interleaves independent circuits.
 * ------------------------------------------------------------------------------------- */
typedef struct tn_batch tn_batch; /* opaque, library-owned, holds device tables */

/* Group plans (batch 1, any target, tile qubits in [6, 12]) for one launch.  The plans must
 * outlive the batch.  TN_ERR_UNSUPPORTED for plans of batch > 1.  Plans of circuits that read
 * parameters are allowed: their gate tables are built in the run (tn_batch_run_params).
 * Plans of 19 qubits and more that carry generated kernels (built without TN_PLAN_NO_SPECIALIZE;
 * any tile size) are not interpreted by the persistent kernel: a run launches their own pass
 * kernels on the batch's four side streams, beside it.  The entries of one parameterised plan
 * share a side stream (its per-call tables are rewritten before each pass); such a plan must not
 * run on another stream while the batch runs. */
tn_status tn_batch_build(const tn_plan *const *plans, int32_t n_plans, tn_batch **out);
/* complex64 entries of the output buffer (all states, each 16-byte aligned) and workspace bytes. */
tn_status tn_batch_sizes(const tn_batch *b, int64_t *state_elems, size_t *workspace_bytes);
/* offsets[i] = first complex64 entry of circuit i's state in the output buffer. */
tn_status tn_batch_state_offsets(const tn_batch *b, int64_t *offsets);
/* Contract every circuit: states_dev receives all final states.  Enqueues one memset of the
 * workspace (its counters) and one kernel launch on s, and, for the batch's wide circuits of
 * generated kernels, their pass launches on the side streams, which wait for s before they start
 * and which s waits for after the launch (a fork and a join of events: capturable in a CUDA graph,
 * where they become parallel branches).  A wait that runs out (about 2 s) is reported by
 * tn_sync_status as TN_ERR_TIMEOUT. */
tn_status tn_batch_run(const tn_batch *b, void *states_dev, void *workspace_dev, tn_stream_t s);
/* As tn_batch_run, for batches with parameterised circuits (spec: many parameter sets in
 * one persistent launch; Sec. 2.2.3: the order is fixed ahead of the values).  params_dev
 * (device, float64) holds every circuit's parameters back to back, circuit i's first at
 * param_offsets[i] of tn_batch_params; NULL allowed when no circuit reads any.  Enqueues one
 * memset, one kernel that builds all parameterised circuits' gate tables into the workspace
 * (FP64 angles, complex64 entries), and the persistent launch; capturable in a CUDA graph. */
tn_status tn_batch_run_params(const tn_batch *b, const double *params_dev, void *states_dev, void *workspace_dev,
                              tn_stream_t s);
/* *n_params = parameters of all circuits together; param_offsets (optional, one per circuit)
 * receives each circuit's first parameter in params_dev. */
tn_status tn_batch_params(const tn_batch *b, int32_t *n_params, int64_t *param_offsets);
void tn_free_batch(tn_batch *b);
/* Testing aid for the failure path (the paper has no counterpart).  Makes the tiles of work-list
 * pass `pass` (1 <= pass < that circuit's passes in the batch; a circuit that fits one tile has
 * one) of circuit `circ` wait for one more completed tile of the previous pass than exists, and
 * bounds every dependency wait of later runs by wait_limit_ns (in [1e6, 1e10]).  The next
 * tn_batch_run then gives up after that bound: the kernel returns, the states are incomplete, and
 * tn_sync_status reports TN_ERR_TIMEOUT.  circ = -1 restores the table and the default bound
 * (about 2 s).  Blocking (one small host-to-device copy); not to be called while a run of this
 * batch is in flight. */
tn_status tn_batch_test_stall(tn_batch *b, int32_t circ, int32_t pass, int64_t wait_limit_ns);

/* Tile autotuner (the paper fixes the contraction order ahead of evaluation, Sec. 2.2.3 /
 * Sec. 3; how a plan is cut into tiles is left to the implementation and chosen here by
 * measurement).  Plans every circuit (fixed angles, 1..34 qubits) for the batched executor
 * and picks each circuit's tile size (qubits per tile) from candidates: circuits are grouped
 * by qubit count, classes are visited in order of decreasing work, and each candidate is
 * timed by launching the whole batch (1 warm-up + reps timed launches, CUDA events on s, the
 * fastest kept).  Blocking: allocates and frees its own scratch device memory, synchronises s.
 * *out receives a batch that owns its plans (tn_free_batch frees them); tiles_out (optional,
 * n_circuits entries) receives the chosen tile sizes.  A circuit of n <= 12 qubits may also run
 * as one tile (T = n).  Candidates here: tile sizes in [6, 12]; all zero = {8, 9, 10, 11, 12}.
 * Circuits of 19 qubits and more are not tuned: they are planned with generated kernels at the
 * default tile size (compiled on a pool of host threads) and run on the side streams, as in
 * tn_batch_build; they take part in every timed launch. */
struct tn_tune_opts {
  int32_t candidates[8]; /* tile sizes, 0-terminated; all zero = the tuner's default set */
  int32_t reps;          /* timed launches per candidate; 0 = 3 */
  int32_t flags;         /* must be 0 */
  int64_t reserved[4];   /* must be 0 */
};
tn_status tn_batch_build_tuned(const tn_circuit *const *circuits, int32_t n_circuits, const tn_tune_opts *opts,
                               tn_stream_t s, tn_batch **out, int32_t *tiles_out);

/* ---------------------------------------------------------------------------------------
 * Status.
 * ------------------------------------------------------------------------------------- */

/* Synchronise stream s, then read and clear this device's status word: TN_OK, or the
 * first device-side failure recorded since the last call (TN_ERR_TIMEOUT / TN_ERR_NUMERIC),
 * or TN_ERR_CUDA if the synchronisation itself failed. */
tn_status tn_sync_status(tn_stream_t s);
/* Measured FP32 multiply-add rate of the current device (the paper has no counterpart; the
 * roofline denominator of the kernels bound by FP32 arithmetic): a kernel of independent packed
 * FP32x2 multiply-add chains (fma.rn.f32x2, 4 flops per instruction and thread) on every SM at
 * full occupancy, timed with CUDA events over a few launches of tens of milliseconds each (on a
 * stream of its own, synchronised).  *tflops receives the best rate in TFLOP/s, *seconds
 * (optional) that launch's duration.  Blocking; allocates no device memory. */
tn_status tn_probe_fma_rate(double *tflops, double *seconds);
/* Message of the last failed call on this thread ("" if none).  Valid until the next call. */
const char *tn_last_error(void);
const char *tn_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TNQ_TN_H */
