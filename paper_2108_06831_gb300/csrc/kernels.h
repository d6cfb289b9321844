// Launchers of libtnq's CUDA kernels (host declarations).
#pragma once

#include <vector>

#include "tnq_internal.h"

namespace tnq {

int num_sms();  // SM count of the current device (cached per device)

#ifdef __CUDACC__
// Programmatic dependent launch (short kernels of the network path).  A kernel launched with
// launch_pdl may be scheduled while the previous kernel on its stream is still running; it calls
// pdl_wait() before it touches any memory (which returns once that kernel has completed and its
// stores are visible), then pdl_trigger() to let the next such kernel be scheduled in turn.  In a
// kernel launched the ordinary way both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}
// The same for a kernel known by address (generated kernels): args as for cudaLaunchKernel.
inline cudaError_t launch_pdl_func(const void *func, dim3 grid, dim3 block, void **args, size_t smem, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, func, args);
}
#endif

// Matrix tables: write the complex64 entries of every slot for each batch element.
cudaError_t launch_materialize(const MatSlot *d_slots, int n_slots, int n_fused_slots, const FusedMember *d_fused,
                               const double *params, int n_params, int batch, long long mstride, float2 *out,
                               cudaStream_t s);
// Reorders a slot table for launch_materialize (fused blocks first); returns their count.
int order_slots_fused_first(std::vector<MatSlot> &slots);

// Kernel (a): all forward passes of a plan (state <- U_G .. U_1 |init>).  Generated pass kernels
// are launched as programmatic dependents of the previous pass (pdl) unless the caller shares the
// GPU with other streams' work, where a pass waiting for its predecessor would hold SM resources.
cudaError_t launch_forward(const tn_plan *p, const float2 *mats, long long mstride, float2 *state, cudaStream_t s,
                           bool pdl = true);

// Adjoint sweep: psi, lambda swept back through the gates; grad[b][k] accumulated (FP64).
cudaError_t launch_backward(const tn_plan *p, const float2 *mats, long long mstride, float2 *psi, float2 *lam,
                            double *grad, cudaStream_t s);

// Pauli-sum reductions (tile passes).  part holds n_partials doubles per batch element.
size_t observable_partials(const tn_observable *o, int batch);
cudaError_t launch_expectation(const tn_observable *o, int batch, const float2 *state, double *part,
                               double *out, cudaStream_t s);
// lam = H psi (complex64); with out != NULL also out[b] = <psi|H|psi> (FP64), summed from the
// finished lam in the last pass (part: observable_partials(o, batch) doubles of scratch).
cudaError_t launch_apply_hamiltonian(const tn_observable *o, int batch, const float2 *psi, float2 *lam,
                                     cudaStream_t s, double *part = nullptr, double *out = nullptr);
// amps[b][i] = state[b][x_i]
cudaError_t launch_gather(const float2 *state, int N, int batch, const uint64_t *xs, long long nx, float2 *amps,
                          cudaStream_t s);
// grad[b][k] *= gout[b] (gout may be NULL -> no-op), zero-fill helper
cudaError_t launch_scale_grad(double *grad, const double *gout, int batch, int P, cudaStream_t s);
cudaError_t launch_zero(void *p, size_t bytes, cudaStream_t s);

// Kernel (b): permutation of binary legs.
cudaError_t launch_permute(int n_legs, const int32_t *perm, long long batch, const float2 *in, float2 *out,
                           cudaStream_t s);

// Kernel (c): batched complex GEMM C[b] = A[b] * B[b]^T (K-contiguous operands).
// Output map: with batch, M and N powers of two, element (b, m, n) has the natural flat index
// f = (b M + m) N + n; a non-identity map stores it at sum_i bit_i(f) << pos[i] instead, so a
// merge writes its result directly in the leg order its consumer reads (a permutation of
// binary legs fused into the epilogue).
struct OutMap {
  int identity = 1;
  int nbits = 0;
  uint8_t pos[64] = {};
};
size_t cgemm_workspace(int precision, long long batch, long long M, long long N, long long K);
// Fixed-point (Q4.28) state contraction: basis state, then every gate once (k_q428.cu).
int32_t q428_quantize(double x);
void q428_build(const tn_circuit &c, std::vector<Q428Gate> &out);
cudaError_t launch_q428(const std::vector<Q428Gate> &gates, int n, unsigned long long init, int32_t *state,
                        cudaStream_t s);
// Fraction of the FP32 GEMM's tile work that falls inside an M x N output (its tile choice).
double cgemm_fp32_tile_fill(long long M, long long N);
cudaError_t launch_cgemm(int precision, long long batch, long long M, long long N, long long K, const float2 *A,
                         const float2 *B, float2 *C, void *ws, size_t ws_bytes, cudaStream_t s,
                         const OutMap *om = nullptr);

// Persistent batched executor.  Circuits of at least kBatchDirectMinQubits qubits whose plans carry
// generated pass kernels run those kernels on side streams instead (at least 128 tiles per pass).
constexpr int kBatchDirectMinQubits = 19;
tn_status batch_build(const tn_plan *const *plans, int n, tn_batch **out);
// params: every parameterised circuit's parameters back to back (NULL when none has any).
cudaError_t batch_run(const tn_batch *b, const double *params, float2 *states, void *ws, cudaStream_t s);
// Parameters of all circuits together; offsets[i] (optional) = circuit i's first parameter.
int batch_num_params(const tn_batch *b, long long *offsets);
void batch_free(tn_batch *b);
tn_status batch_sizes(const tn_batch *b, long long *elems, size_t *ws);
tn_status batch_offsets(const tn_batch *b, long long *offsets);
int batch_device(const tn_batch *b);
tn_status batch_test_stall(tn_batch *b, int circ, int pass, long long wait_ns);
tn_status probe_fma_rate(double *tflops, double *seconds);
// The batch takes ownership of plans (freed with it).
void batch_adopt_plans(tn_batch *b, const std::vector<tn_plan *> &plans);
// Tile autotuner: plans every circuit at measured-best tile sizes and batches them.
tn_status batch_build_tuned(const tn_circuit *const *circuits, int n, const tn_tune_opts &o, cudaStream_t s,
                            tn_batch **out, int32_t *tiles_out);

// Tile autotuner of one plan: plans at each candidate tile size, times the forward contraction,
// returns the fastest plan (the others freed).
tn_status plan_tuned(const tn_circuit *c, const tn_plan_opts &base, const std::vector<int> &cands, int reps,
                     cudaStream_t s, tn_plan **out, int32_t *tile_out);

// Raise a kernel's dynamic shared-memory limit on the current device if `bytes` needs it.
cudaError_t ensure_smem(const void *func, size_t bytes);

// Device status word (timeouts, non-finite values).
void *status_word_ptr();
cudaError_t read_and_clear_status(int *value, cudaStream_t s);

}  // namespace tnq
