// State contraction by uniform square blocks: host structures shared by the planner and the
// launcher (blocks.cpp, blocks_exec.cu).
//
// The paper deploys its contraction as products of square matrices of one size: it
// precontracts small tensors until every tensor is square and congruent (Sec. 3).  Here the
// circuit is cut into blocks of gates that act on k qubits each; every block is precontracted
// into one 2^k x 2^k unitary (per call, in FP64, from the parameters), and each block is
// applied to the state viewed as a [2^(N-k)] x [2^k] matrix, psi' = psi U^T, by the batched
// complex GEMM (kernel c) in the plan's precision -- one uniform GEMM shape for the whole
// circuit.  The GEMM's output map stores each result directly in the layout the next block
// reads (its k qubits as the lowest index bits), so no separate permutation pass runs.
#pragma once

#include <string>
#include <vector>

#include "kernels.h"
#include "tnq_internal.h"

namespace tnq {

// A gate of a block, its qubits named by their local bits in the block's 2^k index.
struct alignas(16) BlockGate {
  int32_t kind;
  int32_t la, lb;       // local bits of the gate's first / second qubit (lb = -1: one qubit)
  int32_t pidx[3][2];   // angle a = angle[a] + sum of params[pidx[a][k]] over pidx >= 0
  int32_t pad;
  double angle[3];
  double pad2;
  double mat[32];       // MAT1 / MAT2 entries (re, im)
};

struct BlockPlan {
  int k = 0;            // qubits per block: every block is a 2^k x 2^k matrix
  int n = 0;            // qubits of the state
  int batch = 1;        // parameter sets per call (a power of two)
  int precision = TN_PREC_FP32;
  uint64_t init = 0;
  std::vector<std::vector<int>> qubits;  // per block: the qubit at each local bit
  std::vector<int> gate_begin, gate_count;
  std::vector<BlockGate> gates;
  std::vector<OutMap> maps;              // per block i >= 1: its GEMM's natural index -> stored index
  std::vector<long long> init_pos;       // block 0 on the basis state: stored index of each output
  int init_local = 0;                    // block 0: local index of the basis state's bits
  int rounds = 0;                        // planner rounds (windows of k qubits at alternating offsets)
  int seeded = 0;                        // blocks seeded by a gate no window contains
  double flops = 0;                      // 8 M N K per GEMM, all GEMMs of one call (per batch element)
  double bytes = 0;                      // state read and written by every GEMM, plus the first block
  // workspace layout (bytes)
  size_t ws_mats = 0, ws_state = 0, ws_gemm = 0, ws_bytes = 0;
  size_t gemm_ws_bytes = 0;
  // device tables
  BlockGate *d_gates = nullptr;
  int *d_meta = nullptr;                 // per block: gate_begin, gate_count
  long long *d_init_pos = nullptr;
  float2 *d_fixed_mats = nullptr;        // fixed-angle circuits: the block matrices, built once
};

tn_status plan_blocks(const tn_circuit &c, int k, int batch, int precision, BlockPlan &bp, std::string &err);
// Workspace layout; device tables unless host_only (and, for fixed angles, the block matrices).
tn_status upload_blocks(BlockPlan &bp, bool host_only, bool param_dependent, std::string &err);
// The block matrices for every batch element (FP64 product of each block's gates, stored complex64).
cudaError_t build_block_mats(const BlockPlan &bp, const double *params, int n_params, float2 *mats, cudaStream_t s);
// state <- the circuit applied to |init> (batch elements back to back, canonical layout).
cudaError_t run_blocks(const BlockPlan &bp, const double *params, int n_params, float2 *state, void *ws,
                       cudaStream_t s);
void free_blocks(BlockPlan &bp);

}  // namespace tnq
