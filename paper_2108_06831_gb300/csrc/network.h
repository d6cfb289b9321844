// Amplitudes by network contraction: host-side structures shared by the planner and the launcher.
#pragma once

#include <complex>
#include <string>
#include <vector>

#include "kernels.h"
#include "tnq_internal.h"

namespace tnq {

enum NodeKind { NODE_FIXED = 0, NODE_OUTPUT = 1 };

struct NetNode {
  int kind = NODE_FIXED;
  std::vector<int> legs;                   // labels, first leg most significant
  std::vector<std::complex<double>> data;  // NODE_FIXED: 2^(legs) entries
  int qubit = -1;                          // NODE_OUTPUT: closed qubit
  int group = 0;                           // largest qubit the node touches (sweep order)
  std::vector<std::complex<double>> rows;  // NODE_OUTPUT: [x][i] = (<x| M_q)_i, or [x][0] = <x|M_q|x0>
};

struct NetStep {
  int a = -1, b = -1, out = -1;  // tensor ids (initial nodes first, then step results)
  std::vector<int> batch, contr, out_legs;
};

// Lowered step: permutations of initial operands, one batched complex GEMM whose output is
// written in the leg order its consumer reads (out_map; identity for the last merge).
struct NetLaunch {
  int a_id, b_id, out_id;
  int a_bits, b_bits;                  // binary legs of the operands
  std::vector<int> perm_a, perm_b;     // tn_permute permutations (empty: already in place)
  long long batch, M, N, K;
  long long off_a, off_b, off_out;     // workspace offsets (complex64) of operands / result
  long long off_pa, off_pb;            // scratch for the permuted operands (-1: not needed)
  long long off_gemm_ws;               // bytes offset of the GEMM split workspace (-1: none)
  size_t gemm_ws_bytes;
  int precision;                       // tn_precision used for this merge
  OutMap out_map;                      // natural [batch][M][N] index -> stored index
};

struct NetPlan {
  int n = 0;
  int log2_batch = 0;
  std::vector<int> label_dim;  // bits per label (label 0 = bitstring index)
  std::vector<NetNode> nodes;
  std::vector<NetStep> steps;
  std::vector<std::vector<int>> all_legs;  // legs of every tensor id
  int max_log2 = 0;
  double flops = 0;  // 8 M N K summed over merges
  // lowering
  std::vector<NetLaunch> launches;
  std::vector<long long> tensor_off;  // workspace offset (complex64) of every tensor id; -1 = plan table
  long long fixed_elems = 0;          // complex64 entries of the fixed node table
  std::vector<long long> fixed_off;   // offset of each fixed node in that table
  size_t ws_bytes = 0;
  long long final_off = 0;
  // device copies
  void *d_fixed = nullptr;   // complex64 fixed node table
  void *d_outputs = nullptr; // output-node descriptors
  int n_outputs = 0;
};

tn_status build_network(const tn_circuit &c, int log2_batch, NetPlan &net, std::string &err);
tn_status plan_network(NetPlan &net, int max_log2, std::string &err);
tn_status lower_network(NetPlan &net, int precision, std::string &err);
tn_status upload_network(NetPlan &net, std::string &err);
cudaError_t run_network(const NetPlan &net, const uint64_t *bitstrings, long long n_bits, float2 *amps, void *ws,
                        cudaStream_t s);
void free_network(NetPlan &net);

}  // namespace tnq
