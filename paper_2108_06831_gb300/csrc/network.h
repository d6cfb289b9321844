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

// Launched merge: one batched complex GEMM whose operands are already laid out as it reads
// them and whose output is written in the leg order its consumer reads (out_map; identity
// for the last merge).
struct NetLaunch {
  int a_id = -1, b_id = -1, out_id = -1;
  long long batch = 1, M = 1, N = 1, K = 1;
  long long off_out = -1;        // workspace offset (complex64) of the result
  long long off_gemm_ws = -1;    // bytes offset of the GEMM split workspace (-1: none)
  size_t gemm_ws_bytes = 0;
  int precision = TN_PREC_FP32;  // tn_precision used for this merge
  OutMap out_map;                // natural [batch][M][N] index -> stored index
};

// Constant folding budget (merges of bitstring-independent tensors evaluated at plan time).
constexpr int kFoldMaxLog2 = 20;       // largest folded result: 2^20 entries
constexpr double kFoldMaxWork = 2e8;   // complex multiply-adds over all folded merges (all slices)

// Order cost of a launched merge: kLaunchBytes (a launch and a short kernel, ~3 us of HBM time;
// charging the ~9 us measured per launch on sliced plans, 6e7, picked orders that ran the Fig. 3.1
// amplitude sweep 24% slower, 37.6 against 30.4 ms, and changed no capped 36-qubit plan)
// + max(bytes read and written, complex flops / kRidge): merges are HBM-bound unless their
// arithmetic intensity exceeds kRidge.
constexpr double kRidge = 32.0;
constexpr double kLaunchBytes = 2e7;

// Orders searched when the default search had to slice (plan_network's default is 256).
constexpr int kSlicedTrials = 1024;

// Slicing: at most 2^16 slices; the constant table of all slices at most 2^27 entries.
constexpr int kMaxSliceBits = 16;
constexpr long long kMaxTableEntries = 1ll << 27;

struct NetPlan {
  int n = 0;
  int log2_batch = 0;  // bitstrings contracted together (label 0 carries 2^log2_batch values)
  int call_log2 = 0;   // bitstrings a call may pass: 2^(call_log2 - log2_batch) passes of the network
  std::vector<int> label_dim;  // bits per label (label 0 = bitstring index)
  std::vector<NetNode> nodes;
  std::vector<NetStep> steps;
  std::vector<std::vector<int>> all_legs;  // legs of every tensor id
  int max_log2 = 0;   // largest intermediate of one slice
  double flops = 0;  // 8 batch M N K of the launched merges of one call (all slices and passes)
  double cost = 0;   // the same merges' fixed launch cost + max(bytes moved, flops / 32) (the order cost)
  double bytes = 0;  // the same merges' operands read and results written (complex64)
  // Slicing, when no order keeps every intermediate within the cap: the indices in `slices`
  // are fixed per slice (bit k of a slice number is the value of label slices[k]); a slice is
  // the network without those indices, and the amplitudes are the sum of all slices' results.
  std::vector<int> slices;
  std::vector<char> sliced;           // per label: 1 if sliced (the planner drops it from every tensor)
  std::vector<uint32_t> slice_dep;    // per tensor id: slice bits its value depends on
  // lowering
  std::vector<NetLaunch> launches;    // launched (bitstring-dependent) merges, in order
  int folded_merges = 0;              // merges evaluated at plan time
  std::vector<long long> tensor_off;  // workspace offset (complex64) of every tensor id, -1 if none
  std::vector<long long> table_off;   // offset in the static table (complex64), -1 if not there
  std::vector<long long> table_stride;  // entries between two slice copies of a static operand
  std::vector<std::complex<double>> table_host;  // static operands of launched merges, as read
  std::vector<char> closure_trans;    // output closure stored [leg][b]
  size_t ws_bytes = 0;
  long long final_off = 0;
  long long off_acc = -1;         // bytes offset of the FP64 slice sum (-1: one slice)
  bool closures_sliced = false;   // some output closure depends on the slice (diagnostic listing)
  // device copies
  void *d_fixed = nullptr;   // complex64 fixed node table
  void *d_outputs = nullptr; // output-node descriptors
  int n_outputs = 0;
};

tn_status build_network(const tn_circuit &c, int log2_batch, NetPlan &net, std::string &err);
tn_status plan_network(NetPlan &net, int max_log2, int order_trials, int order_search, std::string &err);
tn_status lower_network(NetPlan &net, int precision, std::string &err);
tn_status upload_network(NetPlan &net, std::string &err);
cudaError_t run_network(const NetPlan &net, const uint64_t *bitstrings, long long n_bits, float2 *amps, void *ws,
                        cudaStream_t s);
void free_network(NetPlan &net);

}  // namespace tnq
