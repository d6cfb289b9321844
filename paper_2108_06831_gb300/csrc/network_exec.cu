// Amplitudes by network contraction: lowering of the planned merges to permutations and
// batched complex GEMMs, workspace layout, and the per-call launch sequence.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

#include "kernels.h"
#include "network.h"

namespace tnq {

namespace {

struct OutDesc {  // one output closure on the device
  float rows[8];  // (re, im) of rows[0..3]
  long long off;  // complex64 offset in the workspace
  int qubit;
  int has_leg;
};

// u_q^b[i] = rows[2 x_q^b + i] (or the scalar rows[2 x_q^b]); padded bitstrings get zeros.
__global__ void k_build_outputs(const OutDesc *__restrict__ outs, int n_out, const uint64_t *__restrict__ xs,
                                long long n_bits, long long B, int n_qubits, float2 *__restrict__ ws) {
  const long long total = (long long)n_out * B;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int o = (int)(i / B);
    const long long b = i % B;
    const OutDesc &d = outs[o];
    const int x = b < n_bits ? (int)((xs[b] >> (n_qubits - 1 - d.qubit)) & 1ull) : 0;
    const bool pad = b >= n_bits;
    if (d.has_leg) {
      for (int k = 0; k < 2; ++k) {
        const int r = 2 * x + k;
        ws[d.off + 2 * b + k] = pad ? make_float2(0.f, 0.f) : make_float2(d.rows[2 * r], d.rows[2 * r + 1]);
      }
    } else {
      const int r = 2 * x;
      ws[d.off + b] = pad ? make_float2(0.f, 0.f) : make_float2(d.rows[2 * r], d.rows[2 * r + 1]);
    }
  }
}

struct Allocator {
  std::vector<std::pair<size_t, size_t>> free_;  // (offset, size), sorted by offset
  size_t top = 0;
  size_t alloc(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    for (size_t i = 0; i < free_.size(); ++i)
      if (free_[i].second >= bytes) {
        const size_t off = free_[i].first;
        free_[i].first += bytes;
        free_[i].second -= bytes;
        if (free_[i].second == 0) free_.erase(free_.begin() + (long)i);
        return off;
      }
    const size_t off = top;
    top += bytes;
    return off;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    free_.push_back({off, bytes});
    std::sort(free_.begin(), free_.end());
    std::vector<std::pair<size_t, size_t>> m;
    for (auto &f : free_) {
      if (!m.empty() && m.back().first + m.back().second == f.first) m.back().second += f.second;
      else m.push_back(f);
    }
    free_ = m;
    if (!free_.empty() && free_.back().first + free_.back().second == top) {
      top = free_.back().first;
      free_.pop_back();
    }
  }
};

bool tc_ok(int precision, long long M, long long N, long long K) {
  if (precision == TN_PREC_FP32) return false;
  const long long kq = precision == TN_PREC_3XTF32 ? 16 : 32;
  return M % 128 == 0 && N % 64 == 0 && K % kq == 0;
}

}  // namespace

tn_status lower_network(NetPlan &net, int precision, std::string &err) {
  const int n_init = (int)net.nodes.size();
  const int n_tensors = n_init + (int)net.steps.size();
  auto bits_of = [&](const std::vector<int> &ls) {
    int b = 0;
    for (int x : ls) b += net.label_dim[(size_t)x];
    return b;
  };
  // binary expansion of a leg list: (label, sub-bit) pairs, most significant first
  auto expand = [&](const std::vector<int> &ls) {
    std::vector<std::pair<int, int>> e;
    for (int x : ls)
      for (int k = 0; k < net.label_dim[(size_t)x]; ++k) e.push_back({x, k});
    return e;
  };
  auto perm_to = [&](const std::vector<int> &src, const std::vector<int> &dst, std::vector<int> &perm) {
    const auto es = expand(src), ed = expand(dst);
    perm.assign(ed.size(), 0);
    bool ident = true;
    for (size_t j = 0; j < ed.size(); ++j) {
      const auto it = std::find(es.begin(), es.end(), ed[j]);
      perm[j] = (int)(it - es.begin());
      ident &= perm[j] == (int)j;
    }
    if (ident) perm.clear();
  };
  net.tensor_off.assign((size_t)n_tensors, -1);
  Allocator al;
  size_t hw = 0;  // high-water mark of the workspace
  std::vector<size_t> bytes_of((size_t)n_tensors, 0);
  for (int id = 0; id < n_tensors; ++id) bytes_of[(size_t)id] = (sizeof(float2) << bits_of(net.all_legs[(size_t)id]));
  // fixed nodes live in the plan's table, output closures in the workspace
  net.fixed_off.assign((size_t)n_init, -1);
  net.fixed_elems = 0;
  for (int id = 0; id < n_init; ++id) {
    const NetNode &nd = net.nodes[(size_t)id];
    if (nd.kind == NODE_FIXED) {
      net.fixed_off[(size_t)id] = net.fixed_elems;
      net.fixed_elems += ((long long)1 << bits_of(nd.legs));
      net.fixed_elems = (net.fixed_elems + 31) & ~31ll;
    } else {
      net.tensor_off[(size_t)id] = (long long)(al.alloc(bytes_of[(size_t)id]) / sizeof(float2));
      hw = std::max(hw, al.top);
    }
  }
  // Layouts, decided from the last merge back to the first.  Every intermediate has one
  // consumer, which fixes the leg order it reads ([batch][free][contracted]); the producing
  // merge then orders its own batch, row (M) and column (N) legs as they appear in that
  // target, so that its GEMM's output map is monotone within each group, and stores the
  // result directly in the target order (the permutation fused into the GEMM epilogue).
  // Within the contracted group, legs that the operand's producer computes as columns come
  // last: a producer tile (all N bits and the lowest 7 M bits) then lands in a contiguous
  // block of its output.  Only initial tensors are permuted by kernel (b).
  const size_t n_steps = net.steps.size();
  std::vector<int> producer((size_t)n_tensors, -1);
  for (size_t si = 0; si < n_steps; ++si) producer[(size_t)net.steps[si].out] = (int)si;
  auto in = [](const std::vector<int> &v, int x) { return std::find(v.begin(), v.end(), x) != v.end(); };
  auto free_of = [&](const NetStep &st, int id) {
    std::vector<int> f;
    for (int x : net.all_legs[(size_t)id])
      if (!in(st.batch, x) && !in(st.contr, x)) f.push_back(x);
    return f;
  };
  auto map_to = [&](const std::vector<int> &nat, const std::vector<int> &dst, OutMap &om) {
    const auto en = expand(nat), ed = expand(dst);
    const int nb = (int)en.size();
    om = OutMap();
    om.nbits = nb;
    bool ident = true;
    for (int i = 0; i < nb; ++i) {  // flat bit i is expansion entry nb - 1 - i (MSB first)
      const int j = (int)(std::find(ed.begin(), ed.end(), en[(size_t)(nb - 1 - i)]) - ed.begin());
      om.pos[i] = (uint8_t)(nb - 1 - j);
      ident &= om.pos[i] == i;
    }
    om.identity = ident ? 1 : 0;
  };
  // order legs by their position in a target order
  auto by_target = [&](std::vector<int> v, const std::vector<int> &tgt) {
    std::stable_sort(v.begin(), v.end(), [&](int x, int y) {
      return std::find(tgt.begin(), tgt.end(), x) < std::find(tgt.begin(), tgt.end(), y);
    });
    return v;
  };
  std::vector<std::vector<int>> target((size_t)n_tensors);
  net.launches.assign(n_steps, NetLaunch());
  for (size_t k = n_steps; k-- > 0;) {
    const NetStep &st = net.steps[k];
    NetLaunch &L = net.launches[k];
    L.a_id = st.a;
    L.b_id = st.b;
    L.out_id = st.out;
    const std::vector<int> &tgt = target[(size_t)st.out].empty() ? net.all_legs[(size_t)st.out] : target[(size_t)st.out];
    const std::vector<int> batch = by_target(st.batch, tgt);
    const std::vector<int> free_a = by_target(free_of(st, st.a), tgt);
    const std::vector<int> free_b = by_target(free_of(st, st.b), tgt);
    // contracted legs: those the producer of A (else of B) computes as columns go last
    std::vector<int> contr = st.contr;
    int pa = producer[(size_t)st.a] >= 0 ? producer[(size_t)st.a] : producer[(size_t)st.b];
    if (pa >= 0) {
      const NetStep &ps = net.steps[(size_t)pa];
      const std::vector<int> cols = free_of(ps, ps.b);
      std::stable_partition(contr.begin(), contr.end(), [&](int x) { return !in(cols, x); });
    }
    std::vector<int> ta = batch, tb = batch, gemm_out = batch;
    ta.insert(ta.end(), free_a.begin(), free_a.end());
    ta.insert(ta.end(), contr.begin(), contr.end());
    tb.insert(tb.end(), free_b.begin(), free_b.end());
    tb.insert(tb.end(), contr.begin(), contr.end());
    gemm_out.insert(gemm_out.end(), free_a.begin(), free_a.end());
    gemm_out.insert(gemm_out.end(), free_b.begin(), free_b.end());
    map_to(gemm_out, tgt, L.out_map);
    for (int side = 0; side < 2; ++side) {
      const int id = side ? st.b : st.a;
      const std::vector<int> &want = side ? tb : ta;
      if (producer[(size_t)id] >= 0) target[(size_t)id] = want;  // its producer stores it this way
      else perm_to(net.all_legs[(size_t)id], want, side ? L.perm_b : L.perm_a);
    }
    L.a_bits = bits_of(net.all_legs[(size_t)st.a]);
    L.b_bits = bits_of(net.all_legs[(size_t)st.b]);
    L.batch = 1ll << bits_of(batch);
    L.M = 1ll << bits_of(free_a);
    L.N = 1ll << bits_of(free_b);
    L.K = 1ll << bits_of(contr);
    L.precision = tc_ok(precision, L.M, L.N, L.K) ? precision : TN_PREC_FP32;
  }
  // workspace, in execution order (operands freed after their merge)
  for (size_t si = 0; si < n_steps; ++si) {
    const NetStep &st = net.steps[si];
    NetLaunch &L = net.launches[si];
    L.off_pa = L.perm_a.empty() ? -1 : (long long)(al.alloc(bytes_of[(size_t)st.a]) / sizeof(float2));
    L.off_pb = L.perm_b.empty() ? -1 : (long long)(al.alloc(bytes_of[(size_t)st.b]) / sizeof(float2));
    L.gemm_ws_bytes = cgemm_workspace(L.precision, L.batch, L.M, L.N, L.K);
    L.off_gemm_ws = L.gemm_ws_bytes ? (long long)al.alloc(L.gemm_ws_bytes) : -1;
    net.tensor_off[(size_t)st.out] = (long long)(al.alloc(bytes_of[(size_t)st.out]) / sizeof(float2));
    L.off_out = net.tensor_off[(size_t)st.out];
    hw = std::max(hw, al.top);
    L.off_a = net.tensor_off[(size_t)st.a];
    L.off_b = net.tensor_off[(size_t)st.b];
    if (L.off_pa >= 0) al.release((size_t)L.off_pa * sizeof(float2), bytes_of[(size_t)st.a]);
    if (L.off_pb >= 0) al.release((size_t)L.off_pb * sizeof(float2), bytes_of[(size_t)st.b]);
    if (L.off_gemm_ws >= 0) al.release((size_t)L.off_gemm_ws, L.gemm_ws_bytes);
    if (net.tensor_off[(size_t)st.a] >= 0) al.release((size_t)net.tensor_off[(size_t)st.a] * sizeof(float2), bytes_of[(size_t)st.a]);
    if (net.tensor_off[(size_t)st.b] >= 0) al.release((size_t)net.tensor_off[(size_t)st.b] * sizeof(float2), bytes_of[(size_t)st.b]);
  }
  if (getenv("TNQ_DEBUG_NET")) {  // diagnostic listing of the lowered merges (stderr)
    for (const NetLaunch &L : net.launches) {
      fprintf(stderr, "merge %d x %d -> %d: batch %lld M %lld N %lld K %lld prec %d perm %d/%d map %d gflop %.3f",
              L.a_id, L.b_id, L.out_id, L.batch, L.M, L.N, L.K, L.precision, (int)!L.perm_a.empty(),
              (int)!L.perm_b.empty(), (int)!L.out_map.identity, 8.0 * L.batch * L.M * L.N * L.K / 1e9);
      for (const auto *pv : {&L.perm_a, &L.perm_b}) {
        fprintf(stderr, " [");
        for (int v : *pv) fprintf(stderr, "%d ", v);
        fprintf(stderr, "]");
      }
      if (!L.out_map.identity) {  // stored bit of each natural bit, LSB first
        fprintf(stderr, " map{");
        for (int i = 0; i < L.out_map.nbits; ++i) fprintf(stderr, "%d ", (int)L.out_map.pos[i]);
        fprintf(stderr, "}");
      }
      fprintf(stderr, "\n");
    }
  }
  const int last = net.steps.empty() ? 0 : net.steps.back().out;
  if (net.all_legs[(size_t)last].size() != 1 || net.all_legs[(size_t)last][0] != 0) {
    err = "network contraction did not end in the bitstring index alone";
    return TN_ERR_UNSUPPORTED;
  }
  net.final_off = net.tensor_off[(size_t)last];
  net.ws_bytes = hw + 256;
  return TN_OK;
}

tn_status upload_network(NetPlan &net, std::string &err) {
  std::vector<float2> fixed((size_t)std::max<long long>(net.fixed_elems, 1), make_float2(0.f, 0.f));
  std::vector<OutDesc> outs;
  for (size_t id = 0; id < net.nodes.size(); ++id) {
    const NetNode &nd = net.nodes[id];
    if (nd.kind == NODE_FIXED) {
      for (size_t k = 0; k < nd.data.size(); ++k)
        fixed[(size_t)net.fixed_off[id] + k] = make_float2((float)nd.data[k].real(), (float)nd.data[k].imag());
    } else {
      OutDesc d;
      std::memset(&d, 0, sizeof(d));
      for (int k = 0; k < 4; ++k) {
        d.rows[2 * k] = (float)nd.rows[(size_t)k].real();
        d.rows[2 * k + 1] = (float)nd.rows[(size_t)k].imag();
      }
      d.off = net.tensor_off[id];
      d.qubit = nd.qubit;
      d.has_leg = nd.legs.size() == 2 ? 1 : 0;
      outs.push_back(d);
    }
  }
  net.n_outputs = (int)outs.size();
  cudaError_t e = cudaMalloc(&net.d_fixed, fixed.size() * sizeof(float2));
  if (e == cudaSuccess) e = cudaMemcpy(net.d_fixed, fixed.data(), fixed.size() * sizeof(float2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&net.d_outputs, std::max<size_t>(outs.size(), 1) * sizeof(OutDesc));
  if (e == cudaSuccess && !outs.empty())
    e = cudaMemcpy(net.d_outputs, outs.data(), outs.size() * sizeof(OutDesc), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    err = std::string("network tables: ") + cudaGetErrorString(e);
    return TN_ERR_OOM;
  }
  return TN_OK;
}

void free_network(NetPlan &net) {
  cudaFree(net.d_fixed);
  cudaFree(net.d_outputs);
  net.d_fixed = nullptr;
  net.d_outputs = nullptr;
}

cudaError_t run_network(const NetPlan &net, const uint64_t *bitstrings, long long n_bits, float2 *amps, void *ws,
                        cudaStream_t s) {
  const long long B = 1ll << net.log2_batch;
  float2 *w = static_cast<float2 *>(ws);
  const float2 *fixed = static_cast<const float2 *>(net.d_fixed);
  if (net.n_outputs > 0) {
    const long long total = (long long)net.n_outputs * B;
    k_build_outputs<<<(unsigned)std::min<long long>((total + 255) / 256, 65535), 256, 0, s>>>(
        static_cast<const OutDesc *>(net.d_outputs), net.n_outputs, bitstrings, n_bits, B, net.n, w);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int n_init = (int)net.nodes.size();
  auto ptr = [&](int id) -> const float2 * {
    if (id < n_init && net.nodes[(size_t)id].kind == NODE_FIXED) return fixed + net.fixed_off[(size_t)id];
    return w + net.tensor_off[(size_t)id];
  };
  for (const NetLaunch &L : net.launches) {
    const float2 *a = ptr(L.a_id), *b = ptr(L.b_id);
    if (!L.perm_a.empty()) {
      cudaError_t e = launch_permute(L.a_bits, L.perm_a.data(), 1, a, w + L.off_pa, s);
      if (e != cudaSuccess) return e;
      a = w + L.off_pa;
    }
    if (!L.perm_b.empty()) {
      cudaError_t e = launch_permute(L.b_bits, L.perm_b.data(), 1, b, w + L.off_pb, s);
      if (e != cudaSuccess) return e;
      b = w + L.off_pb;
    }
    void *gws = L.off_gemm_ws >= 0 ? static_cast<void *>(static_cast<char *>(ws) + L.off_gemm_ws) : nullptr;
    cudaError_t e =
        launch_cgemm(L.precision, L.batch, L.M, L.N, L.K, a, b, w + L.off_out, gws, L.gemm_ws_bytes, s, &L.out_map);
    if (e != cudaSuccess) return e;
  }
  return cudaMemcpyAsync(amps, w + net.final_off, sizeof(float2) * (size_t)n_bits, cudaMemcpyDeviceToDevice, s);
}

}  // namespace tnq
