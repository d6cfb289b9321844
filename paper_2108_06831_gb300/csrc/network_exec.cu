// Amplitudes by network contraction: lowering of the planned merges to permutations and
// batched complex GEMMs, workspace layout, and the per-call launch sequence.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <utility>
#include <vector>
#include <complex>

#include "kernels.h"
#include "network.h"

namespace tnq {

namespace {

struct OutDesc {  // one output closure on the device
  float rows[8];  // (re, im) of rows[0..3]
  long long off;  // complex64 offset in the workspace
  int qubit;
  int has_leg;
  int trans;      // stored [leg][b] instead of [b][leg] (the order its merge reads)
  int slice_bit;  // the closed leg is sliced: its value is this bit of the slice number (else -1)
};

// u_q^b[i] = rows[2 x_q^b + i] (or the scalar rows[2 x_q^b]; with a sliced leg the scalar
// rows[2 x_q^b + v], v the leg's value in this slice); padded bitstrings get zeros.
__global__ void k_build_outputs(const OutDesc *__restrict__ outs, int n_out, const uint64_t *__restrict__ xs,
                                long long n_bits, long long B, int n_qubits, unsigned long long slice,
                                float2 *__restrict__ ws) {
  pdl_wait();
  pdl_trigger();
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
        ws[d.off + (d.trans ? k * B + b : 2 * b + k)] =
            pad ? make_float2(0.f, 0.f) : make_float2(d.rows[2 * r], d.rows[2 * r + 1]);
      }
    } else {
      const int r = 2 * x + (d.slice_bit >= 0 ? (int)((slice >> d.slice_bit) & 1ull) : 0);
      ws[d.off + b] = pad ? make_float2(0.f, 0.f) : make_float2(d.rows[2 * r], d.rows[2 * r + 1]);
    }
  }
}

// Slice sum (FP64): acc[b] (+)= x[b] for the amplitudes of one slice.
__global__ void k_slice_sum(double2 *__restrict__ acc, const float2 *__restrict__ x, long long n, int first) {
  pdl_wait();
  pdl_trigger();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 v = x[i];
    if (first) {
      acc[i] = make_double2((double)v.x, (double)v.y);
    } else {
      const double2 a = acc[i];
      acc[i] = make_double2(a.x + (double)v.x, a.y + (double)v.y);
    }
  }
}

__global__ void k_slice_store(float2 *__restrict__ amps, const double2 *__restrict__ acc, long long n) {
  pdl_wait();
  pdl_trigger();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 a = acc[i];
    amps[i] = make_float2((float)a.x, (float)a.y);
  }
}

// bits of s at the set positions of mask, packed (the index of a slice copy)
inline long long pack_bits(unsigned long long s, uint32_t mask) {
  long long r = 0;
  int k = 0;
  for (int p = 0; p < 32; ++p)
    if ((mask >> p) & 1u) r |= (long long)((s >> p) & 1ull) << k++;
  return r;
}
inline unsigned long long unpack_bits(long long c, uint32_t mask) {
  unsigned long long s = 0;
  int k = 0;
  for (int p = 0; p < 32; ++p)
    if ((mask >> p) & 1u) s |= (unsigned long long)((c >> k++) & 1) << p;
  return s;
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

// tensor-core shapes (kernel c): 128-row tiles, 128 real columns, 16-byte operand rows
bool tc_ok(int precision, long long M, long long N, long long K) {
  if (precision == TN_PREC_FP32) return false;
  return M % 128 == 0 && N % 64 == 0 && K % (precision == TN_PREC_3XTF32 ? 2 : 4) == 0;
}
// rows the tensor-core launch takes (its row tiles index the grid's y dimension)
bool tc_rows_ok(long long M) { return M / 128 <= 65535; }

}  // namespace

// Tensor of a folded merge, on the host in FP64: out (legs lo) = sum over contr of A (legs
// la) x B (legs lb); every leg binary, first leg most significant.
std::vector<std::complex<double>> contract_host(const std::vector<int> &la, const std::vector<std::complex<double>> &A,
                                                const std::vector<int> &lb, const std::vector<std::complex<double>> &B,
                                                const std::vector<int> &contr, const std::vector<int> &lo) {
  auto stride = [](const std::vector<int> &ls, int x) -> long long {
    for (size_t p = 0; p < ls.size(); ++p)
      if (ls[p] == x) return 1ll << (ls.size() - 1 - p);
    return 0;
  };
  const int no = (int)lo.size(), nc = (int)contr.size();
  std::vector<long long> ca(1ull << nc, 0), cb(1ull << nc, 0);
  for (long long c = 0; c < (1ll << nc); ++c)
    for (int p = 0; p < nc; ++p)
      if ((c >> (nc - 1 - p)) & 1) {
        ca[(size_t)c] += stride(la, contr[(size_t)p]);
        cb[(size_t)c] += stride(lb, contr[(size_t)p]);
      }
  std::vector<long long> sa((size_t)no), sb((size_t)no);
  for (int p = 0; p < no; ++p) {
    sa[(size_t)p] = stride(la, lo[(size_t)p]);
    sb[(size_t)p] = stride(lb, lo[(size_t)p]);
  }
  std::vector<std::complex<double>> out(1ull << no);
  for (long long o = 0; o < (1ll << no); ++o) {
    long long ao = 0, bo = 0;
    for (int p = 0; p < no; ++p)
      if ((o >> (no - 1 - p)) & 1) {
        ao += sa[(size_t)p];
        bo += sb[(size_t)p];
      }
    std::complex<double> acc = 0;
    for (long long c = 0; c < (1ll << nc); ++c) acc += A[(size_t)(ao + ca[(size_t)c])] * B[(size_t)(bo + cb[(size_t)c])];
    out[(size_t)o] = acc;
  }
  return out;
}

// The same tensor with its legs reordered from `from` to `to` (binary legs).
std::vector<std::complex<double>> reorder_host(const std::vector<std::complex<double>> &x, const std::vector<int> &from,
                                               const std::vector<int> &to) {
  const int n = (int)from.size();
  std::vector<long long> st((size_t)n);  // stride in `from` of the leg at position p of `to`
  for (int p = 0; p < n; ++p) {
    const int q = (int)(std::find(from.begin(), from.end(), to[(size_t)p]) - from.begin());
    st[(size_t)p] = 1ll << (n - 1 - q);
  }
  std::vector<std::complex<double>> y(x.size());
  for (long long o = 0; o < (1ll << n); ++o) {
    long long i = 0;
    for (int p = 0; p < n; ++p)
      if ((o >> (n - 1 - p)) & 1) i += st[(size_t)p];
    y[(size_t)o] = x[(size_t)i];
  }
  return y;
}

// A fixed node's data in one slice: sliced legs take their slice value, the others stay.
static std::vector<std::complex<double>> restrict_node(const NetPlan &net, const NetNode &nd, unsigned long long s) {
  const int nl = (int)nd.legs.size();
  long long fixed = 0;
  std::vector<long long> keep;
  for (int p = 0; p < nl; ++p) {
    const long long stride = 1ll << (nl - 1 - p);
    const auto it = std::find(net.slices.begin(), net.slices.end(), nd.legs[(size_t)p]);
    if (it == net.slices.end()) keep.push_back(stride);
    else if ((s >> (it - net.slices.begin())) & 1ull) fixed += stride;
  }
  const int nk = (int)keep.size();
  std::vector<std::complex<double>> out(1ull << nk);
  for (long long o = 0; o < (1ll << nk); ++o) {
    long long i = fixed;
    for (int p = 0; p < nk; ++p)
      if ((o >> (nk - 1 - p)) & 1) i += keep[(size_t)p];
    out[(size_t)o] = nd.data[(size_t)i];
  }
  return out;
}

tn_status lower_network(NetPlan &net, int precision, std::string &err) {
  const int n_init = (int)net.nodes.size();
  const size_t n_steps = net.steps.size();
  const int n_tensors = n_init + (int)n_steps;
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
  std::vector<int> producer((size_t)n_tensors, -1);
  for (size_t si = 0; si < n_steps; ++si) producer[(size_t)net.steps[si].out] = (int)si;

  // Slice dependence: a tensor's value depends on the slice bits of the sliced legs of the
  // nodes below it.
  net.slice_dep.assign((size_t)n_tensors, 0u);
  for (int id = 0; id < n_init; ++id)
    for (int x : net.nodes[(size_t)id].legs)
      for (size_t k = 0; k < net.slices.size(); ++k)
        if (net.slices[k] == x) net.slice_dep[(size_t)id] |= 1u << k;
  for (const NetStep &st : net.steps)
    net.slice_dep[(size_t)st.out] = net.slice_dep[(size_t)st.a] | net.slice_dep[(size_t)st.b];
  auto copies = [&](int id) { return 1ll << __builtin_popcount(net.slice_dep[(size_t)id]); };
  net.closures_sliced = false;
  for (int id = 0; id < n_init; ++id)
    net.closures_sliced |= net.nodes[(size_t)id].kind == NODE_OUTPUT && net.slice_dep[(size_t)id] != 0;

  // 1. Constant folding.  A tensor that does not depend on the bitstrings (the gate tensors
  // and every merge of two such tensors) is the same for every call: those merges are
  // evaluated once at plan time, in FP64 (one copy per slice it depends on), within a size
  // and work budget.  Here the merges are chosen; their values are computed with the table.
  std::vector<char> is_static((size_t)n_tensors, 0), folded(n_steps, 0);
  for (int id = 0; id < n_init; ++id) is_static[(size_t)id] = net.nodes[(size_t)id].kind == NODE_FIXED;
  double fold_work = 0;
  net.folded_merges = 0;
  for (size_t si = 0; si < n_steps; ++si) {
    const NetStep &st = net.steps[si];
    if (!is_static[(size_t)st.a] || !is_static[(size_t)st.b]) continue;
    const int ob = bits_of(net.all_legs[(size_t)st.out]), cb = bits_of(st.contr);
    const double work = std::ldexp(1.0, ob + cb) * (double)copies(st.out);
    if (ob > kFoldMaxLog2 || fold_work + work > kFoldMaxWork) continue;
    fold_work += work;
    is_static[(size_t)st.out] = 1;
    folded[si] = 1;
    ++net.folded_merges;
  }

  // 2. Layouts of the launched merges, from the last back to the first.  Every tensor has one
  // consumer, which fixes the leg order it reads ([batch][free][contracted]):
  //   - a launched merge's result is stored in that order by its own GEMM (output map); the
  //     producing merge orders its batch, row (M) and column (N) legs as they appear in the
  //     target, so the map is monotone within each group;
  //   - a static tensor is laid out in that order on the host before upload;
  //   - an output closure [b][leg] is built in either order by the closure kernel.
  // Within the contracted group, legs that the operand's producer computes as columns go
  // last: a producer tile (its N bits and 7 lowest M bits) then lands in few contiguous runs.
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
  auto by_target = [&](std::vector<int> v, const std::vector<int> &tgt) {
    std::stable_sort(v.begin(), v.end(), [&](int x, int y) {
      return std::find(tgt.begin(), tgt.end(), x) < std::find(tgt.begin(), tgt.end(), y);
    });
    return v;
  };
  std::vector<std::vector<int>> target((size_t)n_tensors);
  std::vector<int> launch_of(n_steps, -1);
  int n_launch = 0;
  for (size_t si = 0; si < n_steps; ++si)
    if (!folded[si]) launch_of[si] = n_launch++;
  net.launches.assign((size_t)n_launch, NetLaunch());
  std::vector<char> closure_trans((size_t)n_tensors, 0);
  for (size_t k = n_steps; k-- > 0;) {
    if (folded[k]) continue;
    const NetStep &st = net.steps[k];
    NetLaunch &L = net.launches[(size_t)launch_of[k]];
    L.a_id = st.a;
    L.b_id = st.b;
    L.out_id = st.out;
    const std::vector<int> &tgt = target[(size_t)st.out].empty() ? net.all_legs[(size_t)st.out] : target[(size_t)st.out];
    const std::vector<int> batch = by_target(st.batch, tgt);
    const std::vector<int> free_a = by_target(free_of(st, st.a), tgt);
    const std::vector<int> free_b = by_target(free_of(st, st.b), tgt);
    std::vector<int> contr = st.contr;
    int pa = producer[(size_t)st.a] >= 0 && !folded[(size_t)producer[(size_t)st.a]] ? producer[(size_t)st.a] : -1;
    if (pa < 0 && producer[(size_t)st.b] >= 0 && !folded[(size_t)producer[(size_t)st.b]]) pa = producer[(size_t)st.b];
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
      target[(size_t)id] = side ? tb : ta;
      if (id < n_init && !is_static[(size_t)id]) {  // output closure: [b][leg] or [leg][b]
        const std::vector<int> &w = target[(size_t)id];
        closure_trans[(size_t)id] = w.size() == 2 && w[0] != 0;
      }
    }
    L.batch = 1ll << bits_of(batch);
    L.M = 1ll << bits_of(free_a);
    L.N = 1ll << bits_of(free_b);
    L.K = 1ll << bits_of(contr);
    // The GEMM computes C = A B^T with both operands K-contiguous, so the transposed product
    // B A^T is the same kernel with the operands exchanged; its natural output index
    // (b N + n) M + m goes to the same stored positions.  Exchanged when the tiles then fit
    // the shape better: tensor-core tiles only after the exchange, or, on the CUDA cores, a
    // short row dimension against a long column one (slicing leaves such merges).
    const bool tc_as_is = tc_ok(precision, L.M, L.N, L.K), tc_swapped = tc_ok(precision, L.N, L.M, L.K) && tc_rows_ok(L.N);
    const bool swap = !tc_as_is && (tc_swapped || cgemm_fp32_tile_fill(L.N, L.M) > cgemm_fp32_tile_fill(L.M, L.N));
    if (swap) {
      const int lgm = bits_of(free_a), lgn = bits_of(free_b);
      OutMap t = L.out_map;
      t.identity = 1;
      for (int i = 0; i < L.out_map.nbits; ++i) {  // bit i of the exchanged product's index
        const int f = i < lgm ? lgn + i : (i < lgm + lgn ? i - lgm : i);
        t.pos[i] = L.out_map.pos[f];
        t.identity &= t.pos[i] == i;
      }
      L.out_map = t;
      std::swap(L.a_id, L.b_id);
      std::swap(L.M, L.N);
    }
    L.precision = tc_ok(precision, L.M, L.N, L.K) && tc_rows_ok(L.M) ? precision : TN_PREC_FP32;
  }

  // 3. The table of static operands of launched merges, each in the order its merge reads,
  // one copy per combination of the slice bits it depends on.
  std::map<std::pair<int, unsigned long long>, std::vector<std::complex<double>>> memo;
  std::vector<int> step_of((size_t)n_tensors, -1);
  for (size_t si = 0; si < n_steps; ++si) step_of[(size_t)net.steps[si].out] = (int)si;
  std::function<const std::vector<std::complex<double>> &(int, unsigned long long)> value =
      [&](int id, unsigned long long sl) -> const std::vector<std::complex<double>> & {
    sl &= net.slice_dep[(size_t)id];
    const auto key = std::make_pair(id, sl);
    auto it = memo.find(key);
    if (it != memo.end()) return it->second;
    std::vector<std::complex<double>> v;
    if (id < n_init) {
      v = restrict_node(net, net.nodes[(size_t)id], sl);
    } else {
      const NetStep &st = net.steps[(size_t)step_of[(size_t)id]];
      const std::vector<std::complex<double>> &A = value(st.a, sl);
      const std::vector<std::complex<double>> &Bv = value(st.b, sl);
      v = contract_host(net.all_legs[(size_t)st.a], A, net.all_legs[(size_t)st.b], Bv, st.contr,
                        net.all_legs[(size_t)st.out]);
    }
    return memo.emplace(key, std::move(v)).first->second;
  };
  net.table_off.assign((size_t)n_tensors, -1);
  net.table_stride.assign((size_t)n_tensors, 0);
  net.table_host.clear();
  for (const NetLaunch &L : net.launches)
    for (int id : {L.a_id, L.b_id}) {
      if (!is_static[(size_t)id]) continue;
      const long long entries = 1ll << bits_of(net.all_legs[(size_t)id]);
      const long long stride = (entries + 31) & ~31ll;  // 256-byte alignment
      if ((long long)net.table_host.size() + stride * copies(id) > kMaxTableEntries) {
        err = "the constant operands of all slices exceed 2^27 entries";
        return TN_ERR_UNSUPPORTED;
      }
      net.table_off[(size_t)id] = (long long)net.table_host.size();
      net.table_stride[(size_t)id] = stride;
      for (long long c = 0; c < copies(id); ++c) {
        const std::vector<std::complex<double>> d =
            reorder_host(value(id, unpack_bits(c, net.slice_dep[(size_t)id])), net.all_legs[(size_t)id],
                         target[(size_t)id]);
        net.table_host.insert(net.table_host.end(), d.begin(), d.end());
        net.table_host.resize((size_t)(net.table_off[(size_t)id] + (c + 1) * stride));
      }
      memo.clear();  // every tensor has one consumer: nothing below this operand is read again
    }

  // 4. Workspace, in execution order: output closures, then every launched result (operands
  // freed after their merge).
  net.tensor_off.assign((size_t)n_tensors, -1);
  net.closure_trans.assign(closure_trans.begin(), closure_trans.end());
  Allocator al;
  size_t hw = 0;
  auto bytes_of = [&](int id) { return sizeof(float2) << bits_of(net.all_legs[(size_t)id]); };
  for (int id = 0; id < n_init; ++id)
    if (!is_static[(size_t)id]) {
      net.tensor_off[(size_t)id] = (long long)(al.alloc(bytes_of(id)) / sizeof(float2));
      hw = std::max(hw, al.top);
    }
  for (NetLaunch &L : net.launches) {
    L.gemm_ws_bytes = cgemm_workspace(L.precision, L.batch, L.M, L.N, L.K);
    L.off_gemm_ws = L.gemm_ws_bytes ? (long long)al.alloc(L.gemm_ws_bytes) : -1;
    net.tensor_off[(size_t)L.out_id] = (long long)(al.alloc(bytes_of(L.out_id)) / sizeof(float2));
    L.off_out = net.tensor_off[(size_t)L.out_id];
    hw = std::max(hw, al.top);
    if (L.off_gemm_ws >= 0) al.release((size_t)L.off_gemm_ws, L.gemm_ws_bytes);
    for (int id : {L.a_id, L.b_id})
      if (net.tensor_off[(size_t)id] >= 0) al.release((size_t)net.tensor_off[(size_t)id] * sizeof(float2), bytes_of(id));
  }
  if (getenv("TNQ_DEBUG_NET")) {  // diagnostic listing of the lowered merges (stderr)
    fprintf(stderr, "folded %d of %zu merges; %zu sliced indices (output closures sliced: %d), constant table %zu entries\n",
            net.folded_merges, n_steps, net.slices.size(), (int)net.closures_sliced, net.table_host.size());
    for (const NetLaunch &L : net.launches) {
      fprintf(stderr, "merge %d x %d -> %d: batch %lld M %lld N %lld K %lld prec %d static %d/%d map %d gflop %.3f",
              L.a_id, L.b_id, L.out_id, L.batch, L.M, L.N, L.K, L.precision, (int)is_static[(size_t)L.a_id],
              (int)is_static[(size_t)L.b_id], (int)!L.out_map.identity, 8.0 * L.batch * L.M * L.N * L.K / 1e9);
      if (!L.out_map.identity) {  // stored bit of each natural bit, LSB first
        fprintf(stderr, " map{");
        for (int i = 0; i < L.out_map.nbits; ++i) fprintf(stderr, "%d ", (int)L.out_map.pos[i]);
        fprintf(stderr, "}");
      }
      fprintf(stderr, "\n");
    }
  }
  if (net.launches.empty() || net.all_legs[(size_t)net.launches.back().out_id].size() != 1 ||
      net.all_legs[(size_t)net.launches.back().out_id][0] != 0) {
    err = "network contraction did not end in the bitstring index alone";
    return TN_ERR_UNSUPPORTED;
  }
  net.final_off = net.tensor_off[(size_t)net.launches.back().out_id];
  // algorithmic flops of one call of 2^call_log2 bitstrings: the launched merges, per slice
  // and per pass of bitstrings (folded merges are plan-time work)
  double fl = 0, cost = 0, by = 0;
  for (const NetLaunch &L : net.launches) {
    const double f = 8.0 * (double)L.batch * (double)L.M * (double)L.N * (double)L.K;
    const double bytes = 8.0 * (double)L.batch * ((double)L.M * L.K + (double)L.N * L.K + (double)L.M * L.N);
    fl += f;
    by += bytes;
    cost += kLaunchBytes + std::max(bytes, f / kRidge);
  }
  const int rep = (int)net.slices.size() + net.call_log2 - net.log2_batch;  // log2 (slices x passes)
  net.flops = std::ldexp(fl, rep);
  net.cost = std::ldexp(cost, rep);
  net.bytes = std::ldexp(by, rep);
  net.off_acc = -1;
  if (!net.slices.empty()) {  // FP64 slice sum after the contraction's own workspace
    net.off_acc = (long long)((hw + 255) & ~(size_t)255);
    hw = (size_t)net.off_acc + (sizeof(double2) << net.log2_batch);
  }
  net.ws_bytes = hw + 256;
  return TN_OK;
}

tn_status upload_network(NetPlan &net, std::string &err) {
  std::vector<float2> table(std::max<size_t>(net.table_host.size(), 1), make_float2(0.f, 0.f));
  for (size_t k = 0; k < net.table_host.size(); ++k)
    table[k] = make_float2((float)net.table_host[k].real(), (float)net.table_host[k].imag());
  std::vector<OutDesc> outs;
  for (size_t id = 0; id < net.nodes.size(); ++id) {
    const NetNode &nd = net.nodes[id];
    if (nd.kind == NODE_FIXED || net.tensor_off[id] < 0) continue;
    OutDesc d;
    std::memset(&d, 0, sizeof(d));
    for (int k = 0; k < 4; ++k) {
      d.rows[2 * k] = (float)nd.rows[(size_t)k].real();
      d.rows[2 * k + 1] = (float)nd.rows[(size_t)k].imag();
    }
    d.off = net.tensor_off[id];
    d.qubit = nd.qubit;
    d.has_leg = net.all_legs[id].size() == 2 ? 1 : 0;  // legs of the (sliced) network
    d.trans = net.closure_trans[id] ? 1 : 0;
    d.slice_bit = -1;
    if (nd.legs.size() == 2)
      for (size_t k = 0; k < net.slices.size(); ++k)
        if (net.slices[k] == nd.legs[1]) d.slice_bit = (int)k;
    outs.push_back(d);
  }
  net.n_outputs = (int)outs.size();
  cudaError_t e = cudaMalloc(&net.d_fixed, table.size() * sizeof(float2));
  if (e == cudaSuccess) e = cudaMemcpy(net.d_fixed, table.data(), table.size() * sizeof(float2), cudaMemcpyHostToDevice);
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
  const unsigned long long n_slices = 1ull << net.slices.size();
  double2 *acc = net.off_acc >= 0 ? reinterpret_cast<double2 *>(static_cast<char *>(ws) + net.off_acc) : nullptr;
  // the call's bitstrings, B at a time
  for (long long c0 = 0; c0 < n_bits; c0 += B) {
    const long long nb = std::min(B, n_bits - c0);
    const uint64_t *xs = bitstrings + c0;
    const unsigned grid_b = (unsigned)std::min<long long>((nb + 255) / 256, 1024);
    for (unsigned long long sl = 0; sl < n_slices; ++sl) {
      // every slice: the closures' buffers are reused by later merges of the slice before
      if (net.n_outputs > 0) {
        const long long total = (long long)net.n_outputs * B;
        cudaError_t e = launch_pdl(k_build_outputs, dim3((unsigned)std::min<long long>((total + 255) / 256, 65535)),
                                   dim3(256), 0, s, static_cast<const OutDesc *>(net.d_outputs), net.n_outputs, xs, nb,
                                   B, net.n, sl, w);
        if (e != cudaSuccess) return e;
      }
      auto ptr = [&](int id) -> const float2 * {
        if (net.table_off[(size_t)id] >= 0)
          return fixed + net.table_off[(size_t)id] +
                 pack_bits(sl, net.slice_dep[(size_t)id]) * net.table_stride[(size_t)id];
        return w + net.tensor_off[(size_t)id];
      };
      for (const NetLaunch &L : net.launches) {
        void *gws = L.off_gemm_ws >= 0 ? static_cast<void *>(static_cast<char *>(ws) + L.off_gemm_ws) : nullptr;
        cudaError_t e = launch_cgemm(L.precision, L.batch, L.M, L.N, L.K, ptr(L.a_id), ptr(L.b_id), w + L.off_out,
                                     gws, L.gemm_ws_bytes, s, &L.out_map);
        if (e != cudaSuccess) return e;
      }
      if (acc) {
        cudaError_t e = launch_pdl(k_slice_sum, dim3(grid_b), dim3(256), 0, s, acc, (const float2 *)(w + net.final_off),
                                   nb, sl == 0 ? 1 : 0);
        if (e != cudaSuccess) return e;
      }
    }
    cudaError_t e;
    if (acc) {
      e = launch_pdl(k_slice_store, dim3(grid_b), dim3(256), 0, s, amps + c0, (const double2 *)acc, nb);
    } else {
      e = cudaMemcpyAsync(amps + c0, w + net.final_off, sizeof(float2) * (size_t)nb, cudaMemcpyDeviceToDevice, s);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace tnq
