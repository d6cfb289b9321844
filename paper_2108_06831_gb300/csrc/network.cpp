// Amplitudes by contracting the circuit's tensor network (host side: network, order, lowering).
//
// Sec. 2.2.2-2.2.3: the state is the network of gate tensors joined to the input legs; an
// amplitude <x|C|x0> closes every output leg with a basis covector and contracts all
// indices; the order is a free choice made before evaluation.  Here:
//   - a qubit's world line is a chain of indices; consecutive one-qubit gates are multiplied
//     (FP64) into one 2x2 tensor, the input vector |x0_q> into the first one; diagonal
//     two-qubit gates (CZ, CP) leave both values unchanged, so they are rank-2 couplings on
//     the two current indices (hyperedges shared with the surrounding tensors), and other
//     two-qubit gates are tensors T[out_a, out_b, in_a, in_b];
//   - every output leg is closed by u_q^b = <x_q^b| M_q (M_q the qubit's trailing one-qubit
//     product), a [B x 2] tensor sharing the bitstring index b (a hyperedge over all outputs)
//     -- built on the device from the bitstrings at call time;
//   - the order is searched over seeded trials run on all host cores (greedy merging by size
//     reduction with Gumbel noise, qubit sweeps, fold-first), the cheapest kept by the cost
//     of one call (launches, bytes, flops; merges of bitstring-independent tensors are folded
//     at plan time and cost nothing per call); an index carried by more than the two merged
//     tensors (a hyperedge, e.g. the bitstring index) is a batch index of the merge;
//   - each merge is lowered to one batched complex GEMM (kernel c) whose operands are laid
//     out as it reads them;
//   - a call's bitstrings may be contracted in smaller passes (every pass size is searched);
//   - when no order keeps every intermediate within the cap, indices are sliced: each chosen
//     index is fixed to 0 and to 1 in turn, every slice is the network without it, and the
//     amplitudes are the sum over all slices (exact: the full contraction sums over that
//     index too).  Indices are picked greedily on every trial that exceeds the cap (the one
//     shrinking the most largest intermediates, then the most flops), and the sliced network
//     is planned again.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <queue>
#include <set>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "network.h"
#include "tnq_internal.h"

namespace tnq {

namespace {

using cd = std::complex<double>;

struct Mat2 {
  cd m[4];
};
Mat2 eye2() { return Mat2{{1.0, 0.0, 0.0, 1.0}}; }
Mat2 mul2(const Mat2 &a, const Mat2 &b) {  // a * b
  Mat2 r;
  r.m[0] = a.m[0] * b.m[0] + a.m[1] * b.m[2];
  r.m[1] = a.m[0] * b.m[1] + a.m[1] * b.m[3];
  r.m[2] = a.m[2] * b.m[0] + a.m[3] * b.m[2];
  r.m[3] = a.m[2] * b.m[1] + a.m[3] * b.m[3];
  return r;
}

void gate_mat(const TnGate &g, cd *out, int *dim) {
  double tmp[32];
  *dim = gate_matrix(g.kind, FORM_U, g.angle, g.mat, tmp);
  for (int i = 0; i < (*dim) * (*dim); ++i) out[i] = cd(tmp[2 * i], tmp[2 * i + 1]);
}

}  // namespace

bool is_diag2(int kind) { return kind == TN_GATE_CZ || kind == TN_GATE_CP; }

tn_status build_network(const tn_circuit &c, int log2_batch, NetPlan &net, std::string &err) {
  for (const TnGate &g : c.gates)
    if (g.param_idx >= 0) {
      err = "network contraction takes fixed-angle circuits";
      return TN_ERR_UNSUPPORTED;
    }
  const int n = c.n;
  net = NetPlan();
  net.n = n;
  net.log2_batch = log2_batch;
  net.call_log2 = log2_batch;
  net.label_dim.push_back(log2_batch);  // label 0: the bitstring index (2^log2_batch values)
  auto new_label = [&]() {
    net.label_dim.push_back(1);
    return (int)net.label_dim.size() - 1;
  };
  // World line of qubit q: label cur[q] carries the qubit's basis value from the last
  // non-diagonal gate on; one-qubit gates accumulate in pend[q] until something couples to
  // the value (a diagonal two-qubit gate) or the line ends.  While in_open[q], cur[q] is the
  // input leg and the input vector |x0_q> has not been placed yet.
  std::vector<int> cur((size_t)n);
  std::vector<char> in_open((size_t)n, 1);
  std::vector<Mat2> pend((size_t)n, eye2());
  std::vector<char> pend_id((size_t)n, 1);
  for (int q = 0; q < n; ++q) cur[(size_t)q] = new_label();
  auto bit0 = [&](int q) { return (int)((c.init >> (n - 1 - q)) & 1); };
  int cur_group = 0;  // qubit the node being added belongs to (the largest qubit it touches)
  auto add_fixed = [&](std::vector<int> legs, std::vector<cd> data) {
    NetNode nd;
    nd.kind = NODE_FIXED;
    nd.legs = std::move(legs);
    nd.data = std::move(data);
    nd.group = cur_group;
    net.nodes.push_back(std::move(nd));
  };
  // make cur[q] carry the value after pend[q] (a tensor U[out, in], or the vector U|x0>)
  auto flush = [&](int q) {
    if (in_open[(size_t)q]) {
      const Mat2 &M = pend[(size_t)q];
      const int x0 = bit0(q);
      const int l = cur[(size_t)q];
      add_fixed({l}, {M.m[0 + x0], M.m[2 + x0]});
      in_open[(size_t)q] = 0;
    } else if (!pend_id[(size_t)q]) {
      const int out = new_label();
      const Mat2 &M = pend[(size_t)q];
      add_fixed({out, cur[(size_t)q]}, {M.m[0], M.m[1], M.m[2], M.m[3]});
      cur[(size_t)q] = out;
    }
    pend[(size_t)q] = eye2();
    pend_id[(size_t)q] = 1;
  };
  for (const TnGate &g : c.gates) {
    cd U[16];
    int dim = 0;
    gate_mat(g, U, &dim);
    if (dim == 2) {
      Mat2 m{{U[0], U[1], U[2], U[3]}};
      pend[(size_t)g.q[0]] = mul2(m, pend[(size_t)g.q[0]]);
      pend_id[(size_t)g.q[0]] = 0;
      continue;
    }
    const int qa = g.q[0], qb = g.q[1];
    cur_group = qa;
    flush(qa);
    cur_group = qb;
    flush(qb);
    cur_group = std::max(qa, qb);
    if (is_diag2(g.kind)) {
      // diagonal: the two values pass through; the gate couples them, d[a][b] = U[ab][ab]
      add_fixed({cur[(size_t)qa], cur[(size_t)qb]}, {U[0], U[5], U[10], U[15]});
      continue;
    }
    const int oa = new_label(), ob = new_label();
    std::vector<cd> d(16);
    for (int i = 0; i < 16; ++i) d[(size_t)i] = U[i];  // legs (out_a, out_b, in_a, in_b)
    add_fixed({oa, ob, cur[(size_t)qa], cur[(size_t)qb]}, d);
    cur[(size_t)qa] = oa;
    cur[(size_t)qb] = ob;
  }
  // output closures: u_q^b = <x_q^b| M_q on the line's last value, or the scalar <x_q^b| M_q |x0_q>
  for (int q = 0; q < n; ++q) {
    NetNode node;
    node.kind = NODE_OUTPUT;
    node.qubit = q;
    node.group = q;
    const Mat2 &M = pend[(size_t)q];
    if (!in_open[(size_t)q]) {
      node.legs = {0, cur[(size_t)q]};
      node.rows = {M.m[0], M.m[1], M.m[2], M.m[3]};  // row x of M
    } else {
      const int i0 = bit0(q);
      node.legs = {0};
      node.rows = {M.m[0 + i0], 0.0, M.m[2 + i0], 0.0};  // <x|M|x0> for x = 0, 1
    }
    net.nodes.push_back(node);
  }
  return TN_OK;
}

namespace {

// Orders tried: per pass size (coarse), and at the chosen pass size.
constexpr int kCoarseTrials = 64;
constexpr int kTrials = 256;

struct Trial {
  std::vector<NetStep> steps;
  std::vector<std::vector<int>> legs;
  int max_log2 = 0;
  double flops = 0;      // of the merges that run on each call
  double fold_work = 0;  // complex multiply-adds of the merges folded at plan time
  // cost of the merges that run on each call (all but those folded at plan time): per merge
  // kLaunchBytes + max(bytes read and written, flops / kRidge), summed
  double dyn_cost = 0;
  // slicing of an order whose peak exceeds the cap: the indices, and the cost of all slices
  bool sliceable = false;
  std::vector<int> slices;
  double sliced_cost = 0, sliced_flops = 0;
};

// Contraction state shared by the order heuristics: live tensors, index ownership, steps.
struct Contractor {
  const NetPlan &net;
  std::vector<std::vector<int>> legs;
  std::vector<char> live;
  std::vector<std::vector<int>> where;  // label -> live tensors carrying it
  std::vector<char> stat;                 // tensor does not depend on the bitstrings
  Trial tr;
  explicit Contractor(const NetPlan &n) : net(n) {
    for (const NetNode &nd : net.nodes) {  // sliced indices are not part of any slice's network
      std::vector<int> l;
      for (int x : nd.legs)
        if (net.sliced.empty() || !net.sliced[(size_t)x]) l.push_back(x);
      legs.push_back(l);
    }
    live.assign(legs.size(), 1);
    where.resize(net.label_dim.size());
    for (const NetNode &nd : net.nodes) stat.push_back(nd.kind == NODE_FIXED ? 1 : 0);
    for (size_t i = 0; i < legs.size(); ++i)
      for (int x : legs[i]) where[x].push_back((int)i);
  }
  int bits_of(const std::vector<int> &ls) const {
    int b = 0;
    for (int x : ls) b += net.label_dim[(size_t)x];
    return b;
  }
  // bits the greedy scores a leg list with: the bitstring index may be weighted as if it were
  // larger (a small batch otherwise makes merging the output closures early look cheap)
  int score_bits0 = -1;
  int score_bits(const std::vector<int> &ls) const {
    int b = 0;
    for (int x : ls) b += (x == 0 && score_bits0 >= 0) ? score_bits0 : net.label_dim[(size_t)x];
    return b;
  }
  void merged(int i, int j, std::vector<int> &res, std::vector<int> &batch, std::vector<int> &contr) {
    res.clear();
    batch.clear();
    contr.clear();
    const std::vector<int> &li = legs[(size_t)i], &lj = legs[(size_t)j];
    for (int x : li) {
      if (std::find(lj.begin(), lj.end(), x) != lj.end()) {
        if (where[x].size() > 2 || x == 0) batch.push_back(x);
        else contr.push_back(x);
      } else {
        res.push_back(x);
      }
    }
    for (int x : lj)
      if (std::find(li.begin(), li.end(), x) == li.end()) res.push_back(x);
    res.insert(res.begin(), batch.begin(), batch.end());
  }
  int merge(int bi, int bj) {
    std::vector<int> res, batch, contr;
    merged(bi, bj, res, batch, contr);
    NetStep st;
    st.a = bi;
    st.b = bj;
    st.out = (int)legs.size();
    st.batch = batch;
    st.contr = contr;
    st.out_legs = res;
    tr.max_log2 = std::max(tr.max_log2, bits_of(res));
    int mb = 0, nb = 0;
    for (int x : legs[(size_t)bi])
      if (std::find(batch.begin(), batch.end(), x) == batch.end() && std::find(contr.begin(), contr.end(), x) == contr.end())
        mb += net.label_dim[(size_t)x];
    for (int x : legs[(size_t)bj])
      if (std::find(batch.begin(), batch.end(), x) == batch.end() && std::find(contr.begin(), contr.end(), x) == contr.end())
        nb += net.label_dim[(size_t)x];
    const double fl = 8.0 * std::ldexp(1.0, bits_of(batch) + mb + nb + bits_of(contr));
    // a merge of two bitstring-independent tensors is folded at plan time when it fits the
    // folding budget (the rule the lowering applies); every other merge runs on each call
    bool folded = false;
    if (stat[(size_t)bi] && stat[(size_t)bj]) {
      const double work = std::ldexp(1.0, bits_of(res) + bits_of(contr));
      if (bits_of(res) <= kFoldMaxLog2 && tr.fold_work + work <= kFoldMaxWork) {
        tr.fold_work += work;
        folded = true;
      }
    }
    if (!folded) {
      tr.flops += fl;
      tr.dyn_cost += kLaunchBytes + std::max(8.0 * (std::ldexp(1.0, bits_of(res)) +
                                                    std::ldexp(1.0, bits_of(legs[(size_t)bi])) +
                                                    std::ldexp(1.0, bits_of(legs[(size_t)bj]))),
                                             fl / kRidge);
    }
    const int out = (int)legs.size();
    for (int x : legs[(size_t)bi]) {
      auto &w = where[x];
      w.erase(std::remove(w.begin(), w.end(), bi), w.end());
    }
    for (int x : legs[(size_t)bj]) {
      auto &w = where[x];
      w.erase(std::remove(w.begin(), w.end(), bj), w.end());
    }
    for (int x : contr) where[(size_t)x].clear();
    legs.push_back(res);
    live.push_back(1);
    stat.push_back(folded ? 1 : 0);
    live[(size_t)bi] = live[(size_t)bj] = 0;
    for (int x : res) where[x].push_back(out);
    tr.steps.push_back(st);
    return out;
  }
  // Greedy by size reduction among live tensors whose flag is set in `allowed` (all if empty):
  // candidate pairs share an index other than the bitstring index; the pair minimising
  // (size(result) - size(A) - size(B)) / max(size(A), size(B)), less Gumbel noise of the given
  // temperature drawn when the pair is scored, is merged next.  Candidates live in a heap: a
  // merge only adds the pairs of its result (the score of a pair not involving the result
  // cannot change: an index's batch/contracted role changes only when two of its carriers
  // merge).  With fold_cap >= 0 only pairs of bitstring-independent tensors whose result
  // has at most 2^fold_cap entries are candidates (merges folded at plan time).
  void greedy(double temperature, uint64_t seed, const std::vector<char> &allowed_in, int fold_cap = -1) {
    uint64_t rs = seed * 6364136223846793005ull + 1442695040888963407ull;
    auto uniform = [&]() {
      rs = rs * 6364136223846793005ull + 1442695040888963407ull;
      return ((rs >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    struct Cand {
      double score, base;  // base: without noise
      int i, j;
      bool operator>(const Cand &o) const {
        return score > o.score || (score == o.score && (i > o.i || (i == o.i && j > o.j)));
      }
    };
    std::priority_queue<Cand, std::vector<Cand>, std::greater<Cand>> heap;
    std::vector<char> allowed = allowed_in;
    std::vector<int> res, batch, contr;
    auto ok = [&](int i) {
      return live[(size_t)i] && (allowed.empty() || allowed[(size_t)i]) && (fold_cap < 0 || stat[(size_t)i]);
    };
    auto push = [&](int i, int j) {
      if (i > j) std::swap(i, j);
      merged(i, j, res, batch, contr);
      if (fold_cap >= 0 && bits_of(res) > fold_cap) return;
      const double sr = std::ldexp(1.0, score_bits(res)), sa = std::ldexp(1.0, score_bits(legs[(size_t)i])),
                   sb = std::ldexp(1.0, score_bits(legs[(size_t)j]));
      const double base = (sr - sa - sb) / std::max(sa, sb);
      const double score = temperature > 0 ? base - temperature * std::log(-std::log(uniform())) : base;
      heap.push({score, base, i, j});
    };
    std::vector<std::pair<int, int>> init;
    for (size_t x = 1; x < where.size(); ++x) {
      const std::vector<int> &own = where[x];
      for (size_t u = 0; u < own.size(); ++u)
        for (size_t v = u + 1; v < own.size(); ++v)
          if (ok(own[u]) && ok(own[v])) init.push_back({std::min(own[u], own[v]), std::max(own[u], own[v])});
    }
    std::sort(init.begin(), init.end());
    init.erase(std::unique(init.begin(), init.end()), init.end());
    for (const auto &pr : init) push(pr.first, pr.second);
    std::vector<int> seen;
    constexpr int kMaxRedraws = 64;
    int redraws = 0;
    while (!heap.empty()) {
      const Cand c = heap.top();
      heap.pop();
      if (!live[(size_t)c.i] || !live[(size_t)c.j]) continue;
      // the noise of the pair on top is drawn again (as if every pair's noise were drawn anew
      // at every step); a pair that no longer wins goes back
      if (temperature > 0 && !heap.empty() && redraws < kMaxRedraws) {
        const double s2 = c.base - temperature * std::log(-std::log(uniform()));
        if (s2 > heap.top().score) {
          heap.push({s2, c.base, c.i, c.j});
          ++redraws;
          continue;
        }
      }
      redraws = 0;
      const int out = merge(c.i, c.j);
      if (!allowed.empty()) {
        allowed.resize(legs.size(), 0);
        allowed[(size_t)out] = 1;
      }
      if (!ok(out)) continue;
      seen.clear();
      for (int x : legs[(size_t)out]) {
        if (x == 0) continue;
        for (int o : where[x])
          if (o != out && ok(o) && std::find(seen.begin(), seen.end(), o) == seen.end()) {
            seen.push_back(o);
            push(out, o);
          }
      }
    }
  }
  // The same greedy choice with the noise of every candidate pair drawn anew at every step
  // (each step samples a pair with probability ~ exp(-score / temperature)); a full scan of the
  // candidates per step.  A pair's score without noise is computed once: it cannot change while
  // both tensors live (as in greedy()).
  void greedy_stepwise(double temperature, uint64_t seed) {
    uint64_t rs = seed * 6364136223846793005ull + 1442695040888963407ull;
    auto uniform = [&]() {
      rs = rs * 6364136223846793005ull + 1442695040888963407ull;
      return ((rs >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    std::vector<int> res, batch, contr;
    std::unordered_map<uint64_t, double> base_of;  // (i, j) -> score without noise
    for (;;) {
      double best = 1e300;
      int bi = -1, bj = -1;
      for (size_t x = 1; x < where.size(); ++x) {
        const std::vector<int> &own = where[x];
        for (size_t u = 0; u < own.size(); ++u)
          for (size_t v = u + 1; v < own.size(); ++v) {
            const int i = std::min(own[u], own[v]), j = std::max(own[u], own[v]);
            const uint64_t key = ((uint64_t)(uint32_t)i << 32) | (uint32_t)j;
            auto it = base_of.find(key);
            if (it == base_of.end()) {
              merged(i, j, res, batch, contr);
              const double sr = std::ldexp(1.0, score_bits(res)), sa = std::ldexp(1.0, score_bits(legs[(size_t)i])),
                           sb = std::ldexp(1.0, score_bits(legs[(size_t)j]));
              it = base_of.emplace(key, (sr - sa - sb) / std::max(sa, sb)).first;
            }
            double score = it->second;
            if (temperature > 0) score -= temperature * std::log(-std::log(uniform()));
            if (score < best) {
              best = score;
              bi = i;
              bj = j;
            }
          }
      }
      if (bi < 0) break;
      merge(bi, bj);
    }
  }
  // join whatever is left (connected only through the bitstring index); in a sliced network
  // also the tensors left without any index (scalars), smallest pair first
  void finish() {
    const bool by_size = !net.slices.empty();
    for (;;) {
      int bi = -1, bj = -1;
      for (size_t i = 0; i < legs.size(); ++i) {
        if (!live[i]) continue;
        if (!by_size) {
          if (bi < 0) bi = (int)i;
          else if (bj < 0) bj = (int)i;
          continue;
        }
        const int b = bits_of(legs[i]);
        if (bi < 0 || b < bits_of(legs[(size_t)bi])) {
          bj = bi;
          bi = (int)i;
        } else if (bj < 0 || b < bits_of(legs[(size_t)bj])) {
          bj = (int)i;
        }
      }
      if (bj < 0) break;
      merge(std::min(bi, bj), std::max(bi, bj));
    }
    tr.legs = legs;
  }
};

// One greedy contraction path (Contractor::greedy over the whole network, with Gumbel noise
// of the given temperature for the randomised trials).
void greedy_trial(const NetPlan &net, double temperature, uint64_t seed, int score_bits0, Trial &tr) {
  Contractor ct(net);
  ct.score_bits0 = score_bits0;
  ct.greedy(temperature, seed, {});
  ct.finish();
  tr = std::move(ct.tr);
}

// One greedy path with step-wise noise (Contractor::greedy_stepwise).
void stepwise_trial(const NetPlan &net, double temperature, uint64_t seed, int score_bits0, Trial &tr) {
  Contractor ct(net);
  ct.score_bits0 = score_bits0;
  ct.greedy_stepwise(temperature, seed);
  ct.finish();
  tr = std::move(ct.tr);
}

// Fold first: merges of bitstring-independent tensors (evaluated once at plan time) are made
// greedily while their results stay within the folding size, then the greedy goes on over
// the whole network.
void fold_first_trial(const NetPlan &net, double temperature, uint64_t seed, int score_bits0, Trial &tr) {
  Contractor ct(net);
  ct.score_bits0 = score_bits0;
  ct.greedy(temperature, seed, {}, kFoldMaxLog2);
  ct.greedy(temperature, seed + 1, {});
  ct.finish();
  tr = std::move(ct.tr);
}

// Sweep order: each qubit's own tensors (its line, its output closure, and the couplings to
// lower qubits) are contracted into a block first, then the blocks are absorbed one by one
// in qubit order into a single frontier tensor (for a 2D grid numbered row by row this is a
// row-by-row boundary contraction).
void sweep_trial(const NetPlan &net, double temperature, uint64_t seed, Trial &tr) {
  Contractor ct(net);
  int frontier = -1;
  for (int q = 0; q < net.n; ++q) {
    std::vector<char> allowed(ct.legs.size(), 0);
    int members = 0, last = -1;
    for (size_t i = 0; i < net.nodes.size(); ++i)
      if (ct.live[i] && net.nodes[i].group == q) {
        allowed[i] = 1;
        ++members;
        last = (int)i;
      }
    if (members == 0) continue;
    const size_t before = ct.legs.size();
    ct.greedy(temperature, seed + (uint64_t)q, allowed);
    // the block is whatever live tensors of this group remain (normally one)
    std::vector<int> parts;
    for (size_t i = 0; i < ct.legs.size(); ++i) {
      if (!ct.live[i]) continue;
      const bool mine = (i < net.nodes.size()) ? (net.nodes[i].group == q) : (i >= before);
      if (mine) parts.push_back((int)i);
    }
    if (parts.empty()) parts.push_back(last);
    int block = parts[0];
    for (size_t k = 1; k < parts.size(); ++k) block = ct.merge(block, parts[k]);
    frontier = frontier < 0 ? block : ct.merge(frontier, block);
  }
  ct.finish();
  tr = std::move(ct.tr);
}

}  // namespace

namespace {

// Indices to slice so that every intermediate of `order` fits 2^max_log2 entries, one at a
// time: among the indices of a largest tensor, the one leaving the smallest peak, then the
// fewest tensors at that peak, then the fewest flops.  Fills order.slices and the cost of all
// slices (the per-merge cost of Trial::dyn_cost with the sliced indices dropped, times the
// number of slices); order.sliceable stays false if more than kMaxSliceBits would be needed.
void choose_slices(const NetPlan &net, Trial &order, int max_log2) {
  const size_t nt = order.legs.size(), nl = net.label_dim.size();
  std::vector<int> size(nt, 0);
  std::vector<std::vector<int>> tens_of(nl), merges_of(nl);
  for (size_t t = 0; t < nt; ++t)
    for (int x : order.legs[t]) {
      size[t] += net.label_dim[(size_t)x];
      tens_of[(size_t)x].push_back((int)t);
    }
  std::vector<int> ub(order.steps.size(), 0);  // bits of the union of both operands' legs
  for (size_t k = 0; k < order.steps.size(); ++k) {
    const NetStep &st = order.steps[k];
    std::vector<int> u = order.legs[(size_t)st.a];
    for (int x : order.legs[(size_t)st.b])
      if (std::find(u.begin(), u.end(), x) == u.end()) u.push_back(x);
    for (int x : u) {
      ub[k] += net.label_dim[(size_t)x];
      merges_of[(size_t)x].push_back((int)k);
    }
  }
  std::vector<int> hist(130, 0);
  for (int b : size) ++hist[(size_t)b];
  std::vector<char> in_s(nl, 0);
  order.slices.clear();
  order.sliceable = false;
  for (;;) {
    int mx = 0;
    for (int b = 129; b >= 0; --b)
      if (hist[(size_t)b] > 0) {
        mx = b;
        break;
      }
    if (mx <= max_log2) break;
    if ((int)order.slices.size() >= kMaxSliceBits) return;
    int best_x = -1, best_m = 0, best_cnt = 0;
    double best_gain = 0;
    std::vector<char> seen(nl, 0);
    for (size_t t = 0; t < nt; ++t) {
      if (size[t] != mx) continue;
      for (int x : order.legs[t]) {
        if (x == 0 || in_s[(size_t)x] || seen[(size_t)x] || net.label_dim[(size_t)x] == 0) continue;
        seen[(size_t)x] = 1;
        int c_mx = 0, c_mx1 = 0;
        for (int u : tens_of[(size_t)x]) {
          c_mx += size[(size_t)u] == mx;
          c_mx1 += size[(size_t)u] == mx - 1;
        }
        int m, cnt;
        if (c_mx == hist[(size_t)mx]) {
          m = mx - 1;
          cnt = hist[(size_t)mx - 1] - c_mx1 + c_mx;
        } else {
          m = mx;
          cnt = hist[(size_t)mx] - c_mx;
        }
        double gain = 0;  // flops of one slice saved by fixing x
        for (int k : merges_of[(size_t)x]) gain += std::ldexp(1.0, ub[(size_t)k] - 1);
        if (best_x < 0 || m < best_m || (m == best_m && (cnt < best_cnt || (cnt == best_cnt && gain > best_gain)))) {
          best_x = x;
          best_m = m;
          best_cnt = cnt;
          best_gain = gain;
        }
      }
    }
    if (best_x < 0) return;  // only the bitstring index is left on a largest tensor
    in_s[(size_t)best_x] = 1;
    order.slices.push_back(best_x);
    for (int u : tens_of[(size_t)best_x]) {
      --hist[(size_t)size[(size_t)u]];
      --size[(size_t)u];
      ++hist[(size_t)size[(size_t)u]];
    }
    for (int k : merges_of[(size_t)best_x]) --ub[(size_t)k];
  }
  order.sliceable = true;
  const double n_slices = std::ldexp(1.0, (int)order.slices.size());
  auto bits = [&](const std::vector<int> &ls) {
    int b = 0;
    for (int x : ls)
      if (!in_s[(size_t)x]) b += net.label_dim[(size_t)x];
    return b;
  };
  // per slice: merges of folded (bitstring-independent) tensors within the folding size are
  // free (the work budget, spent once per slice copy, is not modelled here)
  double cost = 0, flops = 0;
  std::vector<char> fst(nt, 0);
  for (size_t i = 0; i < net.nodes.size() && i < nt; ++i) fst[i] = net.nodes[i].kind == NODE_FIXED;
  for (size_t k = 0; k < order.steps.size(); ++k) {
    const NetStep &st = order.steps[k];
    const std::vector<int> &res = order.legs[(size_t)st.out];
    if (fst[(size_t)st.a] && fst[(size_t)st.b] && bits(res) <= kFoldMaxLog2) {
      fst[(size_t)st.out] = 1;
      continue;
    }
    const double fl = 8.0 * std::ldexp(1.0, ub[k]);
    flops += fl;
    cost += kLaunchBytes + std::max(8.0 * (std::ldexp(1.0, bits(res)) + std::ldexp(1.0, bits(order.legs[(size_t)st.a])) +
                                           std::ldexp(1.0, bits(order.legs[(size_t)st.b]))),
                                    fl / kRidge);
  }
  order.sliced_cost = cost * n_slices;
  order.sliced_flops = flops * n_slices;
}

// Order preference: orders whose largest intermediate fits the cap first, the cheapest (then
// the fewest flops); then orders that fit once sliced, the cheapest over all slices; then the
// smallest peak.
bool better_order(const Trial &tr, const Trial &best, int max_log2) {
  const bool fits = tr.max_log2 <= max_log2, best_fits = best.max_log2 <= max_log2;
  if (fits != best_fits) return fits;
  if (fits) return tr.dyn_cost < best.dyn_cost || (tr.dyn_cost == best.dyn_cost && tr.flops < best.flops);
  if (tr.sliceable != best.sliceable) return tr.sliceable;
  if (tr.sliceable)
    return tr.sliced_cost < best.sliced_cost || (tr.sliced_cost == best.sliced_cost && tr.sliced_flops < best.sliced_flops);
  return tr.max_log2 < best.max_log2 || (tr.max_log2 == best.max_log2 && tr.flops < best.flops);
}

// fn(t) for t in [begin, end) on the host's cores (each t on one thread; fn writes only its own
// slot of a result array, so the outcome does not depend on the thread count).
template <typename F>
void parallel_for(size_t begin, size_t end, F &&fn) {
  std::atomic<size_t> next{begin};
  auto worker = [&]() {
    for (size_t t = next++; t < end; t = next++) fn(t);
  };
  const size_t n = end > begin ? end - begin : 0;
  const int nth = (int)std::max<size_t>(1, std::min<size_t>(n, std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  for (int i = 1; i < nth; ++i) pool.emplace_back(worker);
  worker();
  for (std::thread &th : pool) th.join();
}

// Randomised trials, the preferred one: half greedy (the first deterministic; they score the
// bitstring index at its size or 4, 8, 12 bits larger in turn; half of them with step-wise
// noise), a quarter qubit sweeps, a quarter fold-first.  With `slice`, orders that exceed the cap are sliced to fit
// (choose_slices).  Trials are independent and run on the host's cores; the choice among
// them is made in trial order, so the result does not depend on the thread count.
Trial search_orders(const NetPlan &net, int max_log2, bool slice, int trials) {
  const int ng = trials / 2, ns = trials / 4;
  std::vector<Trial> res((size_t)trials);
  parallel_for(0, (size_t)trials, [&](size_t ti) {
    const int t = (int)ti;
    Trial &tr = res[ti];
    // u: the trial's index within its kind's sequence (kinds offset by 64 and 128)
    const int u = t < ng ? t : (t < ng + ns ? 64 + (t - ng) : 128 + (t - ng - ns));
    const double temp = (u % 64) == 0 ? 0.0 : 0.05 + 0.5 * (double)(u % 16) / 16.0;
    const uint64_t seed = 0x9E3779B97F4A7C15ull * (uint64_t)(u + 1);
    const int w0 = (u & 3) ? net.label_dim[0] + 4 * (u & 3) : -1;
    if (trials == 1) greedy_trial(net, 0.0, seed, -1, tr);  // the deterministic greedy alone
    else if (t < ng / 2) greedy_trial(net, temp, seed, w0, tr);
    else if (t < ng) stepwise_trial(net, temp, seed, w0, tr);
    else if (t < ng + ns) sweep_trial(net, (u % 64) == 0 ? 0.05 : temp, seed, tr);
    else fold_first_trial(net, temp, seed, w0, tr);
    if (slice && tr.max_log2 > max_log2) choose_slices(net, tr, max_log2);
  });
  const bool debug = getenv("TNQ_DEBUG_NET") != nullptr;
  int best_t = 0;
  for (int t = 0; t < trials; ++t) {
    const Trial &tr = res[(size_t)t];
    if (debug)
      fprintf(stderr, "trial %d: peak %d flops %.3e cost %.3e sliced %d (%zu) cost %.3e\n", t, tr.max_log2, tr.flops,
              tr.dyn_cost, (int)tr.sliceable, tr.slices.size(), tr.sliced_cost);
    if (t > 0 && better_order(tr, res[(size_t)best_t], max_log2)) best_t = t;
  }
  if (debug) fprintf(stderr, "best trial %d of %d\n", best_t, trials);
  return std::move(res[(size_t)best_t]);
}

// Adaptive search (a cross-entropy hyper-optimiser over the order generator): the settings of
// a trial are its kind (greedy, step-wise greedy, qubit sweep, fold-first), its noise
// temperature and the extra weight the greedy kinds give the bitstring index (0, 4, 8 or 12
// bits).  The first round draws them uniformly (and includes the deterministic greedy); after
// every round the distribution is refitted to the best quarter of all orders so far (kind and
// weight frequencies with add-one smoothing, temperature mean and spread), so later rounds
// spend their trials where good orders came from.  Settings come from one seeded generator and
// the choice is made in generation order: the result is deterministic.
Trial adaptive_search(const NetPlan &net, int max_log2, bool slice, int trials) {
  struct Spec {
    int kind;
    double temp;
    int extra;  // -1: the bitstring index at its size
    uint64_t seed;
  };
  uint64_t rs = 0x2545F4914F6CDD1Dull;
  auto next_u64 = [&]() {  // splitmix64
    uint64_t z = (rs += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  auto uniform = [&]() { return ((next_u64() >> 11) + 0.5) * (1.0 / 9007199254740992.0); };
  auto pick = [&](const double *p, int n) {
    double r = uniform(), acc = 0;
    for (int i = 0; i < n - 1; ++i) {
      acc += p[i];
      if (r < acc) return i;
    }
    return n - 1;
  };
  double p_kind[4] = {0.25, 0.25, 0.25, 0.25}, p_extra[4] = {0.25, 0.25, 0.25, 0.25};
  double t_mean = 0.3, t_sd = 0.25;
  const int rounds = 4, per_round = std::max(8, trials / rounds);
  std::vector<Spec> specs;
  std::vector<Trial> res;
  for (int r = 0; r < rounds; ++r) {
    const size_t first = specs.size();
    for (int i = 0; i < per_round; ++i) {
      Spec sp;
      if (r == 0 && i == 0) {
        sp = Spec{0, 0.0, -1, 0x9E3779B97F4A7C15ull};  // the deterministic greedy
      } else {
        sp.kind = pick(p_kind, 4);
        // temperature: normal around the elite mean (Box-Muller), kept within [0, 2]
        const double g = std::sqrt(-2.0 * std::log(uniform())) * std::cos(6.283185307179586 * uniform());
        sp.temp = std::min(2.0, std::max(0.0, t_mean + t_sd * g));
        const int e = pick(p_extra, 4);
        sp.extra = e == 0 ? -1 : 4 * e;
        sp.seed = next_u64();
      }
      specs.push_back(sp);
    }
    res.resize(specs.size());
    parallel_for(first, specs.size(), [&](size_t t) {
      const Spec &sp = specs[t];
      Trial &tr = res[t];
      const int w0 = sp.extra < 0 ? -1 : net.label_dim[0] + sp.extra;
      if (sp.kind == 0) greedy_trial(net, sp.temp, sp.seed, w0, tr);
      else if (sp.kind == 1) stepwise_trial(net, sp.temp, sp.seed, w0, tr);
      else if (sp.kind == 2) sweep_trial(net, std::max(sp.temp, 0.05), sp.seed, tr);
      else fold_first_trial(net, sp.temp, sp.seed, w0, tr);
      if (slice && tr.max_log2 > max_log2) choose_slices(net, tr, max_log2);
    });
    // refit to the best quarter of everything so far
    std::vector<size_t> order(res.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t a, size_t b) { return better_order(res[a], res[b], max_log2); });
    const size_t elite = std::max<size_t>(4, order.size() / 4);
    double ck[4] = {1, 1, 1, 1}, ce[4] = {1, 1, 1, 1}, sum = 0, sum2 = 0;
    for (size_t k = 0; k < elite && k < order.size(); ++k) {
      const Spec &sp = specs[order[k]];
      ck[sp.kind] += 1;
      ce[sp.extra < 0 ? 0 : sp.extra / 4] += 1;
      sum += sp.temp;
      sum2 += sp.temp * sp.temp;
    }
    const double ne = (double)std::min(elite, order.size());
    for (int i = 0; i < 4; ++i) {
      p_kind[i] = ck[i] / (ne + 4.0);
      p_extra[i] = ce[i] / (ne + 4.0);
    }
    t_mean = sum / ne;
    t_sd = std::max(0.02, std::sqrt(std::max(0.0, sum2 / ne - t_mean * t_mean)));
  }
  int best_t = 0;
  for (size_t t = 1; t < res.size(); ++t)
    if (better_order(res[t], res[(size_t)best_t], max_log2)) best_t = (int)t;
  if (getenv("TNQ_DEBUG_NET"))
    fprintf(stderr, "adaptive: best trial %d of %zu (kind %d, temperature %.3f, extra %d)\n", best_t, res.size(),
            specs[(size_t)best_t].kind, specs[(size_t)best_t].temp, specs[(size_t)best_t].extra);
  return std::move(res[(size_t)best_t]);
}

// The merges of `order` (planned on the unsliced network) replayed on the sliced one.
Trial replay_order(const NetPlan &net, const Trial &order) {
  Contractor ct(net);
  for (const NetStep &st : order.steps) ct.merge(st.a, st.b);
  ct.finish();
  return std::move(ct.tr);
}

}  // namespace

tn_status plan_network(NetPlan &net, int max_log2, int order_trials, int order_search, std::string &err) {
  const int trials = order_trials > 0 ? order_trials : kTrials;
  const int coarse = std::min(trials, kCoarseTrials);
  // the full searches: the fixed trial mix, or the adaptive search (order_search = 1)
  auto full_search = [&](bool slice) {
    return order_search == 1 && trials > 1 ? adaptive_search(net, max_log2, slice, trials)
                                           : search_orders(net, max_log2, slice, trials);
  };
  net.slices.clear();
  net.sliced.assign(net.label_dim.size(), 0);
  const int lb = net.call_log2;
  auto set_batch = [&](int bits) {
    net.log2_batch = bits;
    net.label_dim[0] = bits;
  };
  // Bitstrings per pass: amplitudes of different bitstrings are independent, so a call may
  // contract its bitstrings 2^(lb - j) at a time in 2^j passes.  A smaller pass shrinks every
  // tensor that carries the bitstring index (a cap may then be met without slicing) and
  // lets the order treat the output closures differently, at the price of more launches.
  // Every pass size is planned; the cheapest over a full call is kept.
  auto usable = [&](const Trial &t) { return t.max_log2 <= max_log2 || t.sliceable; };
  auto call_cost = [&](const Trial &t, int passes_log2) {
    return std::ldexp(t.max_log2 <= max_log2 ? t.dyn_cost : t.sliced_cost, passes_log2);
  };
  // a coarse search per pass size, then the full search at the best one
  Trial best;
  int best_j = -1;
  for (int j = 0; j <= lb; ++j) {
    set_batch(lb - j);
    Trial t = search_orders(net, max_log2, true, coarse);
    if (getenv("TNQ_DEBUG_NET"))
      fprintf(stderr, "pass 2^%d: peak %d, %zu sliced, usable %d, call cost %.4g\n", lb - j, t.max_log2,
              t.slices.size(), (int)usable(t), call_cost(t, j));
    if (best_j < 0 || (usable(t) && (!usable(best) || call_cost(t, j) < call_cost(best, best_j)))) {
      best = std::move(t);
      best_j = j;
    }
  }
  set_batch(lb - best_j);
  Trial full = full_search(true);
  if (usable(full) && (!usable(best) || call_cost(full, best_j) < call_cost(best, best_j))) best = std::move(full);
  if (best.max_log2 > max_log2) {
    if (!best.sliceable) {
      err = "network contraction would create a 2^" + std::to_string(best.max_log2) + "-entry intermediate (cap 2^" +
            std::to_string(max_log2) + ") and more than 2^" + std::to_string(kMaxSliceBits) +
            " slices would be needed to bring it within the cap";
      return TN_ERR_UNSUPPORTED;
    }
    net.slices = best.slices;
    for (int x : net.slices) net.sliced[(size_t)x] = 1;
    // the order found above, on the sliced network, fits by construction; a search on the
    // sliced network itself may find a cheaper one
    Trial replay = replay_order(net, best);
    Trial again = full_search(false);
    best = better_order(again, replay, max_log2) ? std::move(again) : std::move(replay);
  }
  net.steps = best.steps;
  net.all_legs = best.legs;
  net.max_log2 = best.max_log2;
  if (net.max_log2 > max_log2) {
    err = "network contraction would create a 2^" + std::to_string(net.max_log2) + "-entry intermediate (cap 2^" +
          std::to_string(max_log2) + ")";
    return TN_ERR_UNSUPPORTED;
  }
  return TN_OK;
}

}  // namespace tnq
