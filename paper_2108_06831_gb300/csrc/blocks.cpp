// Host planner of the uniform-block state contraction (see blocks.h).
//
// Blocks are formed round by round.  A round cuts the register into windows of k consecutive
// qubits, at offset 0 on even rounds and k/2 on odd ones (so the windows of consecutive rounds
// overlap, like the bricks of a wall), and gives every window the light cone it can take: in
// time order, a pending gate joins the window's block when all its qubits lie in the window
// and no earlier pending gate on those qubits was left out.  Gates that no window can take
// (qubits farther apart than k, or a light cone that keeps being cut) are handled by a seeded
// block: the earliest pending gate's qubits, grown by the qubits of the following pending
// gates while at most k, take their light cone.  The earliest pending gate always qualifies,
// so every seeded block makes progress.  Blocks narrower than k are padded with idle qubits:
// every block is a 2^k x 2^k matrix.
//
// Layouts: block i reads the state with its qubits as the lowest k index bits (local bit t =
// qubit qubits[i][t]); above them come the qubits of block i+1 that block i does not hold,
// then the rest in the canonical order (qubit q at bit N-1-q).  Block i's GEMM stores its
// result in block i+1's layout (the last one in the canonical layout) through its output
// map; since block i+1's lowest qubit sits among the lowest row bits of block i's output,
// consecutive stored elements stay adjacent in the GEMM's store order.
#include <algorithm>
#include <cstring>

#include "blocks.h"

namespace tnq {

namespace {

uint64_t gate_mask(const TnGate &g) {
  uint64_t m = 1ull << g.q[0];
  if (gate_nqubits(g.kind) == 2) m |= 1ull << g.q[1];
  return m;
}

int popc64(uint64_t v) {
  int n = 0;
  while (v) {
    v &= v - 1;
    ++n;
  }
  return n;
}

}  // namespace

tn_status plan_blocks(const tn_circuit &c, int k, int batch, int precision, BlockPlan &bp, std::string &err) {
  const int N = c.n;
  if (k < 6 || k > 7) {
    err = "block_qubits must be 6 or 7 (2^k x 2^k blocks on the GEMM's tiles)";
    return TN_ERR_INVALID_ARG;
  }
  if (N < k + 7 || N > kMaxQubits) {
    err = "uniform blocks need k + 7 <= n_qubits <= 34 (at least 128 rows per GEMM)";
    return TN_ERR_UNSUPPORTED;
  }
  if (precision != TN_PREC_FP32 && N - k > 23) {
    err = "uniform blocks on the tensor cores take at most k + 23 qubits (2^23 rows per GEMM)";
    return TN_ERR_UNSUPPORTED;
  }
  if (batch < 1 || (batch & (batch - 1)) != 0) {
    err = "uniform blocks take a power-of-two batch";
    return TN_ERR_UNSUPPORTED;
  }
  bp = BlockPlan();
  bp.k = k;
  bp.n = N;
  bp.batch = batch;
  bp.precision = precision;
  bp.init = c.init;
  const int G = (int)c.gates.size();
  std::vector<char> done((size_t)G, 0);
  std::vector<uint64_t> gm((size_t)G);
  for (int i = 0; i < G; ++i) gm[(size_t)i] = gate_mask(c.gates[(size_t)i]);
  int remaining = G;
  std::vector<std::vector<int>> blk_gates;
  std::vector<uint64_t> blk_window;
  auto absorb = [&](uint64_t W) {
    std::vector<int> got;
    uint64_t blocked = 0;
    for (int i = 0; i < G; ++i) {
      if (done[(size_t)i]) continue;
      const uint64_t m = gm[(size_t)i];
      if (m & blocked) {
        blocked |= m;
        continue;
      }
      if ((m & ~W) == 0) got.push_back(i);
      else blocked |= m;
    }
    for (int i : got) done[(size_t)i] = 1;
    remaining -= (int)got.size();
    return got;
  };
  int idle_rounds = 0;
  while (remaining > 0) {
    const int off = (bp.rounds & 1) ? k / 2 : 0;
    ++bp.rounds;
    bool any = false;
    std::vector<std::pair<int, int>> wins;
    if (off > 0) wins.push_back({0, off});
    for (int a = off; a < N; a += k) wins.push_back({a, std::min(N, a + k)});
    for (auto [a, b] : wins) {
      uint64_t W = 0;
      for (int q = a; q < b; ++q) W |= 1ull << q;
      std::vector<int> got = absorb(W);
      if (got.empty()) continue;
      any = true;
      blk_gates.push_back(std::move(got));
      blk_window.push_back(W);
    }
    idle_rounds = any ? 0 : idle_rounds + 1;
    if (idle_rounds >= 2 && remaining > 0) {  // both offsets took nothing: seed a block
      uint64_t Q = 0;
      for (int i = 0; i < G; ++i) {
        if (done[(size_t)i]) continue;
        if (Q == 0 || popc64(Q | gm[(size_t)i]) <= k) Q |= gm[(size_t)i];
        if (popc64(Q) == k) break;
      }
      std::vector<int> got = absorb(Q);
      blk_gates.push_back(std::move(got));
      blk_window.push_back(Q);
      ++bp.seeded;
      idle_rounds = 0;
    }
  }
  const int B = (int)blk_gates.size();
  if (B == 0) {  // no gates: one identity block on the lowest qubits
    blk_gates.push_back({});
    blk_window.push_back(0);
  }
  const int nb = (int)blk_gates.size();
  // qubit sets, padded to k: the block's own qubits, then its window's, then the lowest others
  std::vector<uint64_t> qset((size_t)nb);
  for (int i = 0; i < nb; ++i) {
    uint64_t Q = 0;
    for (int g : blk_gates[(size_t)i]) Q |= gm[(size_t)g];
    for (int q = 0; q < N && popc64(Q) < k; ++q)
      if ((blk_window[(size_t)i] >> q) & 1) Q |= 1ull << q;
    for (int q = 0; q < N && popc64(Q) < k; ++q) Q |= 1ull << q;
    qset[(size_t)i] = Q;
  }
  // local orders: block i+1 lists first the qubits block i does not hold (qubit descending),
  // then the shared ones
  bp.qubits.assign((size_t)nb, {});
  for (int q = N - 1; q >= 0; --q)
    if ((qset[0] >> q) & 1) bp.qubits[0].push_back(q);
  for (int i = 1; i < nb; ++i) {
    const uint64_t fresh = qset[(size_t)i] & ~qset[(size_t)i - 1], shared = qset[(size_t)i] & qset[(size_t)i - 1];
    for (int q = N - 1; q >= 0; --q)
      if ((fresh >> q) & 1) bp.qubits[(size_t)i].push_back(q);
    for (int q = N - 1; q >= 0; --q)
      if ((shared >> q) & 1) bp.qubits[(size_t)i].push_back(q);
  }
  // layouts: stored bit -> qubit
  auto canonical = [&]() {
    std::vector<int> L((size_t)N);
    for (int j = 0; j < N; ++j) L[(size_t)j] = N - 1 - j;
    return L;
  };
  auto layout_of = [&](int i) {  // the layout block i reads
    std::vector<int> L;
    uint64_t used = 0;
    for (int q : bp.qubits[(size_t)i]) {
      L.push_back(q);
      used |= 1ull << q;
    }
    if (i + 1 < nb)
      for (int q : bp.qubits[(size_t)i + 1])
        if (!((used >> q) & 1)) {
          L.push_back(q);
          used |= 1ull << q;
        }
    for (int q = N - 1; q >= 0; --q)
      if (!((used >> q) & 1)) L.push_back(q);
    return L;
  };
  auto inverse = [&](const std::vector<int> &L) {
    std::vector<int> inv((size_t)N);
    for (int j = 0; j < N; ++j) inv[(size_t)L[(size_t)j]] = j;
    return inv;
  };
  int lb = 0;
  while ((1 << lb) < batch) ++lb;
  bp.maps.assign((size_t)nb, OutMap());
  for (int i = 1; i < nb; ++i) {
    const std::vector<int> in = layout_of(i);
    const std::vector<int> tgt = inverse(i + 1 < nb ? layout_of(i + 1) : canonical());
    OutMap &om = bp.maps[(size_t)i];
    om.identity = 1;
    om.nbits = N + lb;
    for (int j = 0; j < N; ++j) {
      om.pos[j] = (uint8_t)tgt[(size_t)in[(size_t)j]];
      if (om.pos[j] != j) om.identity = 0;
    }
    for (int j = N; j < N + lb; ++j) om.pos[j] = (uint8_t)j;
  }
  // block 0 on the basis state: where each of its 2^k outputs goes
  {
    const std::vector<int> tgt = inverse(nb > 1 ? layout_of(1) : canonical());
    const std::vector<int> &Q = bp.qubits[0];
    auto bit_of_init = [&](int q) { return (int)((c.init >> (N - 1 - q)) & 1ull); };
    bp.init_local = 0;
    for (int t = 0; t < k; ++t) bp.init_local |= bit_of_init(Q[(size_t)t]) << t;
    uint64_t rest = 0;
    uint64_t inQ = 0;
    for (int q : Q) inQ |= 1ull << q;
    for (int q = 0; q < N; ++q)
      if (!((inQ >> q) & 1) && bit_of_init(q)) rest |= 1ull << tgt[(size_t)q];
    bp.init_pos.resize((size_t)1 << k);
    for (int r = 0; r < (1 << k); ++r) {
      uint64_t s = rest;
      for (int t = 0; t < k; ++t)
        if ((r >> t) & 1) s |= 1ull << tgt[(size_t)Q[(size_t)t]];
      bp.init_pos[(size_t)r] = (long long)s;
    }
  }
  // gates in local bits
  for (int i = 0; i < nb; ++i) {
    std::vector<int> local((size_t)N, -1);
    for (int t = 0; t < k; ++t) local[(size_t)bp.qubits[(size_t)i][(size_t)t]] = t;
    bp.gate_begin.push_back((int)bp.gates.size());
    for (int g : blk_gates[(size_t)i]) {
      const TnGate &tg = c.gates[(size_t)g];
      BlockGate b;
      std::memset(&b, 0, sizeof(b));
      b.kind = tg.kind;
      b.la = local[(size_t)tg.q[0]];
      b.lb = gate_nqubits(tg.kind) == 2 ? local[(size_t)tg.q[1]] : -1;
      for (int a = 0; a < 3; ++a) {
        b.angle[a] = tg.angle[a];
        b.pidx[a][0] = tg.pidx[a][0];
        b.pidx[a][1] = tg.pidx[a][1];
      }
      for (int a = 0; a < 32; ++a) b.mat[a] = tg.mat[a];
      if (b.la < 0 || (gate_nqubits(tg.kind) == 2 && b.lb < 0)) {
        err = "block planner: a gate outside its block (internal error)";
        return TN_ERR_UNSUPPORTED;
      }
      bp.gates.push_back(b);
    }
    bp.gate_count.push_back((int)bp.gates.size() - bp.gate_begin.back());
  }
  const double M = (double)(1ull << (N - k)), K = (double)(1 << k);
  bp.flops = 8.0 * M * K * K * (double)(nb - 1);
  bp.bytes = 16.0 * (double)(1ull << N) * (double)(nb - 1) + 8.0 * (double)(1ull << N);
  return TN_OK;
}

}  // namespace tnq
