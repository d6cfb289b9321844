// Host planner of libtnq: orders and groups the circuit's gate contractions.
//
// The paper treats the contraction order as a hyperparameter chosen before evaluation
// (Sec. 2.2.3) and deploys only the order it selected (Sec. 3).  On one GPU the costly
// contractions are the rank-growing ones, a small gate tensor merged into the large
// state tensor (Sec. 2.2.1: tensor product followed by a contraction over the shared
// index).  Each of them streams the whole state once, so the plan fuses as many of them
// as dependencies allow into one pass over HBM:
//
//   pass   = one launch; a tile of 2^T amplitudes (T "tile bits", always including the
//            kLowBits lowest bits so loads are 128-byte runs) is staged in shared memory;
//   phase  = inside a pass, K tile bits are mapped to registers (2^K amplitudes per
//            thread); every op of the phase touches only registers;
//   op     = one gate.  A gate needs its non-diagonal qubits among the register bits;
//            diagonal factors (Z/S/T/RZ, CZ, CP) and CNOT controls read any bit.
//
// A gate can join a phase only when every earlier gate sharing a qubit with it has
// already been applied (a qubit touched by a deferred gate is "blocked" for the rest of
// the scan).  Passes and phases are built greedily in time order.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "tnq_internal.h"

namespace tnq {
namespace {

struct GateCls {
  int type;        // OpType
  int qa, qb;      // qubits (qb = -1 for one-qubit ops)
  bool need_a, need_b;
  int shape;       // MatShape of its entries (-1: none)
};

bool mat1_is_diagonal(const TnGate &g) {
  return g.mat[2] == 0 && g.mat[3] == 0 && g.mat[4] == 0 && g.mat[5] == 0;
}

GateCls classify(const TnGate &g) {
  GateCls c{};
  c.qa = g.q[0];
  c.qb = -1;
  switch (g.kind) {
    case TN_GATE_Z: case TN_GATE_S: case TN_GATE_SDG: case TN_GATE_T: case TN_GATE_TDG: case TN_GATE_RZ: case KIND_P:
      c.type = OP_D1; c.shape = SHAPE_DIAG2; break;
    case TN_GATE_MAT1:
      if (mat1_is_diagonal(g)) { c.type = OP_D1; c.shape = SHAPE_DIAG2; }
      else { c.type = OP_G1; c.need_a = true; c.shape = SHAPE_M2; }
      break;
    case TN_GATE_CZ: c.type = OP_CZ; c.qb = g.q[1]; c.shape = -1; break;
    case TN_GATE_CP: c.type = OP_DP; c.qb = g.q[1]; c.shape = SHAPE_PHASE; break;
    case TN_GATE_CNOT: c.type = OP_C1; c.qb = g.q[1]; c.need_b = true; c.shape = SHAPE_M2; break;
    case TN_GATE_SWAP: case TN_GATE_MAT2:
      c.type = OP_G2; c.qb = g.q[1]; c.need_a = c.need_b = true; c.shape = SHAPE_M4; break;
    case KIND_F2:
      c.type = OP_G2; c.qb = g.q[1]; c.need_a = c.need_b = true; c.shape = SHAPE_M4X; break;
    default:  // H X Y SX SY SW RX RY U3
      c.type = OP_G1; c.need_a = true; c.shape = SHAPE_M2; break;
  }
  return c;
}

// Real flops per amplitude of one op as executed (complex multiply = 6, add = 2; a real
// coefficient times a complex value = 2): a general 2x2 costs 14, a matrix with a real first
// column (V) 10, a real or real-diagonal/imaginary-off-diagonal one (RY, H, SY, RX, SX) 6;
// a phase diag(1, e) touches half the amplitudes; permutations (X, CNOT's target, SWAP) are
// register exchanges.
double op_flops(int type, int kind) {
  switch (type) {
    case OP_G1:
      if (kind == KIND_V) return 10.0;
      if (kind == TN_GATE_RY || kind == TN_GATE_H || kind == TN_GATE_SY || kind == TN_GATE_RX || kind == TN_GATE_SX)
        return 6.0;
      if (kind == TN_GATE_X) return 0.0;
      return 14.0;
    case OP_D1:
      if (kind == KIND_P || kind == TN_GATE_S || kind == TN_GATE_SDG || kind == TN_GATE_T || kind == TN_GATE_TDG)
        return 3.0;
      if (kind == TN_GATE_Z) return 0.0;
      return 6.0;
    case OP_G2: return kind == TN_GATE_SWAP ? 0.0 : 30.0;  // a SWAP exchanges registers
    case OP_C1: return 7.0;
    case OP_DP: return 1.5;
    default: return 0.0;
  }
}

// Estimated instructions one op adds to a plan-specialised pass kernel (16 amplitudes per
// thread): a pass's straight-line code must stay well inside the instruction cache.
int op_code_cost(int type, int kind, bool adjoint, bool has_grad, int n_grad) {
  int c;
  switch (type) {
    case OP_G1: c = (kind == TN_GATE_X) ? 8 : 110; break;
    case OP_G2: c = (kind == TN_GATE_SWAP) ? 8 : 290; break;
    case OP_C1: c = (kind == TN_GATE_CNOT) ? 12 : 70; break;
    case OP_D1: c = 70; break;
    case OP_CZ: c = 20; break;
    default: c = 40; break;
  }
  if (adjoint) c = 2 * c + (has_grad ? 150 * n_grad : 0);
  return c;
}
constexpr int kPassCodeBudget = 7000;

int shape_entries(int shape) { return shape_units(shape); }

struct Planner {
  int N, T, K;
  std::vector<GateCls> cls;
  std::vector<int> order;  // gate indices in application order
  std::vector<char> done;

  int bit_of(int q) const { return N - 1 - q; }

  // needed register/tile bits of gate g (as global bit positions)
  int needs(int g, int out[2]) const {
    int k = 0;
    if (cls[g].need_a) out[k++] = bit_of(cls[g].qa);
    if (cls[g].need_b) out[k++] = bit_of(cls[g].qb);
    return k;
  }
  void qubits(int g, int out[2], int &k) const {
    k = 0;
    out[k++] = cls[g].qa;
    if (cls[g].qb >= 0) out[k++] = cls[g].qb;
  }
};

uint64_t bitmask(int b) { return 1ull << b; }

bool is_diagonal_kind(const TnGate &g) {
  switch (g.kind) {
    case TN_GATE_Z: case TN_GATE_S: case TN_GATE_SDG: case TN_GATE_T: case TN_GATE_TDG: case TN_GATE_RZ:
    case TN_GATE_CZ: case TN_GATE_CP: case KIND_P:
      return true;
    case TN_GATE_MAT1:
      return mat1_is_diagonal(g);
    default:
      return false;
  }
}

// Cost of a gate in the forward pass kernels, in packed FP32x2 multiply-add instructions per
// amplitude (the FMA pipe's work): U3 3 (after the phase-pushing rewrite below), a real or
// imaginary-off-diagonal rotation 2, a general 2x2 4, a one-sided phase 1, a general diagonal 2,
// permutations (X, CNOT, SWAP) none, a sign (Z, CZ) a quarter; a dense 4x4 costs 8.
double fuse_cost(const TnGate &g) {
  switch (g.kind) {
    case TN_GATE_U3: return 3.0;
    case TN_GATE_RX: case TN_GATE_RY: case TN_GATE_H: case TN_GATE_SX: case TN_GATE_SY: return 2.0;
    case TN_GATE_X: case TN_GATE_CNOT: case TN_GATE_SWAP: return 0.0;
    case TN_GATE_Z: case TN_GATE_CZ: return 0.25;
    case TN_GATE_S: case TN_GATE_SDG: case TN_GATE_T: case TN_GATE_TDG: return 1.0;
    case TN_GATE_CP: return 0.5;
    case TN_GATE_RZ: return 2.0;
    case TN_GATE_MAT1: return mat1_is_diagonal(g) ? 2.0 : 4.0;
    case TN_GATE_MAT2: return 8.0;
    default: return 4.0;  // Y, SW: general 2x2
  }
}
constexpr double kFusedCost = 8.0;
// gates of one block: the phase-pushing rewrite may add two leading phase members later
constexpr int kMaxBlockGates = kMaxFusedMembers - 2;
constexpr double kFuseMargin = 0.5;  // fuse only when it saves more than this

}  // namespace

// Precontracts runs of gates on two qubits into dense 4x4 blocks (KIND_F2), the GPU form of
// the paper's precomputation of small contractions so that what is deployed are square
// matrices of one size (Sec. 3).  Gates are scanned in time order; each qubit has at most one
// open block (one qubit or two).  A one-qubit gate joins its qubit's block.  A two-qubit gate
// joins the block of its pair, or merges two one-qubit blocks into a pair block; otherwise the
// blocks of its qubits are closed, and it is emitted on its own if diagonal (it would only
// couple two blocks) or starts a pair block.  A closed pair block becomes one KIND_F2 when its
// gates cost more than a dense 4x4 (fuse_cost), else its gates are emitted as they are.
// Emitting a block when it closes only moves gates past gates on other qubits, so the result
// applies the same operator.
tn_circuit fuse_pairs(const tn_circuit &c, std::vector<FusedMember> &fused) {
  tn_circuit o;
  o.n = c.n;
  o.init = c.init;
  o.n_params = c.n_params;
  struct Block {
    int qa = -1, qb = -1;  // qb < 0: one-qubit block
    std::vector<int> gates;
    double cost = 0.0;
  };
  std::vector<Block> blocks;
  std::vector<int> open((size_t)c.n, -1);
  auto member_of = [&](const TnGate &g, int qa) {
    FusedMember m;
    std::memset(&m, 0, sizeof(m));
    m.kind = g.kind;
    if (gate_nqubits(g.kind) == 1) m.role = g.q[0] == qa ? ROLE_A : ROLE_B;
    else m.role = g.q[0] == qa ? ROLE_AB : ROLE_BA;
    for (int a = 0; a < 3; ++a) {
      m.angle[a] = g.angle[a];
      m.pidx[a][0] = g.pidx[a][0];
      m.pidx[a][1] = g.pidx[a][1];
    }
    for (int a = 0; a < 32; ++a) m.mat[a] = g.mat[a];
    return m;
  };
  auto close = [&](int q) {
    const int bi = open[(size_t)q];
    if (bi < 0) return;
    Block &b = blocks[(size_t)bi];
    open[(size_t)b.qa] = -1;
    if (b.qb >= 0) open[(size_t)b.qb] = -1;
    if (b.qb >= 0 && b.cost > kFusedCost + kFuseMargin) {
      TnGate f;
      std::memset(&f, 0, sizeof(f));
      f.kind = KIND_F2;
      f.q[0] = b.qa;
      f.q[1] = b.qb;
      f.param_idx = -1;
      for (int a = 0; a < 3; ++a) f.pidx[a][0] = f.pidx[a][1] = -1;
      f.fuse_begin = (int)fused.size();
      for (int gi : b.gates) fused.push_back(member_of(c.gates[(size_t)gi], b.qa));
      f.fuse_count = (int)b.gates.size();
      o.gates.push_back(f);
    } else {
      for (int gi : b.gates) o.gates.push_back(c.gates[(size_t)gi]);
    }
    b.gates.clear();
  };
  auto add = [&](int bi, int gi) {
    blocks[(size_t)bi].gates.push_back(gi);
    blocks[(size_t)bi].cost += fuse_cost(c.gates[(size_t)gi]);
  };
  for (int gi = 0; gi < (int)c.gates.size(); ++gi) {
    const TnGate &g = c.gates[(size_t)gi];
    if (gate_nqubits(g.kind) == 1) {
      const int q = g.q[0];
      int bi = open[(size_t)q];
      if (bi >= 0 && (int)blocks[(size_t)bi].gates.size() >= kMaxBlockGates) {
        close(q);
        bi = -1;
      }
      if (bi < 0) {
        blocks.emplace_back();
        bi = (int)blocks.size() - 1;
        blocks[(size_t)bi].qa = q;
        open[(size_t)q] = bi;
      }
      add(bi, gi);
      continue;
    }
    const int a = g.q[0], b = g.q[1];
    const int A = open[(size_t)a], B = open[(size_t)b];
    if (A >= 0 && A == B && (int)blocks[(size_t)A].gates.size() < kMaxBlockGates) {
      add(A, gi);
      continue;
    }
    const bool a_free = A < 0 || blocks[(size_t)A].qb < 0;
    const bool b_free = B < 0 || blocks[(size_t)B].qb < 0;
    const size_t na = A >= 0 ? blocks[(size_t)A].gates.size() : 0, nb = B >= 0 ? blocks[(size_t)B].gates.size() : 0;
    if (A != B && a_free && b_free && (int)(na + nb) < kMaxBlockGates) {
      Block nbk;
      nbk.qa = a;
      nbk.qb = b;
      for (int k : {A, B}) {
        if (k < 0) continue;
        for (int x : blocks[(size_t)k].gates) nbk.gates.push_back(x);
        nbk.cost += blocks[(size_t)k].cost;
        blocks[(size_t)k].gates.clear();
      }
      blocks.push_back(std::move(nbk));
      const int bi = (int)blocks.size() - 1;
      open[(size_t)a] = open[(size_t)b] = bi;
      add(bi, gi);
      continue;
    }
    close(a);
    close(b);
    if (is_diagonal_kind(g)) {
      o.gates.push_back(g);
      continue;
    }
    blocks.emplace_back();
    const int bi = (int)blocks.size() - 1;
    blocks[(size_t)bi].qa = a;
    blocks[(size_t)bi].qb = b;
    open[(size_t)a] = open[(size_t)b] = bi;
    add(bi, gi);
  }
  for (int q = 0; q < c.n; ++q) close(q);
  return o;
}

// Rewrites every U3(t, p, l) as P(p) V(t, l) (exact: U3 = P(p) RY(t) P(l)) and carries each
// pending P(p) forward along its qubit while it commutes with what follows (diagonal gates,
// the control of a CNOT, a SWAP that relabels it), merging it into the next V as
// V(t', l' + p).  A pending phase that meets anything else is emitted as a gate P(p) first;
// the remaining ones are emitted at the end.  V costs 12 real multiply-adds per amplitude
// pair instead of 16 for a general 2x2 matrix, because its first column is real.
tn_circuit push_phases(const tn_circuit &c, std::vector<FusedMember> &fused) {
  tn_circuit o;
  o.n = c.n;
  o.init = c.init;
  o.n_params = c.n_params;
  struct Pending {
    bool on = false;
    double val = 0;
    int idx = -1;
  };
  std::vector<Pending> pend((size_t)c.n);
  auto emit_p = [&](int q) {
    Pending &pp = pend[(size_t)q];
    if (!pp.on) return;
    TnGate g;
    std::memset(&g, 0, sizeof(g));
    g.kind = KIND_P;
    g.q[0] = q;
    g.q[1] = -1;
    g.param_idx = -1;
    for (int a = 0; a < 3; ++a) g.pidx[a][0] = g.pidx[a][1] = -1;
    g.angle[0] = pp.val;
    g.pidx[0][0] = pp.idx;
    o.gates.push_back(g);
    pp = Pending();
  };
  for (const TnGate &g : c.gates) {
    if (g.kind == TN_GATE_U3) {
      const int q = g.q[0];
      TnGate v;
      std::memset(&v, 0, sizeof(v));
      v.kind = KIND_V;
      v.q[0] = q;
      v.q[1] = -1;
      v.param_idx = -1;
      for (int a = 0; a < 3; ++a) v.pidx[a][0] = v.pidx[a][1] = -1;
      v.angle[0] = g.angle[0];
      v.pidx[0][0] = g.pidx[0][0];
      v.angle[1] = g.angle[2] + (pend[(size_t)q].on ? pend[(size_t)q].val : 0.0);
      v.pidx[1][0] = g.pidx[2][0];
      v.pidx[1][1] = pend[(size_t)q].on ? pend[(size_t)q].idx : -1;
      o.gates.push_back(v);
      pend[(size_t)q].on = true;
      pend[(size_t)q].val = g.angle[1];
      pend[(size_t)q].idx = g.pidx[1][0];
      continue;
    }
    if (is_diagonal_kind(g)) {
      o.gates.push_back(g);
      continue;
    }
    if (g.kind == TN_GATE_CNOT) {
      emit_p(g.q[1]);
      o.gates.push_back(g);
      continue;
    }
    if (g.kind == TN_GATE_SWAP) {
      std::swap(pend[(size_t)g.q[0]], pend[(size_t)g.q[1]]);
      o.gates.push_back(g);
      continue;
    }
    if (g.kind == KIND_F2 && (pend[(size_t)g.q[0]].on || pend[(size_t)g.q[1]].on)) {
      // a fused block is a dense 4x4 anyway: the pending phases become its first members
      TnGate f = g;
      f.fuse_begin = (int)fused.size();
      for (int r = 0; r < 2; ++r) {
        Pending &pp = pend[(size_t)g.q[r]];
        if (!pp.on) continue;
        FusedMember m;
        std::memset(&m, 0, sizeof(m));
        m.kind = KIND_P;
        m.role = r == 0 ? ROLE_A : ROLE_B;
        for (int a = 0; a < 3; ++a) m.pidx[a][0] = m.pidx[a][1] = -1;
        m.angle[0] = pp.val;
        m.pidx[0][0] = pp.idx;
        fused.push_back(m);
        pp = Pending();
      }
      for (int k = 0; k < g.fuse_count; ++k) fused.push_back(fused[(size_t)(g.fuse_begin + k)]);
      f.fuse_count = (int)fused.size() - f.fuse_begin;  // at most kMaxFusedMembers (fuse_pairs leaves room)
      o.gates.push_back(f);
      continue;
    }
    emit_p(g.q[0]);
    if (gate_nqubits(g.kind) == 2) emit_p(g.q[1]);
    o.gates.push_back(g);
  }
  for (int q = 0; q < c.n; ++q) emit_p(q);
  return o;
}

tn_status build_pass_plan(const tn_circuit &c, int T, int K, bool adjoint, std::vector<MatSlot> &slots,
                          PassPlan &out, std::string &err) {
  Planner P;
  P.N = c.n;
  P.T = T;
  P.K = K;
  const int G = (int)c.gates.size();
  P.cls.resize(G);
  for (int i = 0; i < G; ++i) P.cls[i] = classify(c.gates[i]);
  P.order.resize(G);
  for (int i = 0; i < G; ++i) P.order[i] = adjoint ? G - 1 - i : i;
  P.done.assign(G, 0);

  out = PassPlan();
  const int N = c.n;
  std::vector<int> pending = P.order;
  int first_pass = 1;
  // per-gate matrix slot offsets (allocated lazily, once per gate and form)
  auto add_slot = [&](int gi, int form, int shape) -> int {
    MatSlot s;
    std::memset(&s, 0, sizeof(s));
    const TnGate &g = c.gates[gi];
    s.kind = g.kind;
    s.form = form;
    s.shape = shape;
    for (int a = 0; a < 3; ++a) {
      s.angle[a] = g.angle[a];
      s.pidx[a][0] = g.pidx[a][0];
      s.pidx[a][1] = g.pidx[a][1];
    }
    for (int a = 0; a < 32; ++a) s.fixed[a] = g.mat[a];
    s.fuse_begin = g.fuse_begin;
    s.fuse_count = g.fuse_count;
    int off = 0;
    if (!slots.empty()) {
      const MatSlot &l = slots.back();
      off = l.offset + ((shape_entries(l.shape) + 1) & ~1);  // 16-byte aligned entries
    }
    s.offset = off;
    slots.push_back(s);
    return off;
  };

  while (!pending.empty() || (first_pass && !adjoint)) {
    // ---- 1. tile bits
    uint64_t S = 0;
    int nS = 0;
    if (N <= T) {
      S = (N == 64) ? ~0ull : ((1ull << N) - 1);
      nS = N;
    } else {
      for (int b = 0; b < kLowBits; ++b) S |= bitmask(b);
      nS = kLowBits;
      uint64_t blockedq = 0;  // bitmask over qubits
      std::vector<int> wish;  // bits wanted by deferred gates, for filling
      for (int g : pending) {
        int qs[2], nq;
        P.qubits(g, qs, nq);
        bool blk = false;
        for (int i = 0; i < nq; ++i) blk |= (blockedq >> qs[i]) & 1;
        int nb[2];
        int nn = P.needs(g, nb);
        if (!blk) {
          int add = 0;
          for (int i = 0; i < nn; ++i) add += ((S >> nb[i]) & 1) ? 0 : 1;
          if (nS + add <= T) {
            for (int i = 0; i < nn; ++i) if (!((S >> nb[i]) & 1)) { S |= bitmask(nb[i]); ++nS; }
            continue;
          }
        }
        for (int i = 0; i < nn; ++i) wish.push_back(nb[i]);
        for (int i = 0; i < nq; ++i) blockedq |= 1ull << qs[i];
      }
      for (int b : wish) {
        if (nS >= T) break;
        if (!((S >> b) & 1)) { S |= bitmask(b); ++nS; }
      }
      for (int b = kLowBits; b < N && nS < T; ++b)
        if (!((S >> b) & 1)) { S |= bitmask(b); ++nS; }
    }
    PassDesc pd;
    std::memset(&pd, 0, sizeof(pd));
    pd.T = nS;
    pd.K = std::min(K, nS);
    pd.init_mode = (!adjoint && first_pass) ? 1 : 0;
    int tl = 0, ol = 0;
    int glob2tile[64];
    for (int b = 0; b < 64; ++b) glob2tile[b] = -1;
    for (int b = 0; b < N; ++b) {
      if ((S >> b) & 1) { glob2tile[b] = tl; pd.tile_pos[tl++] = (uint8_t)b; }
      else pd.outer_pos[ol++] = (uint8_t)b;
    }
    pd.n_outer = ol;
    pd.phase_begin = (int)out.phases.size();
    pd.grad_begin = (int)out.grads.size();
    int pass_code = 0;      // estimated instructions of this pass's specialised kernel
    bool pass_full = false;  // the code budget is used up: the remaining gates go to the next pass
    pd.mat_begin = slots.empty() ? 0 : slots.back().offset + ((shape_entries(slots.back().shape) + 1) & ~1);
    const int Kp = pd.K;
    int grad_slots = 0;

    // ---- 2. phases
    for (;;) {
      if (pending.empty() || pass_full) break;
      // choose register bits R (global positions) among S
      uint64_t R = 0;
      int nR = 0;
      uint64_t blockedq = 0;
      for (int g : pending) {
        int qs[2], nq;
        P.qubits(g, qs, nq);
        bool blk = false;
        for (int i = 0; i < nq; ++i) blk |= (blockedq >> qs[i]) & 1;
        int nb[2];
        int nn = P.needs(g, nb);
        bool ok = !blk;
        for (int i = 0; i < nn && ok; ++i) ok = (S >> nb[i]) & 1;
        if (ok) {
          int add = 0;
          for (int i = 0; i < nn; ++i) add += ((R >> nb[i]) & 1) ? 0 : 1;
          if (nR + add <= Kp) {
            for (int i = 0; i < nn; ++i) if (!((R >> nb[i]) & 1)) { R |= bitmask(nb[i]); ++nR; }
            continue;
          }
        }
        for (int i = 0; i < nq; ++i) blockedq |= 1ull << qs[i];
      }
      for (int b = N - 1; b >= 0 && nR < Kp; --b)  // fill from the high tile bits
        if (((S >> b) & 1) && !((R >> b) & 1)) { R |= bitmask(b); ++nR; }

      // emit ops
      PhaseDesc ph;
      std::memset(&ph, 0, sizeof(ph));
      ph.op_begin = (int)out.ops.size();
      int regpos_of_bit[64];
      for (int b = 0; b < 64; ++b) regpos_of_bit[b] = -1;
      {
        int r = 0;
        for (int b = 0; b < N; ++b)
          if ((R >> b) & 1) { ph.reg_pos[r] = (uint8_t)glob2tile[b]; regpos_of_bit[b] = r; ++r; }
      }
      // thread-index bits: non-register tile positions; lanes first, chosen so that the
      // residues (position mod 4) of the first five cover 0..3 when possible
      {
        std::vector<int> rest;
        for (int l = 0; l < nS; ++l) {
          int b = pd.tile_pos[l];
          if (!((R >> b) & 1)) rest.push_back(l);
        }
        std::vector<int> lanes, others;
        std::vector<char> used(rest.size(), 0);
        for (int res = 0; res < 4 && (int)lanes.size() < 5; ++res)
          for (size_t i = 0; i < rest.size(); ++i)
            if (!used[i] && (rest[i] & 3) == res) { lanes.push_back(rest[i]); used[i] = 1; break; }
        for (size_t i = 0; i < rest.size() && lanes.size() < 5; ++i)
          if (!used[i]) { lanes.push_back(rest[i]); used[i] = 1; }
        for (size_t i = 0; i < rest.size(); ++i) if (!used[i]) others.push_back(rest[i]);
        int t = 0;
        for (int l : lanes) ph.thr_pos[t++] = (uint8_t)l;
        for (int l : others) ph.thr_pos[t++] = (uint8_t)l;
      }
      auto src_of = [&](int q, uint8_t &kind, uint8_t &pos) {
        int b = P.bit_of(q);
        if (regpos_of_bit[b] >= 0) { kind = SRC_REG; pos = (uint8_t)regpos_of_bit[b]; }
        else if (glob2tile[b] >= 0) { kind = SRC_TILE; pos = (uint8_t)glob2tile[b]; }
        else { kind = SRC_GLOB; pos = (uint8_t)b; }
      };
      int emitted = 0;
      uint32_t pending_sign_bits = 0;  // register positions the accumulated CZ signs depend on
      blockedq = 0;
      std::vector<int> rest_pending;
      rest_pending.reserve(pending.size());
      for (int g : pending) {
        int qs[2], nq;
        P.qubits(g, qs, nq);
        bool blk = false;
        for (int i = 0; i < nq; ++i) blk |= (blockedq >> qs[i]) & 1;
        int nb[2];
        int nn = P.needs(g, nb);
        bool ok = !blk;
        for (int i = 0; i < nn && ok; ++i) ok = (R >> nb[i]) & 1;
        if (ok && !pass_full) {
          const GateCls &gq = P.cls[g];
          const TnGate &tq = c.gates[g];
          const bool hg = adjoint && tq.param_idx >= 0;
          const int cost = op_code_cost(gq.type, tq.kind, adjoint, hg, hg ? gate_arity(tq.kind) : 0);
          if (pass_code > 0 && pass_code + cost > kPassCodeBudget) pass_full = true;
          else pass_code += cost;
        }
        if (pass_full) ok = false;
        // a pass accumulates at most kMaxGradSlots parameter derivatives per tile
        if (ok && adjoint && c.gates[g].param_idx >= 0 &&
            grad_slots + gate_arity(c.gates[g].kind) > kMaxGradSlots)
          ok = false;
        if (!ok) {
          for (int i = 0; i < nq; ++i) blockedq |= 1ull << qs[i];
          rest_pending.push_back(g);
          continue;
        }
        const GateCls &gc = P.cls[g];
        OpDesc op;
        std::memset(&op, 0, sizeof(op));
        op.type = (uint8_t)gc.type;
        if (gc.shape == SHAPE_M4X) op.flags |= OPF_PACKED;
        if (c.gates[g].kind == TN_GATE_SWAP) op.flags |= OPF_SWAP;
        src_of(gc.qa, op.a_kind, op.a_pos);
        if (gc.qb >= 0) src_of(gc.qb, op.b_kind, op.b_pos);
        op.mat = gc.shape >= 0 ? add_slot(g, adjoint ? FORM_ADJ : FORM_U, gc.shape) : 0;
        op.aux = -1;
        const TnGate &tg = c.gates[g];
        if (adjoint && tg.param_idx >= 0) {
          int ar = gate_arity(tg.kind);
          op.has_grad = 1;
          op.n_grad = (uint8_t)ar;
          op.aux = (int)out.grads.size();
          for (int a = 0; a < ar; ++a) {
            // the derivative matrix applied to psi (same structure as the gate) and the real
            // part of <lambda|.> (two FMAs per amplitude)
            out.grad_flops += (op_flops(gc.type, tg.kind) + 4.0) * (double)(1ull << N);
            GradRec gr;
            gr.mat = add_slot(g, FORM_D0 + a, gc.shape);
            gr.param = tg.param_idx + a;
            gr.slot = grad_slots++;
            gr.pad = 0;
            out.grads.push_back(gr);
          }
        }
        if (gc.type == OP_CZ) {
          if (op.a_kind == SRC_REG) pending_sign_bits |= 1u << op.a_pos;
          if (op.b_kind == SRC_REG) pending_sign_bits |= 1u << op.b_pos;
        } else if (gc.type == OP_G1 || gc.type == OP_G2 || gc.type == OP_C1) {
          uint32_t touched = 0;
          if (gc.type == OP_G1) touched = 1u << op.a_pos;
          if (gc.type == OP_G2) touched = (1u << op.a_pos) | (1u << op.b_pos);
          if (gc.type == OP_C1) touched = 1u << op.b_pos;
          // signs that depend only on other bits commute with this op; otherwise apply them first
          if ((pending_sign_bits & touched) || (adjoint && op.has_grad)) {
            op.flags |= OPF_FLUSH;
            pending_sign_bits = 0;
          }
        }
        out.ops.push_back(op);
        out.op_gate.push_back(g);
        // the first pass computes only the tile that holds the basis state
        out.flops += op_flops(gc.type, c.gates[g].kind) * (double)(1ull << (pd.init_mode ? nS : N));
        ++emitted;
      }
      if (emitted == 0) break;
      ph.op_end = (int)out.ops.size();
      out.phases.push_back(ph);
      pending.swap(rest_pending);
    }
    pd.phase_end = (int)out.phases.size();
    pd.op_begin = pd.phase_begin < pd.phase_end ? out.phases[pd.phase_begin].op_begin : (int)out.ops.size();
    pd.op_end = (int)out.ops.size();
    pd.grad_slots = grad_slots;
    out.max_grad_slots = std::max(out.max_grad_slots, grad_slots);
    pd.mat_end = slots.empty() ? 0 : slots.back().offset + ((shape_entries(slots.back().shape) + 1) & ~1);
    if (pd.mat_end < pd.mat_begin) pd.mat_end = pd.mat_begin;
    if (pd.phase_end == pd.phase_begin && !pd.init_mode) {
      err = "planner made no progress (internal error)";
      return TN_ERR_UNSUPPORTED;
    }
    out.passes.push_back(pd);
    first_pass = 0;
  }
  return TN_OK;
}

}  // namespace tnq
