// Internal declarations of libtnq shared by the host planner and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <complex>
#include <string>
#include <vector>

#include "../../include/tn.h"

#if defined(__CUDACC__)
#define TNQ_HD __host__ __device__ __forceinline__
#else
#define TNQ_HD inline
#endif

namespace tnq {

constexpr int kMaxQubits = 34;   // 2^34 complex64 = 128 GiB, the largest state one GB300 holds twice
constexpr int kMaxTile = 13;     // qubits per on-chip tile (2^13 complex64 = 64 KiB of shared memory)
constexpr int kLowBits = 4;      // the lowest bits always inside a tile: runs of 16 amplitudes = 128 B
constexpr int kMaxReg = 4;       // register qubits per thread and phase (2^4 amplitudes)
constexpr int kMaxGradSlots = 256;  // parameter derivatives accumulated per pass of the adjoint sweep

// ---------------------------------------------------------------------------------------
// Register-level operations of the fused gate-apply kernel.
//
// A pass loads one tile of 2^T amplitudes (T tile bits) into shared memory, runs a list of
// phases and writes the tile back.  In a phase every thread holds 2^K amplitudes in
// registers whose tile-local indices differ in the K "register" bits; an op then touches
// only registers.  Bit operands of an op are named by where their value comes from:
//   SRC_REG  - register bit r (the value differs between a thread's amplitudes)
//   SRC_TILE - tile-local bit l that is a thread-index bit in this phase (one value per thread)
//   SRC_GLOB - global bit p outside the tile (one value per tile)
// ---------------------------------------------------------------------------------------
enum OpType : uint8_t {
  OP_G1 = 1,  // general 2x2 on register bit a                          (4 matrix entries)
  OP_G2 = 2,  // general 4x4 on register bits a (high), b (low)         (16 entries)
  OP_C1 = 3,  // 2x2 on register bit b where bit a (any source) is 1   (4 entries)
  OP_D1 = 4,  // diagonal diag(d0, d1) on bit a (any source)            (2 entries)
  OP_CZ = 5,  // sign flip where bits a and b are both 1                (0 entries)
  OP_DP = 6,  // phase e where bits a and b are both 1                  (1 entry)
};
enum SrcKind : uint8_t { SRC_REG = 0, SRC_TILE = 1, SRC_GLOB = 2 };
enum OpFlags : uint8_t {
  OPF_FLUSH = 1,   // apply the pending CZ signs first
  OPF_PACKED = 2,  // OP_G2 entries in the packed layout of SHAPE_M4X
  OPF_SWAP = 4,    // OP_G2 of a SWAP: an exchange of registers, its entries are not read
};

struct alignas(16) OpDesc {
  uint8_t type;
  uint8_t a_kind, a_pos;
  uint8_t b_kind, b_pos;
  uint8_t has_grad;  // adjoint sweep: this op carries a parameter derivative
  uint8_t n_grad;    // number of derivative forms (angles) that follow at aux
  uint8_t flags;     // OPF_FLUSH: apply the pending CZ signs first (they touch this op's register bits)
  int32_t mat;       // offset (complex64 units) of the op's entries in a batch's matrix table
  int32_t aux;       // adjoint sweep: index of the first derivative record (GradRec) or -1
};
static_assert(sizeof(OpDesc) == 16, "OpDesc layout");

// One derivative of an op w.r.t. one parameter (adjoint sweep).
struct alignas(16) GradRec {
  int32_t mat;    // offset of the derivative entries dU/da (same shape as the op's entries)
  int32_t param;  // parameter index k in params[b][k]
  int32_t slot;   // per-tile accumulation slot
  int32_t pad;
};

struct alignas(16) PhaseDesc {
  int32_t op_begin, op_end;
  uint8_t reg_pos[8];   // K tile-local positions of the register bits
  uint8_t thr_pos[16];  // T-K tile-local positions of the thread-index bits (lane bits first)
};

struct alignas(16) PassDesc {
  int32_t T, K;
  int32_t phase_begin, phase_end;
  int32_t init_mode;  // 1: the tile is synthesised from the initial basis state instead of loaded
  int32_t n_outer;    // N - T
  int32_t grad_slots; // adjoint sweep: accumulation slots used by this pass
  int32_t grad_begin; // adjoint sweep: index of the pass's first GradRec (slot s = record grad_begin + s)
  int32_t op_begin, op_end;    // the pass's ops (contiguous)
  int32_t mat_begin, mat_end;  // the pass's matrix-table entries (contiguous, complex64 units)
  uint8_t tile_pos[16];   // tile-local bit -> global bit (tile_pos[i] = i for i < kLowBits)
  uint8_t outer_pos[40];  // outer (tile-index) bit -> global bit, ascending
};

// How one entry range of a batch's matrix table is produced from the parameters.
enum MatForm : int32_t { FORM_U = 0, FORM_ADJ = 1, FORM_D0 = 2, FORM_D1 = 3, FORM_D2 = 4 };
// Entry layouts per op type: G1/C1 2x2 row-major, G2 4x4, D1 (d0, d1), DP (phase).  SHAPE_M4X is
// the 4x4 of a fused block laid out for packed FP32x2 arithmetic: entry k = (re, im) becomes the
// four floats (re, re, -im, im), so that u * v = (re, re) * (v.re, v.im) + (-im, im) * (v.im, v.re)
// reads both packed factors straight from one 16-byte load.
enum MatShape : int32_t { SHAPE_M2 = 0, SHAPE_M4 = 1, SHAPE_DIAG2 = 2, SHAPE_PHASE = 3, SHAPE_M4X = 4 };

// complex64 units a slot of the given shape occupies
TNQ_HD int shape_units(int shape) {
  switch (shape) {
    case SHAPE_M2: return 4;
    case SHAPE_M4: return 16;
    case SHAPE_DIAG2: return 2;
    case SHAPE_PHASE: return 1;
    case SHAPE_M4X: return 32;
  }
  return 0;
}

struct alignas(16) MatSlot {
  int32_t kind;       // tn_gate_kind or an internal kind (KIND_V, KIND_P, KIND_F2)
  int32_t form;       // MatForm
  int32_t shape;      // MatShape
  int32_t offset;     // destination offset (complex64 units)
  int32_t pidx[3][2]; // angle a = angle[a] + sum of params[pidx[a][k]] over pidx >= 0
  int32_t fuse_begin, fuse_count;  // KIND_F2: its member gates in the plan's FusedMember table
  double angle[3];
  double pad2;
  double fixed[32];   // MAT1/MAT2 entries (re, im)
};

// Internal gate kinds produced by the planner (never in the ABI):
//   V(t, a) = RY(t) P(a) = [[cos t/2, -sin t/2 e^{ia}], [sin t/2, cos t/2 e^{ia}]]
//   P(a)    = diag(1, e^{ia})
// so that U3(t, p, l) = P(p) V(t, l) (the phase-pushing rewrite); and
//   F2      = the product of a run of gates on two qubits (a, b), precontracted into one 4x4
//             matrix indexed 2 bit(a) + bit(b) (Sec. 3: small contractions computed ahead so
//             that the tensors applied are square matrices of one size).  Its members are
//             listed in the plan's FusedMember table; the product is formed per call from
//             the parameters, in FP64.
constexpr int KIND_V = 64;
constexpr int KIND_P = 65;
constexpr int KIND_F2 = 66;
constexpr int kMaxFusedMembers = 24;  // gates precontracted into one F2 at most
// Parameterised circuits are precontracted into 4x4 blocks from this many qubits on: each block's
// FP64 product per call and batch element costs more than the passes save on smaller states
// (measured on a 10-qubit brickwork with 512 parameter sets: 59 us per call fused, 37 unfused).
constexpr int kFuseMinQubitsParam = 14;

// One gate of a fused block: its kind, which of the block's qubits it acts on, its angles.
enum FuseRole : int32_t { ROLE_A = 0, ROLE_B = 1, ROLE_AB = 2, ROLE_BA = 3 };
struct alignas(16) FusedMember {
  int32_t kind;        // tn_gate_kind, KIND_V or KIND_P
  int32_t role;        // FuseRole: one-qubit on a / on b, two-qubit on (a, b) / on (b, a)
  int32_t pidx[3][2];  // angle a = angle[a] + sum of params[pidx[a][k]] over pidx >= 0
  double angle[3];
  double pad;
  double mat[32];      // MAT1 / MAT2 entries (re, im)
};

// ---------------------------------------------------------------------------------------
// Gate matrices in double precision (shared by the plan-time host path and the per-call
// device path).  Formulas: see include/tn.h.  out holds (re, im) pairs, row-major.
// ---------------------------------------------------------------------------------------
TNQ_HD void cset(double *o, int i, double re, double im) { o[2 * i] = re; o[2 * i + 1] = im; }

// sin and cos of one angle with one shared argument reduction on the device (FP64 is slow on this
// GPU, and every gate table is built per call from the parameters).
TNQ_HD void sincos2(double x, double *s, double *c) {
#if defined(__CUDA_ARCH__)
  sincos(x, s, c);
#else
  *s = std::sin(x);
  *c = std::cos(x);
#endif
}

// Full 2x2 / 4x4 matrix of a gate kind (form FORM_U), or its derivative w.r.t. angle a
// (FORM_D0 + a).  Returns the dimension (2 or 4); 0 for an unknown kind.
TNQ_HD int gate_nqubits(int kind) {
  return (kind == TN_GATE_CZ || kind == TN_GATE_CNOT || kind == TN_GATE_CP || kind == TN_GATE_SWAP ||
          kind == TN_GATE_MAT2 || kind == KIND_F2) ? 2 : 1;
}

TNQ_HD int gate_matrix(int kind, int form, const double *ang, const double *fixed, double *o) {
  const double r2 = 0.70710678118654752440;
  int dim = gate_nqubits(kind) == 2 ? 4 : 2;
  for (int i = 0; i < 2 * dim * dim; ++i) o[i] = 0.0;
  const bool deriv = form >= FORM_D0;
  const int a = form - FORM_D0;
  switch (kind) {
    case TN_GATE_H: cset(o, 0, r2, 0); cset(o, 1, r2, 0); cset(o, 2, r2, 0); cset(o, 3, -r2, 0); break;
    case TN_GATE_X: cset(o, 1, 1, 0); cset(o, 2, 1, 0); break;
    case TN_GATE_Y: cset(o, 1, 0, -1); cset(o, 2, 0, 1); break;
    case TN_GATE_Z: cset(o, 0, 1, 0); cset(o, 3, -1, 0); break;
    case TN_GATE_S: cset(o, 0, 1, 0); cset(o, 3, 0, 1); break;
    case TN_GATE_SDG: cset(o, 0, 1, 0); cset(o, 3, 0, -1); break;
    case TN_GATE_T: cset(o, 0, 1, 0); cset(o, 3, r2, r2); break;
    case TN_GATE_TDG: cset(o, 0, 1, 0); cset(o, 3, r2, -r2); break;
    case TN_GATE_SX:  // RX(pi/2)
      cset(o, 0, r2, 0); cset(o, 1, 0, -r2); cset(o, 2, 0, -r2); cset(o, 3, r2, 0); break;
    case TN_GATE_SY:  // RY(pi/2)
      cset(o, 0, r2, 0); cset(o, 1, -r2, 0); cset(o, 2, r2, 0); cset(o, 3, r2, 0); break;
    case TN_GATE_SW:  // cos(pi/4) I - i sin(pi/4) (X+Y)/sqrt2
      cset(o, 0, r2, 0); cset(o, 1, -0.5, -0.5); cset(o, 2, 0.5, -0.5); cset(o, 3, r2, 0); break;
    case TN_GATE_RX: {
      double c, s;
      sincos2(ang[0] * 0.5, &s, &c);
      if (!deriv) { cset(o, 0, c, 0); cset(o, 1, 0, -s); cset(o, 2, 0, -s); cset(o, 3, c, 0); }
      else { cset(o, 0, -0.5 * s, 0); cset(o, 1, 0, -0.5 * c); cset(o, 2, 0, -0.5 * c); cset(o, 3, -0.5 * s, 0); }
      break;
    }
    case TN_GATE_RY: {
      double c, s;
      sincos2(ang[0] * 0.5, &s, &c);
      if (!deriv) { cset(o, 0, c, 0); cset(o, 1, -s, 0); cset(o, 2, s, 0); cset(o, 3, c, 0); }
      else { cset(o, 0, -0.5 * s, 0); cset(o, 1, -0.5 * c, 0); cset(o, 2, 0.5 * c, 0); cset(o, 3, -0.5 * s, 0); }
      break;
    }
    case TN_GATE_RZ: {
      double c, s;
      sincos2(ang[0] * 0.5, &s, &c);
      if (!deriv) { cset(o, 0, c, -s); cset(o, 3, c, s); }
      else { cset(o, 0, -0.5 * s, -0.5 * c); cset(o, 3, -0.5 * s, 0.5 * c); }
      break;
    }
    case TN_GATE_U3: {
      double c, s, cp, sp, cl, sl;
      sincos2(ang[0] * 0.5, &s, &c);
      sincos2(ang[1], &sp, &cp);
      sincos2(ang[2], &sl, &cl);
      const double cpl = cp * cl - sp * sl, spl = sp * cl + cp * sl;  // e^{i(p+l)}
      if (!deriv) {
        cset(o, 0, c, 0); cset(o, 1, -cl * s, -sl * s); cset(o, 2, cp * s, sp * s); cset(o, 3, cpl * c, spl * c);
      } else if (a == 0) {
        cset(o, 0, -0.5 * s, 0); cset(o, 1, -0.5 * cl * c, -0.5 * sl * c);
        cset(o, 2, 0.5 * cp * c, 0.5 * sp * c); cset(o, 3, -0.5 * cpl * s, -0.5 * spl * s);
      } else if (a == 1) {  // i e^{ip} s, i e^{i(p+l)} c in the bottom row
        cset(o, 2, -sp * s, cp * s); cset(o, 3, -spl * c, cpl * c);
      } else {              // -i e^{il} s top right, i e^{i(p+l)} c bottom right
        cset(o, 1, sl * s, -cl * s); cset(o, 3, -spl * c, cpl * c);
      }
      break;
    }
    case TN_GATE_CZ: cset(o, 0, 1, 0); cset(o, 5, 1, 0); cset(o, 10, 1, 0); cset(o, 15, -1, 0); break;
    case TN_GATE_CNOT: cset(o, 0, 1, 0); cset(o, 5, 1, 0); cset(o, 11, 1, 0); cset(o, 14, 1, 0); break;
    case TN_GATE_CP: {
      double c, s;
      sincos2(ang[0], &s, &c);
      if (!deriv) { cset(o, 0, 1, 0); cset(o, 5, 1, 0); cset(o, 10, 1, 0); cset(o, 15, c, s); }
      else { cset(o, 15, -s, c); }
      break;
    }
    case TN_GATE_SWAP: cset(o, 0, 1, 0); cset(o, 6, 1, 0); cset(o, 9, 1, 0); cset(o, 15, 1, 0); break;
    case TN_GATE_MAT1: for (int i = 0; i < 8; ++i) o[i] = fixed[i]; break;
    case KIND_V: {
      double c, s, ca, sa;
      sincos2(ang[0] * 0.5, &s, &c);
      sincos2(ang[1], &sa, &ca);
      cset(o, 0, c, 0); cset(o, 1, -s * ca, -s * sa); cset(o, 2, s, 0); cset(o, 3, c * ca, c * sa);
      break;
    }
    case KIND_P: {
      double c, s;
      sincos2(ang[0], &s, &c);
      cset(o, 0, 1, 0);
      cset(o, 3, c, s);
      break;
    }
    case TN_GATE_MAT2: for (int i = 0; i < 32; ++i) o[i] = fixed[i]; break;
    default: return 0;
  }
  return dim;
}

// Number of angles a kind reads.
TNQ_HD int gate_arity(int kind) {
  return kind == TN_GATE_U3 ? 3 : kind == KIND_V ? 2
       : (kind == TN_GATE_RX || kind == TN_GATE_RY || kind == TN_GATE_RZ || kind == TN_GATE_CP || kind == KIND_P) ? 1 : 0;
}

// Entries of a matrix slot: the full matrix in the shape the op consumes, optionally
// conjugate-transposed (FORM_ADJ).  Writes complex64 (float2) entries to dst.
TNQ_HD int slot_entries(const MatSlot &s, const double *ang, double *tmp /*32*/, float *dst) {
  int form = s.form == FORM_ADJ ? FORM_U : s.form;
  int dim = gate_matrix(s.kind, form, ang, s.fixed, tmp);
  bool adj = s.form == FORM_ADJ;
  auto put = [&](int k, int i, int j) {  // dst entry k <- (adj ? conj(m[j][i]) : m[i][j])
    int src = adj ? (j * dim + i) : (i * dim + j);
    dst[2 * k] = (float)tmp[2 * src];
    dst[2 * k + 1] = (float)(adj ? -tmp[2 * src + 1] : tmp[2 * src + 1]);
  };
  switch (s.shape) {
    case SHAPE_M2:
      if (dim == 2) { put(0, 0, 0); put(1, 0, 1); put(2, 1, 0); put(3, 1, 1); return 4; }
      // controlled 2x2: the lower-right block of the 4x4
      put(0, 2, 2); put(1, 2, 3); put(2, 3, 2); put(3, 3, 3); return 4;
    case SHAPE_M4:
      for (int i = 0; i < 4; ++i) for (int j = 0; j < 4; ++j) put(4 * i + j, i, j);
      return 16;
    case SHAPE_DIAG2: put(0, 0, 0); put(1, 1, 1); return 2;
    case SHAPE_PHASE: put(0, 3, 3); return 1;
  }
  return 0;
}


// M <- G M for one member of a fused block, M a 4x4 indexed 2 bit(a) + bit(b) (FP64 (re, im)
// pairs): a one-qubit member mixes pairs of rows (half the work of a dense product), a diagonal
// two-qubit member scales rows, any other two-qubit member is a dense product.
TNQ_HD void fused_apply_member(const FusedMember &f, const double *param_row, double *M /*32*/) {
  double ang[3] = {f.angle[0], f.angle[1], f.angle[2]};
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < 2; ++k)
      if (f.pidx[a][k] >= 0 && param_row) ang[a] += param_row[f.pidx[a][k]];
  double g[32];
  const int dim = gate_matrix(f.kind, FORM_U, ang, f.mat, g);
  if (dim == 2) {
    const int step = f.role == ROLE_A ? 2 : 1;  // rows i and i + step differ in the member's qubit
    for (int i = 0; i < 4; ++i) {
      if (i & step) continue;
      const int i1 = i + step;
      for (int j = 0; j < 4; ++j) {
        const double xr = M[2 * (4 * i + j)], xi = M[2 * (4 * i + j) + 1];
        const double yr = M[2 * (4 * i1 + j)], yi = M[2 * (4 * i1 + j) + 1];
        M[2 * (4 * i + j)] = g[0] * xr - g[1] * xi + g[2] * yr - g[3] * yi;
        M[2 * (4 * i + j) + 1] = g[0] * xi + g[1] * xr + g[2] * yi + g[3] * yr;
        M[2 * (4 * i1 + j)] = g[4] * xr - g[5] * xi + g[6] * yr - g[7] * yi;
        M[2 * (4 * i1 + j) + 1] = g[4] * xi + g[5] * xr + g[6] * yi + g[7] * yr;
      }
    }
    return;
  }
  // the member's own index is 2 bit(first) + bit(second); ROLE_BA swaps the two bits
  auto perm = [&](int i) { return f.role == ROLE_AB ? i : ((i & 1) << 1) | (i >> 1); };
  bool diag = true;
  for (int i = 0; i < 4 && diag; ++i)
    for (int j = 0; j < 4; ++j)
      if (i != j && (g[2 * (4 * i + j)] != 0.0 || g[2 * (4 * i + j) + 1] != 0.0)) diag = false;
  if (diag) {
    for (int i = 0; i < 4; ++i) {
      const int ii = perm(i);
      const double dr = g[2 * (5 * ii)], di = g[2 * (5 * ii) + 1];
      for (int j = 0; j < 4; ++j) {
        const double xr = M[2 * (4 * i + j)], xi = M[2 * (4 * i + j) + 1];
        M[2 * (4 * i + j)] = dr * xr - di * xi;
        M[2 * (4 * i + j) + 1] = dr * xi + di * xr;
      }
    }
    return;
  }
  double r[32];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double re = 0.0, im = 0.0;
      for (int q = 0; q < 4; ++q) {
        const double ur = g[2 * (4 * perm(i) + perm(q))], ui = g[2 * (4 * perm(i) + perm(q)) + 1];
        const double xr = M[2 * (4 * q + j)], xi = M[2 * (4 * q + j) + 1];
        re += ur * xr - ui * xi;
        im += ur * xi + ui * xr;
      }
      r[2 * (4 * i + j)] = re;
      r[2 * (4 * i + j) + 1] = im;
    }
  for (int i = 0; i < 32; ++i) M[i] = r[i];
}

// One member of a fused block as a 4x4 on (a, b), indexed 2 bit(a) + bit(b), FP64 (re, im) pairs.
TNQ_HD void fused_embed(const FusedMember &f, const double *param_row, double *e /*32*/) {
  double ang[3] = {f.angle[0], f.angle[1], f.angle[2]};
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < 2; ++k)
      if (f.pidx[a][k] >= 0 && param_row) ang[a] += param_row[f.pidx[a][k]];
  double g[32];
  const int dim = gate_matrix(f.kind, FORM_U, ang, f.mat, g);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      const int ia = i >> 1, ib = i & 1, ja = j >> 1, jb = j & 1;
      double re = 0.0, im = 0.0;
      if (dim == 2) {
        if (f.role == ROLE_A && ib == jb) { re = g[2 * (2 * ia + ja)]; im = g[2 * (2 * ia + ja) + 1]; }
        if (f.role == ROLE_B && ia == ja) { re = g[2 * (2 * ib + jb)]; im = g[2 * (2 * ib + jb) + 1]; }
      } else {
        // ROLE_BA: the member's first qubit is b, so its index is 2 bit(b) + bit(a)
        const int ii = f.role == ROLE_AB ? i : 2 * ib + ia, jj = f.role == ROLE_AB ? j : 2 * jb + ja;
        re = g[2 * (4 * ii + jj)];
        im = g[2 * (4 * ii + jj) + 1];
      }
      e[2 * (4 * i + j)] = re;
      e[2 * (4 * i + j) + 1] = im;
    }
}


}  // namespace tnq

// ---------------------------------------------------------------------------------------
// Host-side objects behind the opaque handles.
// ---------------------------------------------------------------------------------------
struct TnGate {
  int kind;
  int q[2];
  int param_idx;   // ABI parameter index (first angle), -1 if fixed; -1 for internal kinds
  int pidx[3][2];  // angle a = angle[a] + sum of params[pidx[a][k]] over pidx >= 0
  double angle[3];
  double mat[32];
  int fuse_begin, fuse_count;  // KIND_F2: members in the plan's FusedMember table (else 0, 0)
};

struct tn_circuit {
  int n;
  uint64_t init;
  int n_params;
  std::vector<TnGate> gates;
};

// One direction (forward or adjoint) of a fused pass plan.
struct PassPlan {
  std::vector<tnq::PassDesc> passes;
  std::vector<tnq::PhaseDesc> phases;
  std::vector<tnq::OpDesc> ops;
  std::vector<int> op_gate;  // circuit gate index of every op
  std::vector<tnq::GradRec> grads;
  double flops = 0;   // per batch element
  double grad_flops = 0;  // adjoint plans: derivative products and dots, per batch element
  int max_grad_slots = 0;
};

namespace tnq {
struct NetPlan;
}

namespace tnq {
// A gate of a fixed-point plan: the matrix rounded to Q4.28 (value q / 2^28), row-major,
// (re, im) interleaved; pos: state bits of the gate's qubits (first qubit first).
struct Q428Gate {
  int nq;
  int pos[2];
  int32_t u[32];
};
}  // namespace tnq

namespace tnq {
struct BlockPlan;
}

struct tn_plan {
  tnq::NetPlan *net = nullptr;  // TN_PLAN_NETWORK plans: pairwise network contraction
  tnq::BlockPlan *blocks = nullptr;  // TN_PLAN_BLOCKS plans: uniform square blocks
  std::vector<tnq::Q428Gate> *q428 = nullptr;  // TN_PLAN_Q428 plans: quantised gate list
  int n;
  long long n_gates;
  int batch;
  int n_params;
  uint64_t init;
  int T, K;
  tn_plan_opts opts;
  bool host_only;
  int device;
  std::vector<tnq::MatSlot> slots;  // forward + adjoint + derivative entries
  std::vector<tnq::FusedMember> fused;  // members of the forward plan's F2 gates
  int n_fused = 0;                      // F2 gates in the forward plan
  int n_fused_slots = 0;                // F2 slots (listed first in d_slots)
  int mstride;                      // complex64 entries per batch element's matrix table
  bool param_dependent;
  PassPlan fwd, bwd;
  // device copies (NULL when host_only)
  tnq::MatSlot *d_slots = nullptr;
  tnq::FusedMember *d_fused = nullptr;
  tnq::PassDesc *d_fwd_pass = nullptr, *d_bwd_pass = nullptr;
  tnq::PhaseDesc *d_fwd_phase = nullptr, *d_bwd_phase = nullptr;
  tnq::OpDesc *d_fwd_ops = nullptr, *d_bwd_ops = nullptr;
  tnq::GradRec *d_bwd_grads = nullptr;
  float *d_fixed_mats = nullptr;  // materialised once when !param_dependent
  // plan-specialised forward kernels (generated; empty when the interpreting kernel runs)
  std::vector<cudaLibrary_t> jit_libs;
  std::vector<cudaKernel_t> jit_kernels;
  std::vector<int> jit_threads, jit_grid;
  std::vector<size_t> jit_smem;
  std::vector<void *> jit_cm_ptr;    // per forward pass: device address of its __constant__ matrix table
  std::vector<size_t> jit_cm_bytes;  //   and the bytes the pass reads (copied before its launch)
  std::vector<cudaLibrary_t> jit_bwd_libs;
  std::vector<cudaKernel_t> jit_bwd_kernels;
  std::vector<int> jit_bwd_threads, jit_bwd_grid;
  std::vector<size_t> jit_bwd_smem;
  size_t ws_bytes = 0;
  // workspace layout (byte offsets)
  size_t ws_mats = 0, ws_psi = 0, ws_lam = 0, ws_part = 0, ws_gacc = 0;
};

namespace tnq {
// One Pauli term on the device: P|x> = i^ny (-1)^popc(x & zm) |x ^ xm>.
struct alignas(16) DevTerm {
  double coef;
  unsigned long long xm, zm;
  int32_t xl;   // xm in tile-local bit positions of the term's reduction pass
  int32_t ny;   // number of Y factors
};
static_assert(sizeof(DevTerm) == 32, "DevTerm layout");
// One tile pass of a Pauli-sum reduction: the terms whose flip bits all lie in the tile.
struct alignas(16) RedPass {
  int32_t T, n_outer;
  int32_t term_begin, term_end;
  uint8_t tile_pos[16];
  uint8_t outer_pos[40];
};
}  // namespace tnq

struct tn_observable {
  int n;
  int n_terms;
  int T;
  std::vector<tnq::DevTerm> terms;   // pass order
  std::vector<tnq::RedPass> passes;
  tnq::DevTerm *d_terms = nullptr;
  tnq::RedPass *d_passes = nullptr;
  int device = -1;
};

// ---------------------------------------------------------------------------------------
// Host helpers implemented in abi.cu / plan.cpp / kernels.
// ---------------------------------------------------------------------------------------
namespace tnq {
void set_error(const char *fmt, ...);
tn_status cuda_fail(cudaError_t e, const char *what);
tn_status build_pass_plan(const tn_circuit &c, int T, int K, bool adjoint, std::vector<MatSlot> &slots,
                          PassPlan &out, std::string &err);
tn_circuit push_phases(const tn_circuit &c, std::vector<FusedMember> &fused);
tn_circuit fuse_pairs(const tn_circuit &c, std::vector<FusedMember> &fused);
}  // namespace tnq
