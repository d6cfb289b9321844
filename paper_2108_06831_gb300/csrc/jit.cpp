// Plan-specialised fused gate-apply kernels, generated as CUDA C++ and compiled with NVRTC.
//
// The interpreting kernel (k_apply.cu) reads every op record at run time and dispatches on
// its type and register positions, which keeps the compiler from scheduling arithmetic
// across gates.  Here the planner's passes are turned into source in which each phase's
// register positions, shared-memory offsets, CZ sign patterns, control bits and the
// position of every matrix entry are constants, so one pass compiles to straight-line
// FFMA code.  Gate matrices still come from the per-call table (so parameterised circuits
// share the compiled code); they are staged in shared memory once per batch element.
//
// Compiled cubins are cached in-process by a 64-bit hash of the source, the NVRTC options and
// the NVRTC version, and on disk in $TNQ_CACHE_DIR (default ~/.cache/tnq) under the same key,
// so repeated plans of the same circuit structure skip compilation.
#include <nvrtc.h>
#include <sys/stat.h>
#include <sys/types.h>
#include <unistd.h>

#include <algorithm>
#include <cctype>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include "jit.h"
#include "tnq_internal.h"

namespace tnq {

namespace {

// Complex arithmetic of the generated kernels.  Each helper evaluates the same products and
// sums, in the same order, as the scalar form noted beside it, but on (re, im) pairs with the
// packed FP32x2 instructions (fma/mul.rn.f32x2, two independent IEEE operations per
// instruction), which halves the FMA-pipe instruction count of a gate.
const char *kPrelude = R"(
typedef unsigned long long u64;
struct __align__(8) c2 { float x, y; };
__device__ __forceinline__ u64 pk(float lo, float hi) { u64 r; asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi)); return r; }
__device__ __forceinline__ float2 up(u64 v) { float lo, hi; asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v)); return make_float2(lo, hi); }
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) { u64 d; asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c)); return d; }
__device__ __forceinline__ u64 mul2(u64 a, u64 b) { u64 d; asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b)); return d; }
__device__ __forceinline__ u64 add2(u64 a, u64 b) { u64 d; asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b)); return d; }
// a*x + b*y: re = a.x x.x - a.y x.y + b.x y.x - b.y y.y, im = a.x x.y + a.y x.x + b.x y.y + b.y y.x
__device__ __forceinline__ float2 cm2(float2 a, float2 x, float2 b, float2 y) {
  u64 t = mul2(pk(a.x, a.x), pk(x.x, x.y));
  t = fma2(pk(-a.y, a.y), pk(x.y, x.x), t);
  t = fma2(pk(b.x, b.x), pk(y.x, y.y), t);
  t = fma2(pk(-b.y, b.y), pk(y.y, y.x), t);
  return up(t);
}
// a*b: re = a.x b.x + (a.y)(-b.y), im = a.x b.y + a.y b.x (second product first)
__device__ __forceinline__ float2 cm(float2 a, float2 b) {
  return up(fma2(pk(a.x, a.x), pk(b.x, b.y), mul2(pk(a.y, a.y), pk(-b.y, b.x))));
}
__device__ __forceinline__ float2 ng(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return up(add2(pk(a.x, a.y), pk(b.x, b.y))); }
// r*x + b*y with r real
__device__ __forceinline__ float2 rc(float r, float2 x, float2 b, float2 y) {
  u64 t = mul2(pk(r, r), pk(x.x, x.y));
  t = fma2(pk(b.x, b.x), pk(y.x, y.y), t);
  t = fma2(pk(-b.y, b.y), pk(y.y, y.x), t);
  return up(t);
}
// r*x + s*y with r, s real
__device__ __forceinline__ float2 rr(float r, float2 x, float s, float2 y) {
  return up(fma2(pk(s, s), pk(y.x, y.y), mul2(pk(r, r), pk(x.x, x.y))));
}
// r*x + (i t)*y with r, t real
__device__ __forceinline__ float2 ri(float r, float2 x, float t, float2 y) {
  return up(fma2(pk(-t, t), pk(y.y, y.x), mul2(pk(r, r), pk(x.x, x.y))));
}
__device__ __forceinline__ float2 f2(float4 v, int hi) { return hi ? make_float2(v.z, v.w) : make_float2(v.x, v.y); }
__device__ __forceinline__ int swz(int i) { int h = i >> 4; h ^= h >> 4; h ^= h >> 8; return i ^ (h & 15); }
)";

uint64_t fnv1a(const std::string &s) {
  uint64_t h = 1469598103934665603ull;
  for (unsigned char c : s) {
    h ^= c;
    h *= 1099511628211ull;
  }
  return h;
}

int swz_host(int i) {
  int h = i >> 4;
  h ^= h >> 4;
  h ^= h >> 8;
  return i ^ (h & 15);
}

struct Emitter {
  std::ostringstream o;
  int K = 4;
  int R = 16;  // registers per thread
  void line(const std::string &s) { o << s << "\n"; }
};

// condition expression (thread- or tile-uniform) for a non-register bit operand
std::string cond_expr(uint8_t kind, uint8_t pos) {
  char b[96];
  if (kind == SRC_TILE) snprintf(b, sizeof b, "((tb >> %d) & 1)", (int)pos);
  else snprintf(b, sizeof b, "((int)((base >> %d) & 1ull))", (int)pos);
  return b;
}

void emit_op(Emitter &E, const OpDesc &op, int kind) {
  const int R = E.R;
  char buf[256];
  auto mat = [&](int k) {  // k-th complex entry of the op's matrix
    snprintf(buf, sizeof buf, "f2(M4[%d], %d)", (op.mat + k) >> 1, (op.mat + k) & 1);
    return std::string(buf);
  };
  switch (op.type) {
    case OP_G1: {
      const int r = op.a_pos;
      if (kind == TN_GATE_X) {  // permutation: swap register pairs
        for (int j = 0; j < R; ++j)
          if (!(j & (1 << r))) {
            snprintf(buf, sizeof buf, "{ const float2 t = a[%d]; a[%d] = a[%d]; a[%d] = t; }", j, j, j | (1 << r), j | (1 << r));
            E.line(buf);
          }
        return;
      }
      E.line("{ const float2 u00 = " + mat(0) + ", u01 = " + mat(1) + ", u10 = " + mat(2) + ", u11 = " + mat(3) + ";");
      // arithmetic specialised to the matrix structure the gate kind guarantees
      const char *pair_fmt;
      if (kind == KIND_V)  // real first column
        pair_fmt = "  { const float2 x = a[%d], y = a[%d]; a[%d] = rc(u00.x, x, u01, y); a[%d] = rc(u10.x, x, u11, y); }";
      else if (kind == TN_GATE_RY || kind == TN_GATE_H || kind == TN_GATE_SY)  // real matrix
        pair_fmt = "  { const float2 x = a[%d], y = a[%d]; a[%d] = rr(u00.x, x, u01.x, y); a[%d] = rr(u10.x, x, u11.x, y); }";
      else if (kind == TN_GATE_RX || kind == TN_GATE_SX)  // real diagonal, imaginary off-diagonal
        pair_fmt = "  { const float2 x = a[%d], y = a[%d]; a[%d] = ri(u00.x, x, u01.y, y); a[%d] = ri(u11.x, y, u10.y, x); }";
      else
        pair_fmt = "  { const float2 x = a[%d], y = a[%d]; a[%d] = cm2(u00, x, u01, y); a[%d] = cm2(u10, x, u11, y); }";
      for (int j = 0; j < R; ++j)
        if (!(j & (1 << r))) {
          const int j1 = j | (1 << r);
          snprintf(buf, sizeof buf, pair_fmt, j, j1, j, j1);
          E.line(buf);
        }
      E.line("}");
      return;
    }
    case OP_C1: {
      const int r = op.b_pos;
      const bool ctrl_reg = op.a_kind == SRC_REG;
      const bool is_x = kind == TN_GATE_CNOT;
      if (!ctrl_reg) E.line("if (" + cond_expr(op.a_kind, op.a_pos) + ") {");
      if (!is_x) E.line("{ const float2 u00 = " + mat(0) + ", u01 = " + mat(1) + ", u10 = " + mat(2) + ", u11 = " + mat(3) + ";");
      for (int j = 0; j < R; ++j) {
        if (j & (1 << r)) continue;
        if (ctrl_reg && !(j & (1 << op.a_pos))) continue;
        const int j1 = j | (1 << r);
        if (is_x) snprintf(buf, sizeof buf, "{ const float2 t = a[%d]; a[%d] = a[%d]; a[%d] = t; }", j, j, j1, j1);
        else
          snprintf(buf, sizeof buf,
                   "  { const float2 x = a[%d], y = a[%d]; a[%d] = cm2(u00, x, u01, y); a[%d] = cm2(u10, x, u11, y); }", j,
                   j1, j, j1);
        E.line(buf);
      }
      if (!is_x) E.line("}");
      if (!ctrl_reg) E.line("}");
      return;
    }
    case OP_G2: {
      const int ra = op.a_pos, rb = op.b_pos;
      if (kind == TN_GATE_SWAP) {
        for (int j = 0; j < R; ++j)
          if ((j & (1 << ra)) && !(j & (1 << rb))) {
            const int j2 = (j & ~(1 << ra)) | (1 << rb);
            snprintf(buf, sizeof buf, "{ const float2 t = a[%d]; a[%d] = a[%d]; a[%d] = t; }", j, j, j2, j2);
            E.line(buf);
          }
        return;
      }
      if (op.flags & OPF_PACKED) {
        // fused block: entries in the packed layout (re, re, -im, im); every output is a chain of
        // 8 packed multiply-adds, each input is swapped once for its 4 uses
        E.line("{");
        for (int k = 0; k < 16; ++k) {
          snprintf(buf, sizeof buf, "  const float4 e%d = M4[%d];", k, (op.mat >> 1) + k);
          E.line(buf);
        }
        for (int j = 0; j < R; ++j) {
          if (j & ((1 << ra) | (1 << rb))) continue;
          const int idx[4] = {j, j | (1 << rb), j | (1 << ra), j | (1 << ra) | (1 << rb)};
          E.line("  {");
          for (int m = 0; m < 4; ++m) {
            snprintf(buf, sizeof buf, "    const float2 v%d = a[%d]; const u64 p%d = pk(v%d.x, v%d.y), s%d = pk(v%d.y, v%d.x);", m,
                     idx[m], m, m, m, m, m, m);
            E.line(buf);
          }
          for (int k = 0; k < 4; ++k) {
            std::string t = "    { u64 t = mul2(pk(e" + std::to_string(4 * k) + ".x, e" + std::to_string(4 * k) + ".y), p0);";
            snprintf(buf, sizeof buf, " t = fma2(pk(e%d.z, e%d.w), s0, t);", 4 * k, 4 * k);
            t += buf;
            for (int m = 1; m < 4; ++m) {
              snprintf(buf, sizeof buf, " t = fma2(pk(e%d.x, e%d.y), p%d, t); t = fma2(pk(e%d.z, e%d.w), s%d, t);", 4 * k + m,
                       4 * k + m, m, 4 * k + m, 4 * k + m, m);
              t += buf;
            }
            snprintf(buf, sizeof buf, " a[%d] = up(t); }", idx[k]);
            t += buf;
            E.line(t);
          }
          E.line("  }");
        }
        E.line("}");
        return;
      }
      E.line("{ float2 u[16];");
      for (int k = 0; k < 16; ++k) E.line("  u[" + std::to_string(k) + "] = " + mat(k) + ";");
      for (int j = 0; j < R; ++j) {
        if (j & ((1 << ra) | (1 << rb))) continue;
        const int i0 = j, i1 = j | (1 << rb), i2 = j | (1 << ra), i3 = j | (1 << ra) | (1 << rb);
        snprintf(buf, sizeof buf, "  { const float2 v0 = a[%d], v1 = a[%d], v2 = a[%d], v3 = a[%d];", i0, i1, i2, i3);
        E.line(buf);
        const int idx[4] = {i0, i1, i2, i3};
        for (int k = 0; k < 4; ++k) {
          snprintf(buf, sizeof buf,
                   "    { const float2 s = cm2(u[%d], v0, u[%d], v1), t = cm2(u[%d], v2, u[%d], v3); a[%d] = cadd(s, t); }",
                   4 * k, 4 * k + 1, 4 * k + 2, 4 * k + 3, idx[k]);
          E.line(buf);
        }
        E.line("  }");
      }
      E.line("}");
      return;
    }
    case OP_D1: {
      if (kind == TN_GATE_Z) {  // sign on bit value 1
        if (op.a_kind == SRC_REG) {
          for (int j = 0; j < R; ++j)
            if (j & (1 << op.a_pos)) E.line("a[" + std::to_string(j) + "] = ng(a[" + std::to_string(j) + "]);");
        } else {
          E.line("if (" + cond_expr(op.a_kind, op.a_pos) + ") {");
          for (int j = 0; j < R; ++j) E.line("  a[" + std::to_string(j) + "] = ng(a[" + std::to_string(j) + "]);");
          E.line("}");
        }
        return;
      }
      if (kind == KIND_P || kind == TN_GATE_S || kind == TN_GATE_SDG || kind == TN_GATE_T || kind == TN_GATE_TDG) {
        // diag(1, e): only amplitudes whose bit is 1 change
        E.line("{ const float2 d1 = " + mat(1) + ";");
        if (op.a_kind == SRC_REG) {
          for (int j = 0; j < R; ++j)
            if (j & (1 << op.a_pos)) {
              snprintf(buf, sizeof buf, "  a[%d] = cm(a[%d], d1);", j, j);
              E.line(buf);
            }
        } else {
          E.line("  if (" + cond_expr(op.a_kind, op.a_pos) + ") {");
          for (int j = 0; j < R; ++j) {
            snprintf(buf, sizeof buf, "    a[%d] = cm(a[%d], d1);", j, j);
            E.line(buf);
          }
          E.line("  }");
        }
        E.line("}");
        return;
      }
      E.line("{ const float2 d0 = " + mat(0) + ", d1 = " + mat(1) + ";");
      if (op.a_kind == SRC_REG) {
        for (int j = 0; j < R; ++j) {
          snprintf(buf, sizeof buf, "  a[%d] = cm(a[%d], %s);", j, j, (j & (1 << op.a_pos)) ? "d1" : "d0");
          E.line(buf);
        }
      } else {
        E.line("  const float2 d = " + cond_expr(op.a_kind, op.a_pos) + " ? d1 : d0;");
        for (int j = 0; j < R; ++j) {
          snprintf(buf, sizeof buf, "  a[%d] = cm(a[%d], d);", j, j);
          E.line(buf);
        }
      }
      E.line("}");
      return;
    }
    case OP_CZ:
    case OP_DP: {
      // set of register indices j where both operands are 1, under a uniform condition
      std::string cond;
      uint32_t mask = (R >= 32) ? 0xFFFFFFFFu : ((1u << R) - 1u);
      auto take = [&](uint8_t k, uint8_t p) {
        if (k == SRC_REG) {
          uint32_t m = 0;
          for (int j = 0; j < R; ++j)
            if (j & (1 << p)) m |= 1u << j;
          mask &= m;
        } else {
          cond += (cond.empty() ? "" : " & ") + cond_expr(k, p);
        }
      };
      take(op.a_kind, op.a_pos);
      take(op.b_kind, op.b_pos);
      if (mask == 0) return;
      if (!cond.empty()) E.line("if (" + cond + ") {");
      if (op.type == OP_DP) E.line("{ const float2 e = " + mat(0) + ";");
      for (int j = 0; j < R; ++j)
        if (mask & (1u << j)) {
          if (op.type == OP_CZ) snprintf(buf, sizeof buf, "  a[%d] = ng(a[%d]);", j, j);
          else snprintf(buf, sizeof buf, "  a[%d] = cm(a[%d], e);", j, j);
          E.line(buf);
        }
      if (op.type == OP_DP) E.line("}");
      if (!cond.empty()) E.line("}");
      return;
    }
  }
}

}  // namespace

// Forward pass kernels read their matrix entries from a per-pass __constant__ table when one
// table serves every tile: fixed angles (one table for all batch elements) or batch 1.
bool jit_const_mats(const tn_plan &p) {
  if (const char *e = getenv("TNQ_JIT_CONST"))
    if (atoi(e) == 0) return false;
  return !p.param_dependent || p.batch == 1;
}

namespace {

std::string gen_pass(const tn_plan &p, int pi, const std::vector<int> &op_kind, int *threads_out, size_t *smem_out) {
  const PassDesc &pd = p.fwd.passes[pi];
  const int T = pd.T, K = pd.K, L = T < kLowBits ? T : kLowBits;
  const int NTHR = 1 << (T - K);
  const int TILE = 1 << T;
  const int N = p.n;
  const int mat_n = pd.mat_end - pd.mat_begin;  // even
  Emitter E;
  E.K = K;
  E.R = 1 << K;
  char buf[512];
  // Matrix entries: in a __constant__ table of this pass's module when every batch element reads
  // the same table (fixed angles) or there is one (batch 1): warp-uniform operands from the
  // constant cache, no shared-memory copy and no registers to hold them.  Otherwise staged in
  // shared memory per batch element.
  const bool cmem = jit_const_mats(p);
  // resident CTAs per SM requested from the register allocator (TNQ_JIT_MIN_BLOCKS overrides): three
  // when the entries come from constant memory (a few spilled registers, but a third CTA covers
  // another's barriers and tile loads: 1% faster alone, 7% on the serving mix, whose wide circuits share
  // the SMs across streams); two when each batch element's entries are staged in shared memory (the
  // 64-set adjoint configuration's forward passes ran 8% slower at three)
  int min_blocks = cmem ? 3 : 2;
  if (const char *mb = getenv("TNQ_JIT_MIN_BLOCKS")) min_blocks = std::max(1, std::min(4, atoi(mb)));
  if (cmem) {
    snprintf(buf, sizeof buf, "__constant__ float4 tnq_cm%d[%d];", pi, std::max(1, mat_n / 2));
    E.line(buf);
  }
  snprintf(buf, sizeof buf,
           "extern \"C\" __global__ void __launch_bounds__(%d, %d) tnq_p%d(const float2 *__restrict__ mats_g, long long mstride, "
           "float2 *__restrict__ state, long long work, u64 init_basis) {",
           NTHR, min_blocks, pi);
  E.line(buf);
  E.line("  extern __shared__ __align__(16) unsigned char smraw[];");
  // launched as programmatic dependents: wait for the previous pass before any memory access
  E.line("  asm volatile(\"griddepcontrol.wait;\" ::: \"memory\");");
  E.line("  asm volatile(\"griddepcontrol.launch_dependents;\" ::: \"memory\");");
  const int nbuf = pd.init_mode ? 1 : 2;  // loaded passes double-buffer their tiles
  E.line("  float2 *const sm0 = reinterpret_cast<float2 *>(smraw);");
  snprintf(buf, sizeof buf, "  float2 *const sm1 = sm0 + %d;", (nbuf - 1) * TILE);
  E.line(buf);
  if (!cmem) {
    snprintf(buf, sizeof buf, "  float4 *smat = reinterpret_cast<float4 *>(sm0 + %d);", nbuf * TILE);
    E.line(buf);
  }
  E.line("  const int tid = threadIdx.x;");
  // per-thread part of the load/store deposit: tile index i = 2*tid + 2*k*NTHR
  {
    std::string dep = "0ll";
    for (int j = 1; j <= T - K; ++j) {
      snprintf(buf, sizeof buf, " | ((long long)((tid >> %d) & 1) << %d)", j - 1, (int)pd.tile_pos[j]);
      dep += buf;
    }
    E.line("  const long long dep_t = " + dep + ";");
    E.line("  const int sw_t = swz(2 * tid);");
  }
  E.line("  long long cur_b = -1;");
  const int chunks = TILE / 2 / NTHR;
  auto emit_base = [&](const char *tv, const char *bv) {
    std::string base = "0ull";
    for (int j = 0; j < pd.n_outer; ++j) {
      snprintf(buf, sizeof buf, " | ((u64)((%s >> %d) & 1) << %d)", tv, j, (int)pd.outer_pos[j]);
      base += buf;
    }
    return std::string("const u64 ") + bv + " = " + base + ";";
  };
  if (!pd.init_mode) {
    // asynchronous copy of one tile into a buffer (8-byte cp.async keeps the element swizzle)
    E.line("  auto issue = [&](long long w2, float2 *dst) {");
    snprintf(buf, sizeof buf, "    const long long b2 = w2 >> %d; const long long t2 = w2 & %lldll;", pd.n_outer,
             (long long)((1ll << pd.n_outer) - 1));
    E.line(buf);
    E.line("    " + emit_base("t2", "base2"));
    snprintf(buf, sizeof buf, "    const float2 *src = state + (b2 << %d) + base2 + dep_t;", N);
    E.line(buf);
    E.line("    const unsigned d0 = (unsigned)__cvta_generic_to_shared(dst);");
    for (int k = 0; k < chunks; ++k) {
      const int ik = 2 * k * NTHR;
      long long depk = 0;
      for (int j = 0; j < T; ++j)
        if ((ik >> j) & 1) depk |= 1ll << pd.tile_pos[j];
      const int swk = swz_host(ik);
      snprintf(buf, sizeof buf,
               "    asm volatile(\"cp.async.ca.shared.global [%%0], [%%1], 8;\" :: \"r\"(d0 + 8u * (unsigned)(sw_t ^ %d)), \"l\"(src + %lldll));",
               swk, depk);
      E.line(buf);
      snprintf(buf, sizeof buf,
               "    asm volatile(\"cp.async.ca.shared.global [%%0], [%%1], 8;\" :: \"r\"(d0 + 8u * (unsigned)(sw_t ^ %d ^ 1)), \"l\"(src + %lldll + 1));",
               swk, depk);
      E.line(buf);
    }
    E.line("  };");
    E.line("  if (blockIdx.x < work) issue(blockIdx.x, sm0);");
    E.line("  asm volatile(\"cp.async.commit_group;\" ::: \"memory\");");
  }
  E.line("  int cur = 0;");
  snprintf(buf, sizeof buf, "  for (long long w = blockIdx.x; w < work; w += gridDim.x) {");
  E.line(buf);
  E.line("    float2 *const sm = cur ? sm1 : sm0;");
  snprintf(buf, sizeof buf, "    const long long b = w >> %d; const long long t = w & %lldll;", pd.n_outer,
           (long long)((1ll << pd.n_outer) - 1));
  E.line(buf);
  E.line("    " + emit_base("t", "base"));
  if (!pd.init_mode) {
    // prefetch the next tile into the other buffer, then wait for this one
    E.line("    if (w + gridDim.x < work) issue(w + gridDim.x, cur ? sm0 : sm1);");
    E.line("    asm volatile(\"cp.async.commit_group;\" ::: \"memory\");");
    E.line("    asm volatile(\"cp.async.wait_group 1;\" ::: \"memory\");");
    E.line("    __syncthreads();");
  }
  snprintf(buf, sizeof buf, "    float2 *st = state + (b << %d);", N);
  E.line(buf);
  if (pd.init_mode && pd.n_outer > 0) {
    // a basis state is zero outside the one tile that holds it: store zeros, skip the phases
    unsigned long long outer_mask = 0;
    for (int j = 0; j < pd.n_outer; ++j) outer_mask |= 1ull << pd.outer_pos[j];
    snprintf(buf, sizeof buf, "    if ((init_basis & %lluull) != base) {", outer_mask);
    E.line(buf);
    for (int k = 0; k < chunks; ++k) {
      const int ik = 2 * k * NTHR;
      long long depk = 0;
      for (int j = 0; j < T; ++j)
        if ((ik >> j) & 1) depk |= 1ll << pd.tile_pos[j];
      snprintf(buf, sizeof buf,
               "      *reinterpret_cast<float4 *>(st + base + dep_t + %lldll) = make_float4(0.f, 0.f, 0.f, 0.f);", depk);
      E.line(buf);
    }
    E.line("      continue;");
    E.line("    }");
  }
  if (cmem) {
    snprintf(buf, sizeof buf, "    const float4 *M4 = tnq_cm%d - %d;", pi, pd.mat_begin / 2);
    E.line(buf);
  } else {
    // stage this batch element's matrix entries
    E.line("    if (b != cur_b) {");
    snprintf(buf, sizeof buf,
             "      const float4 *src = reinterpret_cast<const float4 *>(mats_g + b * mstride + %d);", pd.mat_begin);
    E.line(buf);
    snprintf(buf, sizeof buf, "      for (int i = tid; i < %d; i += %d) smat[i] = src[i];", mat_n / 2, NTHR);
    E.line(buf);
    E.line("      cur_b = b;");
    E.line("      __syncthreads();");
    E.line("    }");
    snprintf(buf, sizeof buf, "    const float4 *M4 = smat - %d;", pd.mat_begin / 2);
    E.line(buf);
  }
  // synthesise the first pass's tile (loaded passes were filled by cp.async above)
  if (pd.init_mode) {
    snprintf(buf, sizeof buf, "    for (int i = tid; i < %d; i += %d) sm[i] = make_float2(0.f, 0.f);", TILE, NTHR);
    E.line(buf);
    E.line("    __syncthreads();");
    unsigned long long outer_mask = 0;
    for (int j = 0; j < pd.n_outer; ++j) outer_mask |= 1ull << pd.outer_pos[j];
    snprintf(buf, sizeof buf, "    if (tid == 0 && (init_basis & %lluull) == base) {", outer_mask);
    E.line(buf);
    std::string li = "0";
    for (int j = 0; j < T; ++j) {
      snprintf(buf, sizeof buf, " | ((int)((init_basis >> %d) & 1ull) << %d)", (int)pd.tile_pos[j], j);
      li += buf;
    }
    E.line("      const int li = " + li + ";");
    E.line("      sm[swz(li)] = make_float2(1.f, 0.f);");
    E.line("    }");
    E.line("    __syncthreads();");
  }
  // phases
  for (int ph = pd.phase_begin; ph < pd.phase_end; ++ph) {
    const PhaseDesc &d = p.fwd.phases[ph];
    E.line("    {");
    std::string tb = "0";
    for (int j = 0; j < T - K; ++j) {
      snprintf(buf, sizeof buf, " | (((tid >> %d) & 1) << %d)", j, (int)d.thr_pos[j]);
      tb += buf;
    }
    E.line("      const int tb = " + tb + ";");
    E.line("      const int pb = swz(tb);");
    E.line("      float2 a[" + std::to_string(E.R) + "];");
    int ro[32];
    for (int j = 0; j < E.R; ++j) {
      int off = 0;
      for (int r = 0; r < K; ++r)
        if ((j >> r) & 1) off |= 1 << d.reg_pos[r];
      ro[j] = swz_host(off);
      snprintf(buf, sizeof buf, "      a[%d] = sm[pb ^ %d];", j, ro[j]);
      E.line(buf);
    }
    for (int o = d.op_begin; o < d.op_end; ++o) emit_op(E, p.fwd.ops[o], op_kind[o]);
    for (int j = 0; j < E.R; ++j) {
      snprintf(buf, sizeof buf, "      sm[pb ^ %d] = a[%d];", ro[j], j);
      E.line(buf);
    }
    E.line("    }");
    E.line("    __syncthreads();");
  }
  // store
  for (int k = 0; k < chunks; ++k) {
    const int ik = 2 * k * NTHR;
    long long depk = 0;
    for (int j = 0; j < T; ++j)
      if ((ik >> j) & 1) depk |= 1ll << pd.tile_pos[j];
    const int swk = swz_host(ik);
    snprintf(buf, sizeof buf,
             "    { const float2 x = sm[sw_t ^ %d], y = sm[sw_t ^ %d ^ 1]; "
             "*reinterpret_cast<float4 *>(st + base + dep_t + %lldll) = make_float4(x.x, x.y, y.x, y.y); }",
             swk, swk, depk);
    E.line(buf);
  }
  E.line("    __syncthreads();");
  E.line("    cur ^= 1;");
  E.line("  }");
  if (!pd.init_mode) E.line("  asm volatile(\"cp.async.wait_group 0;\" ::: \"memory\");");
  E.line("}");
  *threads_out = NTHR;
  *smem_out = (size_t)nbuf * TILE * 8 + (cmem ? 0 : (size_t)mat_n * 8);
  return E.o.str();
}


// Derivative dot 2 Re <lambda| D |psi> of one parameter of an op, reduced over the warp and
// added to the pass's accumulation slot.  D has the structure of the gate kind.
// Parameter derivative of a Pauli rotation U = exp(-i t P / 2) (RX, RY, RZ): dU/dt = (-i/2) P U, so
// 2 Re <lambda_k| dU psi_{k-1}> = Im <lambda_k| P |psi_k>, evaluated from the tiles before U is
// undone (no derivative matrix applied): 2 multiply-adds per amplitude instead of a gate
// application and a dot.
bool pauli_rotation(int kind) { return kind == TN_GATE_RX || kind == TN_GATE_RY || kind == TN_GATE_RZ; }

void emit_grad_pauli(Emitter &E, const OpDesc &op, int kind, const GradRec &gr, int nwarps) {
  const int R = E.R;
  char buf[320];
  E.line("{ float acc = 0.f;");
  if (kind == TN_GATE_RZ) {  // Im <l|Z|a> = sum_j (-1)^{bit_j} (l.x a.y - l.y a.x)
    const bool reg = op.a_kind == SRC_REG;
    for (int j = 0; j < R; ++j) {
      const bool neg = reg && (j & (1 << op.a_pos));
      snprintf(buf, sizeof buf, "  acc = fmaf(%sl[%d].x, a[%d].y, acc); acc = fmaf(%sl[%d].y, a[%d].x, acc);",
               neg ? "-" : "", j, j, neg ? "" : "-", j, j);
      E.line(buf);
    }
    if (!reg) E.line("  if (" + cond_expr(op.a_kind, op.a_pos) + ") acc = -acc;");
  } else {
    const int r = op.a_pos;  // X or Y on register bit r: pairs (x = a[j], y = a[j1])
    for (int j = 0; j < R; ++j) {
      if (j & (1 << r)) continue;
      const int j1 = j | (1 << r);
      if (kind == TN_GATE_RY)  // Im: (ly . x) - (lx . y), dot = re re + im im
        snprintf(buf, sizeof buf,
                 "  acc = fmaf(l[%d].x, a[%d].x, acc); acc = fmaf(l[%d].y, a[%d].y, acc); "
                 "acc = fmaf(-l[%d].x, a[%d].x, acc); acc = fmaf(-l[%d].y, a[%d].y, acc);",
                 j1, j, j1, j, j, j1, j, j1);
      else  // RX: Im(conj(lx) y) + Im(conj(ly) x)
        snprintf(buf, sizeof buf,
                 "  acc = fmaf(l[%d].x, a[%d].y, acc); acc = fmaf(-l[%d].y, a[%d].x, acc); "
                 "acc = fmaf(l[%d].x, a[%d].y, acc); acc = fmaf(-l[%d].y, a[%d].x, acc);",
                 j, j1, j, j1, j1, j, j1, j);
      E.line(buf);
    }
  }
  E.line("  acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 16); acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 8);");
  E.line("  acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 4); acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 2);");
  E.line("  acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 1);");
  snprintf(buf, sizeof buf, "  if (lane == 0) wacc[%d + warp] += acc;", gr.slot * nwarps);
  E.line(buf);
  E.line("}");
}

void emit_grad(Emitter &E, const OpDesc &op, int kind, const GradRec &gr, int nwarps) {
  const int R = E.R;
  char buf[320];
  auto mat = [&](int k) {
    snprintf(buf, sizeof buf, "f2(M4[%d], %d)", (gr.mat + k) >> 1, (gr.mat + k) & 1);
    return std::string(buf);
  };
  E.line("{ float acc = 0.f;");
  if (op.type == OP_G1) {
    const int r = op.a_pos;
    const char *fn = (kind == TN_GATE_RY || kind == TN_GATE_SY || kind == TN_GATE_H) ? "rr"
                     : (kind == TN_GATE_RX || kind == TN_GATE_SX) ? "ri" : "cm2";
    E.line("  const float2 d00 = " + mat(0) + ", d01 = " + mat(1) + ", d10 = " + mat(2) + ", d11 = " + mat(3) + ";");
    for (int j = 0; j < R; ++j) {
      if (j & (1 << r)) continue;
      const int j1 = j | (1 << r);
      std::string z0, z1;
      if (std::string(fn) == "rr") {
        z0 = "rr(d00.x, x, d01.x, y)";
        z1 = "rr(d10.x, x, d11.x, y)";
      } else if (std::string(fn) == "ri") {
        z0 = "ri(d00.x, x, d01.y, y)";
        z1 = "ri(d11.x, y, d10.y, x)";
      } else {
        z0 = "cm2(d00, x, d01, y)";
        z1 = "cm2(d10, x, d11, y)";
      }
      snprintf(buf, sizeof buf,
               "  { const float2 x = a[%d], y = a[%d]; const float2 z0 = %s, z1 = %s; "
               "acc = fmaf(l[%d].x, z0.x, acc); acc = fmaf(l[%d].y, z0.y, acc); "
               "acc = fmaf(l[%d].x, z1.x, acc); acc = fmaf(l[%d].y, z1.y, acc); }",
               j, j1, z0.c_str(), z1.c_str(), j, j, j1, j1);
      E.line(buf);
    }
  } else if (op.type == OP_D1) {
    E.line("  const float2 d0 = " + mat(0) + ", d1 = " + mat(1) + ";");
    if (op.a_kind == SRC_REG) {
      for (int j = 0; j < R; ++j) {
        snprintf(buf, sizeof buf, "  { const float2 z = cm(a[%d], %s); acc = fmaf(l[%d].x, z.x, acc); acc = fmaf(l[%d].y, z.y, acc); }",
                 j, (j & (1 << op.a_pos)) ? "d1" : "d0", j, j);
        E.line(buf);
      }
    } else {
      E.line("  const float2 d = " + cond_expr(op.a_kind, op.a_pos) + " ? d1 : d0;");
      for (int j = 0; j < R; ++j) {
        snprintf(buf, sizeof buf, "  { const float2 z = cm(a[%d], d); acc = fmaf(l[%d].x, z.x, acc); acc = fmaf(l[%d].y, z.y, acc); }",
                 j, j, j);
        E.line(buf);
      }
    }
  } else if (op.type == OP_DP) {
    std::string cond;
    uint32_t mask = R >= 32 ? 0xFFFFFFFFu : ((1u << R) - 1u);
    auto take = [&](uint8_t k, uint8_t p) {
      if (k == SRC_REG) {
        uint32_t m = 0;
        for (int j = 0; j < R; ++j)
          if (j & (1 << p)) m |= 1u << j;
        mask &= m;
      } else {
        cond += (cond.empty() ? "" : " & ") + cond_expr(k, p);
      }
    };
    take(op.a_kind, op.a_pos);
    take(op.b_kind, op.b_pos);
    E.line("  const float2 e = " + mat(0) + ";");
    if (!cond.empty()) E.line("  if (" + cond + ") {");
    for (int j = 0; j < R; ++j)
      if (mask & (1u << j)) {
        snprintf(buf, sizeof buf, "    { const float2 z = cm(a[%d], e); acc = fmaf(l[%d].x, z.x, acc); acc = fmaf(l[%d].y, z.y, acc); }",
                 j, j, j);
        E.line(buf);
      }
    if (!cond.empty()) E.line("  }");
  }
  E.line("  acc = 2.f * acc;");
  E.line("  acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 16); acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 8);");
  E.line("  acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 4); acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 2);");
  E.line("  acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 1);");
  snprintf(buf, sizeof buf, "  if (lane == 0) wacc[%d + warp] += acc;", gr.slot * nwarps);
  E.line(buf);
  E.line("}");
}

std::string rename_array(const std::string &code, const char *to) {
  std::string out;
  out.reserve(code.size());
  for (size_t i = 0; i < code.size(); ++i) {
    // the emitted op code names its register array only as "a[" (never inside another identifier)
    if (code[i] == 'a' && i + 1 < code.size() && code[i + 1] == '[' &&
        (i == 0 || !(isalnum((unsigned char)code[i - 1]) || code[i - 1] == '_'))) {
      out += to;
      continue;
    }
    out += code[i];
  }
  return out;
}

// Adjoint-sweep pass: psi and lambda tiles double-buffered in shared memory, every op
// applied (conjugate-transposed) to both, derivative dots accumulated per slot.
std::string gen_bwd_pass(const tn_plan &p, int pi, const std::vector<int> &op_kind, int *threads_out,
                         size_t *smem_out) {
  const PassDesc &pd = p.bwd.passes[pi];
  const int T = pd.T, K = pd.K;
  const int NTHR = 1 << (T - K);
  const int NW = NTHR / 32;
  const int TILE = 1 << T;
  const int N = p.n;
  const int mat_n = pd.mat_end - pd.mat_begin;
  const int SLOTS = pd.grad_slots;
  Emitter E;
  E.K = K;
  E.R = 1 << K;
  char buf[512];
  if (SLOTS > 0) {
    std::string tab;
    for (int sl = 0; sl < SLOTS; ++sl) tab += (sl ? ", " : "") + std::to_string(p.bwd.grads[(size_t)(pd.grad_begin + sl)].param);
    snprintf(buf, sizeof buf, "__device__ const int tnq_bp%d[%d] = {", pi, SLOTS);
    E.line(std::string(buf) + tab + "};");
  }
  // resident CTAs per SM requested from the register allocator (TNQ_JIT_BWD_MIN_BLOCKS overrides)
  int bwd_blocks = 4;
  if (const char *mb = getenv("TNQ_JIT_BWD_MIN_BLOCKS")) bwd_blocks = std::max(1, std::min(8, atoi(mb)));
  snprintf(buf, sizeof buf,
           "extern \"C\" __global__ void __launch_bounds__(%d, %d) tnq_b%d(const float2 *__restrict__ mats_g, long long mstride, "
           "float2 *__restrict__ psi, float2 *__restrict__ lam, double *__restrict__ grad, int n_params) {",
           NTHR, bwd_blocks, pi);
  E.line(buf);
  E.line("  extern __shared__ __align__(16) unsigned char smraw[];");
  // launched as programmatic dependents: wait for the previous pass before any memory access
  E.line("  asm volatile(\"griddepcontrol.wait;\" ::: \"memory\");");
  E.line("  asm volatile(\"griddepcontrol.launch_dependents;\" ::: \"memory\");");
  E.line("  float2 *const p0 = reinterpret_cast<float2 *>(smraw);");
  // one psi and one lambda tile (no prefetch buffer): four CTAs per SM cover the load latency
  snprintf(buf, sizeof buf, "  float2 *const l0 = p0 + %d;", TILE);
  E.line(buf);
  snprintf(buf, sizeof buf, "  float4 *const smat = reinterpret_cast<float4 *>(p0 + %d);", 2 * TILE);
  E.line(buf);
  const int wacc_n = ((SLOTS * NW) + 1) & ~1;
  snprintf(buf, sizeof buf, "  float *const wacc = reinterpret_cast<float *>(smat + %d);", mat_n / 2);
  E.line(buf);
  snprintf(buf, sizeof buf, "  double *const gacc = reinterpret_cast<double *>(wacc + %d);", wacc_n);
  E.line(buf);
  E.line("  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;");
  E.line("  const long long b = blockIdx.y;");
  snprintf(buf, sizeof buf, "  { const float4 *src = reinterpret_cast<const float4 *>(mats_g + b * mstride + %d);", pd.mat_begin);
  E.line(buf);
  snprintf(buf, sizeof buf, "    for (int i = tid; i < %d; i += %d) smat[i] = src[i]; }", mat_n / 2, NTHR);
  E.line(buf);
  snprintf(buf, sizeof buf, "  for (int i = tid; i < %d; i += %d) wacc[i] = 0.f;", wacc_n, NTHR);
  E.line(buf);
  snprintf(buf, sizeof buf, "  for (int i = tid; i < %d; i += %d) gacc[i] = 0.0;", SLOTS, NTHR);
  E.line(buf);
  snprintf(buf, sizeof buf, "  const float4 *M4 = smat - %d;", pd.mat_begin / 2);
  E.line(buf);
  {
    std::string dep = "0ll";
    for (int j = 1; j <= T - K; ++j) {
      snprintf(buf, sizeof buf, " | ((long long)((tid >> %d) & 1) << %d)", j - 1, (int)pd.tile_pos[j]);
      dep += buf;
    }
    E.line("  const long long dep_t = " + dep + ";");
    E.line("  const int sw_t = swz(2 * tid);");
  }
  snprintf(buf, sizeof buf, "  float2 *const gp = psi + (b << %d); float2 *const gl = lam + (b << %d);", N, N);
  E.line(buf);
  auto emit_base = [&](const char *tv, const char *bv) {
    std::string base = "0ull";
    for (int j = 0; j < pd.n_outer; ++j) {
      snprintf(buf, sizeof buf, " | ((u64)((%s >> %d) & 1) << %d)", tv, j, (int)pd.outer_pos[j]);
      base += buf;
    }
    return std::string("const u64 ") + bv + " = " + base + ";";
  };
  const int chunks = TILE / 2 / NTHR;
  std::vector<long long> depk(chunks);
  std::vector<int> swk(chunks);
  for (int k = 0; k < chunks; ++k) {
    const int ik = 2 * k * NTHR;
    long long d = 0;
    for (int j = 0; j < T; ++j)
      if ((ik >> j) & 1) d |= 1ll << pd.tile_pos[j];
    depk[k] = d;
    swk[k] = swz_host(ik);
  }
  E.line("  auto issue = [&](long long t2, float2 *dp, float2 *dl) {");
  E.line("    " + emit_base("t2", "base2"));
  E.line("    const float2 *sp = gp + base2 + dep_t; const float2 *sl = gl + base2 + dep_t;");
  E.line("    const unsigned ap = (unsigned)__cvta_generic_to_shared(dp), al = (unsigned)__cvta_generic_to_shared(dl);");
  for (int k = 0; k < chunks; ++k) {
    for (int h = 0; h < 2; ++h) {
      snprintf(buf, sizeof buf,
               "    asm volatile(\"cp.async.ca.shared.global [%%0], [%%1], 8;\" :: \"r\"(ap + 8u * (unsigned)(sw_t ^ %d)), \"l\"(sp + %lldll));",
               swk[k] ^ h, depk[k] + h);
      E.line(buf);
      snprintf(buf, sizeof buf,
               "    asm volatile(\"cp.async.ca.shared.global [%%0], [%%1], 8;\" :: \"r\"(al + 8u * (unsigned)(sw_t ^ %d)), \"l\"(sl + %lldll));",
               swk[k] ^ h, depk[k] + h);
      E.line(buf);
    }
  }
  E.line("  };");
  const long long NT = 1ll << pd.n_outer;
  snprintf(buf, sizeof buf, "  for (long long t = blockIdx.x; t < %lldll; t += gridDim.x) {", NT);
  E.line(buf);
  E.line("    float2 *const smp = p0; float2 *const sml = l0;");
  E.line("    " + emit_base("t", "base"));
  E.line("    issue(t, p0, l0);");
  E.line("    asm volatile(\"cp.async.commit_group;\" ::: \"memory\");");
  E.line("    asm volatile(\"cp.async.wait_group 0;\" ::: \"memory\");");
  E.line("    __syncthreads();");
  for (int ph = pd.phase_begin; ph < pd.phase_end; ++ph) {
    const PhaseDesc &d = p.bwd.phases[ph];
    E.line("    {");
    std::string tb = "0";
    for (int j = 0; j < T - K; ++j) {
      snprintf(buf, sizeof buf, " | (((tid >> %d) & 1) << %d)", j, (int)d.thr_pos[j]);
      tb += buf;
    }
    E.line("      const int tb = " + tb + ";");
    E.line("      const int pb = swz(tb);");
    E.line("      float2 a[" + std::to_string(E.R) + "], l[" + std::to_string(E.R) + "];");
    int ro[32];
    for (int j = 0; j < E.R; ++j) {
      int off = 0;
      for (int r = 0; r < K; ++r)
        if ((j >> r) & 1) off |= 1 << d.reg_pos[r];
      ro[j] = swz_host(off);
      snprintf(buf, sizeof buf, "      a[%d] = smp[pb ^ %d]; l[%d] = sml[pb ^ %d];", j, ro[j], j, ro[j]);
      E.line(buf);
    }
    for (int o = d.op_begin; o < d.op_end; ++o) {
      const OpDesc &op = p.bwd.ops[o];
      Emitter tmp;
      tmp.K = K;
      tmp.R = E.R;
      emit_op(tmp, op, op_kind[o]);
      const std::string code_a = tmp.o.str();
      const bool pauli = op.has_grad && pauli_rotation(op_kind[o]);
      if (pauli)  // from psi_k, lambda_k
        for (int g = 0; g < op.n_grad; ++g) emit_grad_pauli(E, op, op_kind[o], p.bwd.grads[(size_t)(op.aux + g)], NW);
      E.o << code_a;  // psi_{k-1} = U^dag psi_k
      if (op.has_grad && !pauli)
        for (int g = 0; g < op.n_grad; ++g) emit_grad(E, op, op_kind[o], p.bwd.grads[(size_t)(op.aux + g)], NW);
      E.o << rename_array(code_a, "l");  // lambda_{k-1} = U^dag lambda_k
    }
    for (int j = 0; j < E.R; ++j) {
      snprintf(buf, sizeof buf, "      smp[pb ^ %d] = a[%d]; sml[pb ^ %d] = l[%d];", ro[j], j, ro[j], j);
      E.line(buf);
    }
    E.line("    }");
    E.line("    __syncthreads();");
  }
  for (int k = 0; k < chunks; ++k) {
    snprintf(buf, sizeof buf,
             "    { const float2 x = smp[sw_t ^ %d], y = smp[sw_t ^ %d ^ 1]; "
             "*reinterpret_cast<float4 *>(gp + base + dep_t + %lldll) = make_float4(x.x, x.y, y.x, y.y); "
             "const float2 u = sml[sw_t ^ %d], v = sml[sw_t ^ %d ^ 1]; "
             "*reinterpret_cast<float4 *>(gl + base + dep_t + %lldll) = make_float4(u.x, u.y, v.x, v.y); }",
             swk[k], swk[k], depk[k], swk[k], swk[k], depk[k]);
    E.line(buf);
  }
  if (SLOTS > 0) {
    snprintf(buf, sizeof buf,
             "    for (int s = tid; s < %d; s += %d) { float v = 0.f; for (int w2 = 0; w2 < %d; ++w2) { v += wacc[s * %d + w2]; "
             "wacc[s * %d + w2] = 0.f; } gacc[s] += (double)v; }",
             SLOTS, NTHR, NW, NW, NW);
    E.line(buf);
  }
  E.line("    __syncthreads();");
  E.line("  }");
  if (SLOTS > 0) {
    snprintf(buf, sizeof buf,
             "  for (int s = tid; s < %d; s += %d) atomicAdd(grad + b * n_params + tnq_bp%d[s], gacc[s]);", SLOTS, NTHR, pi);
    E.line(buf);
  }
  E.line("}");
  *threads_out = NTHR;
  *smem_out = (size_t)2 * TILE * 8 + (size_t)mat_n * 8 + (size_t)wacc_n * 4 + (size_t)SLOTS * 8;
  return E.o.str();
}

std::mutex g_cache_mu;
std::map<uint64_t, std::string> g_cubins;

std::string cache_dir() {
  const char *d = getenv("TNQ_CACHE_DIR");
  if (d && *d) return d;
  const char *h = getenv("HOME");
  return std::string(h && *h ? h : "/tmp") + "/.cache/tnq";
}

bool read_file(const std::string &path, std::string &out) {
  std::ifstream f(path, std::ios::binary);
  if (!f) return false;
  std::ostringstream ss;
  ss << f.rdbuf();
  out = ss.str();
  return !out.empty();
}

void write_file(const std::string &dir, const std::string &path, const std::string &data) {
  std::string acc;
  for (size_t i = 1; i <= dir.size(); ++i)
    if (i == dir.size() || dir[i] == '/') mkdir(dir.substr(0, i).c_str(), 0755);
  const std::string tmp = path + ".tmp" + std::to_string((unsigned long long)getpid());
  std::ofstream f(tmp, std::ios::binary);
  if (!f) return;
  f.write(data.data(), (std::streamsize)data.size());
  f.close();
  rename(tmp.c_str(), path.c_str());
}

// NVRTC options of every generated kernel; they are part of the cache key.
const char *const kNvrtcOpts[] = {"-arch=sm_103a", "-std=c++17", "-default-device", "-lineinfo"};
constexpr int kNvrtcNumOpts = (int)(sizeof(kNvrtcOpts) / sizeof(kNvrtcOpts[0]));

// Cache key of a generated source: the source, the compile options and the NVRTC version,
// so that a cubin cached by another toolkit or with other options is never reused.
uint64_t cubin_key(const std::string &src) {
  int major = 0, minor = 0;
  nvrtcVersion(&major, &minor);
  std::string key = src;
  key += "\n// nvrtc ";
  key += std::to_string(major) + "." + std::to_string(minor);
  for (int i = 0; i < kNvrtcNumOpts; ++i) {
    key += ' ';
    key += kNvrtcOpts[i];
  }
  return fnv1a(key);
}

tn_status compile_cubin(const std::string &src, std::string &cubin, std::string &err) {
  const uint64_t h = cubin_key(src);
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = g_cubins.find(h);
    if (it != g_cubins.end()) {
      cubin = it->second;
      return TN_OK;
    }
  }
  char name[64];
  snprintf(name, sizeof name, "%016llx.cubin", (unsigned long long)h);
  const std::string dir = cache_dir();
  const std::string path = dir + "/" + name;
  if (!read_file(path, cubin)) {
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, src.c_str(), "tnq_pass.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
      err = "nvrtcCreateProgram failed";
      return TN_ERR_UNSUPPORTED;
    }
    nvrtcResult r = nvrtcCompileProgram(prog, kNvrtcNumOpts, kNvrtcOpts);
    if (r != NVRTC_SUCCESS) {
      size_t n = 0;
      nvrtcGetProgramLogSize(prog, &n);
      std::string log(n, '\0');
      nvrtcGetProgramLog(prog, &log[0]);
      nvrtcDestroyProgram(&prog);
      err = "NVRTC compile failed: " + log.substr(0, 800);
      return TN_ERR_UNSUPPORTED;
    }
    size_t n = 0;
    nvrtcGetCUBINSize(prog, &n);
    cubin.assign(n, '\0');
    nvrtcGetCUBIN(prog, &cubin[0]);
    nvrtcDestroyProgram(&prog);
    write_file(dir, path, cubin);
  }
  std::lock_guard<std::mutex> lk(g_cache_mu);
  g_cubins[h] = cubin;
  return TN_OK;
}

}  // namespace

bool jit_supported(const tn_plan &p) {
  if (p.fwd.passes.empty()) return false;
  for (const PassDesc &pd : p.fwd.passes)
    if (pd.K != 4 || pd.T < kLowBits + 2) return false;
  return true;
}

bool jit_bwd_supported(const tn_plan &p) {
  if (p.bwd.passes.empty()) return false;
  for (const PassDesc &pd : p.bwd.passes)
    if (pd.K != 4 || pd.T - pd.K < 5) return false;  // whole warps (the dots reduce with shuffles)
  return true;
}

tn_status jit_build(tn_plan &p, const std::vector<int> &op_kind, bool backward, bool compile_only, std::string &err) {
  // one NVRTC program per pass: compile time grows faster than linearly with module size,
  // and separate programs compile in parallel and are cached independently
  const PassPlan &pp = backward ? p.bwd : p.fwd;
  const size_t np = pp.passes.size();
  std::vector<std::string> srcs(np), cubins(np), errs(np);
  std::vector<int> threads(np);
  std::vector<size_t> smem(np);
  std::vector<tn_status> sts(np, TN_OK);
  for (size_t i = 0; i < np; ++i) {
    int th = 0;
    size_t sm = 0;
    srcs[i] = std::string(kPrelude) + (backward ? gen_bwd_pass(p, (int)i, op_kind, &th, &sm)
                                                : gen_pass(p, (int)i, op_kind, &th, &sm));
    threads[i] = th;
    smem[i] = sm;
    if (const char *dump = getenv("TNQ_JIT_DUMP_DIR")) {
      char name[64];
      snprintf(name, sizeof name, "/%016llx.cu", (unsigned long long)fnv1a(srcs[i]));
      write_file(dump, std::string(dump) + name, srcs[i]);
    }
  }
  {
    unsigned hw = std::thread::hardware_concurrency();
    const size_t nthreads = std::max<size_t>(1, std::min<size_t>(np, hw ? hw : 4));
    std::atomic<size_t> next(0);
    std::vector<std::thread> pool;
    for (size_t t = 0; t < nthreads; ++t)
      pool.emplace_back([&]() {
        for (size_t i = next++; i < np; i = next++) sts[i] = compile_cubin(srcs[i], cubins[i], errs[i]);
      });
    for (auto &th : pool) th.join();
  }
  for (size_t i = 0; i < np; ++i)
    if (sts[i] != TN_OK) {
      err = errs[i];
      return sts[i];
    }
  if (compile_only) return TN_OK;
  std::vector<cudaLibrary_t> &libs = backward ? p.jit_bwd_libs : p.jit_libs;
  std::vector<cudaKernel_t> &kers = backward ? p.jit_bwd_kernels : p.jit_kernels;
  libs.assign(np, nullptr);
  kers.assign(np, nullptr);
  (backward ? p.jit_bwd_threads : p.jit_threads) = threads;
  (backward ? p.jit_bwd_smem : p.jit_smem) = smem;
  for (size_t i = 0; i < np; ++i) {
    cudaError_t e = cudaLibraryLoadData(&libs[i], cubins[i].data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e != cudaSuccess) {
      err = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(e);
      return TN_ERR_CUDA;
    }
    char name[32];
    snprintf(name, sizeof name, backward ? "tnq_b%zu" : "tnq_p%zu", i);
    cudaKernel_t k = nullptr;
    e = cudaLibraryGetKernel(&k, libs[i], name);
    if (e == cudaSuccess && smem[i] > 48 * 1024)
      e = cudaFuncSetAttribute((const void *)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem[i]);
    if (e != cudaSuccess) {
      err = std::string("loading generated kernel: ") + cudaGetErrorString(e);
      return TN_ERR_CUDA;
    }
    kers[i] = k;
  }
  {
    // resident CTAs per SM of each pass kernel, queried once here (not per launch)
    std::vector<int> &grid = backward ? p.jit_bwd_grid : p.jit_grid;
    grid.assign(np, 1);
    for (size_t i = 0; i < np; ++i) {
      int per_sm = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)kers[i], threads[i], smem[i]);
      if (e != cudaSuccess) {
        err = std::string("occupancy of a generated kernel: ") + cudaGetErrorString(e);
        return TN_ERR_CUDA;
      }
      grid[i] = per_sm < 1 ? 1 : per_sm;
    }
  }
  if (!backward) {
    p.jit_cm_ptr.assign(np, nullptr);
    p.jit_cm_bytes.assign(np, 0);
    if (jit_const_mats(p))
      for (size_t i = 0; i < np; ++i) {
        char name[32];
        snprintf(name, sizeof name, "tnq_cm%zu", i);
        void *ptr = nullptr;
        size_t bytes = 0;
        cudaError_t e = cudaLibraryGetGlobal(&ptr, &bytes, libs[i], name);
        if (e != cudaSuccess) {
          err = std::string("generated kernel's matrix table: ") + cudaGetErrorString(e);
          return TN_ERR_CUDA;
        }
        p.jit_cm_ptr[i] = ptr;
        p.jit_cm_bytes[i] = (size_t)(pp.passes[i].mat_end - pp.passes[i].mat_begin) * sizeof(float2);
      }
  }
  return TN_OK;
}

void jit_release(tn_plan &p) {
  p.jit_grid.clear();
  p.jit_bwd_grid.clear();
  p.jit_cm_ptr.clear();
  p.jit_cm_bytes.clear();
  for (cudaLibrary_t l : p.jit_libs)
    if (l) cudaLibraryUnload(l);
  for (cudaLibrary_t l : p.jit_bwd_libs)
    if (l) cudaLibraryUnload(l);
  p.jit_libs.clear();
  p.jit_kernels.clear();
  p.jit_bwd_libs.clear();
  p.jit_bwd_kernels.clear();
}

}  // namespace tnq
