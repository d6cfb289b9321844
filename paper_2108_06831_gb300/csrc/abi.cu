// C ABI of libtnq (declared in include/tn.h): argument checks, plan construction and
// upload, workspace layout, and the launch sequences of the contraction calls.
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "jit.h"
#include "network.h"
#include "blocks.h"
#include "kernels.h"
#include "tnq_internal.h"

namespace tnq {

namespace {
thread_local std::string g_err;
constexpr int kMaxRedPasses = 16;   // reduction passes an observable may need (workspace bound)
constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

struct SmCache {
  std::mutex m;
  int count[64] = {0};
};
SmCache g_sms;
}  // namespace

void set_error(const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

tn_status cuda_fail(cudaError_t e, const char *what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return TN_ERR_CUDA;
}

int num_sms() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  std::lock_guard<std::mutex> lk(g_sms.m);
  if (g_sms.count[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    g_sms.count[dev] = v > 0 ? v : 1;
  }
  return g_sms.count[dev];
}

// The dynamic shared-memory limit of a kernel is a per-device function attribute: raise it on
// the current device when a launch needs more than was set there before.
cudaError_t ensure_smem(const void *func, size_t bytes) {
  static std::mutex m;
  static std::map<std::pair<const void *, int>, size_t> set;
  if (bytes <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(m);
  size_t &cur = set[{func, dev}];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

}  // namespace tnq

using namespace tnq;

#define TN_CHECK_ARG(cond, ...)       \
  do {                                \
    if (!(cond)) {                    \
      set_error(__VA_ARGS__);         \
      return TN_ERR_INVALID_ARG;      \
    }                                 \
  } while (0)

#define TN_CUDA(call, what)                       \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

namespace {

template <typename T>
tn_status upload(const std::vector<T> &v, T **dst) {
  *dst = nullptr;
  if (v.empty()) return TN_OK;
  cudaError_t e = cudaMalloc((void **)dst, sizeof(T) * v.size());
  if (e != cudaSuccess) {
    *dst = nullptr;
    set_error("cudaMalloc of %zu bytes for a plan table: %s", sizeof(T) * v.size(), cudaGetErrorString(e));
    return TN_ERR_OOM;
  }
  e = cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "upload of a plan table");
  return TN_OK;
}

void free_plan_device(tn_plan *p) {
  cudaFree(p->d_slots);
  cudaFree(p->d_fused);
  cudaFree(p->d_fwd_pass);
  cudaFree(p->d_bwd_pass);
  cudaFree(p->d_fwd_phase);
  cudaFree(p->d_bwd_phase);
  cudaFree(p->d_fwd_ops);
  cudaFree(p->d_bwd_ops);
  cudaFree(p->d_bwd_grads);
  cudaFree(p->d_fixed_mats);
}

tn_status check_device(int dev) {
  int cur = -1;
  TN_CUDA(cudaGetDevice(&cur), "cudaGetDevice");
  if (cur != dev) {
    set_error("plan/observable was built on device %d but device %d is current", dev, cur);
    return TN_ERR_INVALID_ARG;
  }
  return TN_OK;
}

// Gate tables for one call: per-call materialisation when the circuit reads parameters.
tn_status call_mats(const tn_plan *p, const double *params, void *ws, cudaStream_t s, const float2 **mats,
                    long long *mstride) {
  if (!p->param_dependent) {
    *mats = reinterpret_cast<const float2 *>(p->d_fixed_mats);
    *mstride = 0;
    return TN_OK;
  }
  TN_CHECK_ARG(params != nullptr, "this circuit reads %d parameters: params_dev must not be NULL", p->n_params);
  TN_CHECK_ARG(ws != nullptr, "workspace_dev must not be NULL (plan needs %zu bytes)", p->ws_bytes);
  float2 *m = reinterpret_cast<float2 *>(static_cast<char *>(ws) + p->ws_mats);
  TN_CUDA(launch_materialize(p->d_slots, (int)p->slots.size(), p->n_fused_slots, p->d_fused, params, p->n_params,
                             p->batch, p->mstride,
                             m, s),
          "gate table kernel");
  *mats = m;
  *mstride = p->mstride;
  return TN_OK;
}

tn_status common_checks(const tn_plan *p) {
  TN_CHECK_ARG(p != nullptr, "plan is NULL");
  TN_CHECK_ARG(!p->host_only, "plan was built with TN_PLAN_HOST_ONLY and cannot run");
  TN_CHECK_ARG(p->q428 == nullptr, "a TN_PLAN_Q428 plan runs through tn_contract_state_q428 only");
  return check_device(p->device);
}

}  // namespace

extern "C" {

const char *tn_last_error(void) { return g_err.c_str(); }
const char *tn_version(void) { return "libtnq 0.1 (sm_103a)"; }

tn_status tn_build_from_circuit(int32_t n_qubits, const tn_gate *gates, int64_t n_gates, uint64_t init_basis,
                                tn_circuit **out) {
  TN_CHECK_ARG(out != nullptr, "out is NULL");
  *out = nullptr;
  TN_CHECK_ARG(n_qubits >= 1 && n_qubits <= 63, "n_qubits=%d outside [1, 63]", n_qubits);
  TN_CHECK_ARG(n_gates >= 0 && n_gates <= (1ll << 26), "n_gates=%lld out of range", (long long)n_gates);
  TN_CHECK_ARG(n_gates == 0 || gates != nullptr, "gates is NULL");
  TN_CHECK_ARG(init_basis < (1ull << n_qubits), "init_basis >= 2^%d", n_qubits);
  tn_circuit *c = new tn_circuit();
  c->n = n_qubits;
  c->init = init_basis;
  c->n_params = 0;
  c->gates.resize((size_t)n_gates);
  for (int64_t i = 0; i < n_gates; ++i) {
    const tn_gate &g = gates[i];
    TnGate &t = c->gates[(size_t)i];
    std::memset(&t, 0, sizeof(t));
    auto bad = [&](const char *why) {
      set_error("gate %lld: %s", (long long)i, why);
      delete c;
      return TN_ERR_INVALID_ARG;
    };
    if (g.kind < 0 || g.kind >= TN_GATE_KIND_COUNT) return bad("unknown kind");
    const int nq = gate_nqubits(g.kind);
    for (int k = 0; k < nq; ++k)
      if (g.q[k] < 0 || g.q[k] >= n_qubits) return bad("qubit index out of range");
    if (nq == 2 && g.q[0] == g.q[1]) return bad("two-qubit gate on equal qubits");
    const int ar = gate_arity(g.kind);
    if (g.param_idx >= 0 && ar == 0) return bad("param_idx set on a kind without angles");
    if (g.param_idx < -1) return bad("param_idx < -1");
    if ((g.kind == TN_GATE_MAT1 || g.kind == TN_GATE_MAT2) && g.mat == nullptr) return bad("MAT gate without mat");
    t.kind = g.kind;
    t.q[0] = g.q[0];
    t.q[1] = nq == 2 ? g.q[1] : -1;
    t.param_idx = g.param_idx;
    for (int a = 0; a < 3; ++a) {
      t.angle[a] = (g.param_idx >= 0 && a < ar) ? 0.0 : g.angle[a];
      t.pidx[a][0] = (g.param_idx >= 0 && a < ar) ? g.param_idx + a : -1;
      t.pidx[a][1] = -1;
    }
    if (g.kind == TN_GATE_MAT1) std::memcpy(t.mat, g.mat, 8 * sizeof(double));
    if (g.kind == TN_GATE_MAT2) std::memcpy(t.mat, g.mat, 32 * sizeof(double));
    if (g.param_idx >= 0 && g.param_idx + ar > c->n_params) c->n_params = g.param_idx + ar;
  }
  *out = c;
  return TN_OK;
}

tn_status tn_circuit_num_params(const tn_circuit *c, int32_t *n_params) {
  TN_CHECK_ARG(c != nullptr && n_params != nullptr, "NULL argument");
  *n_params = c->n_params;
  return TN_OK;
}

void tn_free_circuit(tn_circuit *c) { delete c; }

tn_status tn_plan_contraction(const tn_circuit *c, const tn_plan_opts *opts, tn_plan **out) {
  TN_CHECK_ARG(c != nullptr && out != nullptr, "NULL argument");
  *out = nullptr;
  tn_plan_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.batch == 0) o.batch = 1;
  TN_CHECK_ARG(o.batch >= 1 && o.batch <= (1 << 20), "batch=%d out of range", o.batch);
  TN_CHECK_ARG(o.target >= TN_TARGET_STATE && o.target <= TN_TARGET_EXPECTATION, "bad target %d", o.target);
  TN_CHECK_ARG(o.precision >= TN_PREC_FP32 && o.precision <= TN_PREC_SPLIT_BF16, "bad precision %d", o.precision);
  TN_CHECK_ARG(o.tile_qubits == 0 || (o.tile_qubits >= kLowBits + 2 && o.tile_qubits <= kMaxTile), "tile_qubits=%d not in {0, 6..%d}",
               o.tile_qubits, kMaxTile);
  for (int i = 0; i < 2; ++i) TN_CHECK_ARG(o.reserved[i] == 0, "reserved fields must be zero");
  if (o.flags & TN_PLAN_BLOCKS) {
    TN_CHECK_ARG(!(o.flags & (TN_PLAN_NETWORK | TN_PLAN_Q428)), "TN_PLAN_BLOCKS excludes TN_PLAN_NETWORK and TN_PLAN_Q428");
    TN_CHECK_ARG(o.target == TN_TARGET_STATE, "TN_PLAN_BLOCKS contracts states (TN_TARGET_STATE)");
    if (o.block_qubits == 0) o.block_qubits = 6;
    TN_CHECK_ARG(o.block_qubits == 6 || o.block_qubits == 7, "block_qubits must be 6 or 7 (got %lld)",
                 (long long)o.block_qubits);
  } else {
    TN_CHECK_ARG(o.block_qubits == 0, "block_qubits is for TN_PLAN_BLOCKS plans");
  }
  TN_CHECK_ARG(o.order_search == 0 || o.order_search == 1, "order_search must be 0 or 1 (got %lld)",
               (long long)o.order_search);
  TN_CHECK_ARG(o.order_trials == 0 || o.order_trials == 1 || (o.order_trials >= 4 && o.order_trials <= 4096),
               "order_trials must be 0, 1 or 4..4096 (got %lld)", (long long)o.order_trials);
  if (o.flags & TN_PLAN_Q428) {
    TN_CHECK_ARG(!(o.flags & TN_PLAN_NETWORK), "TN_PLAN_Q428 and TN_PLAN_NETWORK exclude each other");
    TN_CHECK_ARG(o.target == TN_TARGET_STATE && o.batch == 1, "TN_PLAN_Q428 contracts one state (batch 1)");
    TN_CHECK_ARG(c->n_params == 0, "TN_PLAN_Q428 takes fixed-angle circuits");
    TN_CHECK_ARG(c->n <= kMaxQubits, "TN_PLAN_Q428 holds at most %d qubits", kMaxQubits);
  }
  if (o.flags & TN_PLAN_NETWORK) {
    TN_CHECK_ARG(o.target == TN_TARGET_AMPLITUDES, "TN_PLAN_NETWORK needs TN_TARGET_AMPLITUDES");
    TN_CHECK_ARG(o.batch == 1, "TN_PLAN_NETWORK takes one parameter set (batch 1)");
    TN_CHECK_ARG(o.amp_batch >= 1 && o.amp_batch <= (1 << 20) && (o.amp_batch & (o.amp_batch - 1)) == 0,
                 "amp_batch=%lld must be a power of two in [1, 2^20]", (long long)o.amp_batch);
    TN_CHECK_ARG(c->n_params == 0, "TN_PLAN_NETWORK takes fixed-angle circuits");
  } else {
    TN_CHECK_ARG(c->n <= kMaxQubits, "state contraction holds at most %d qubits (circuit has %d); "
                 "use TN_PLAN_NETWORK for amplitudes", kMaxQubits, c->n);
  }
  if (o.max_intermediate_log2 == 0) o.max_intermediate_log2 = 28;
  // the state of every batch element must be addressable with 64-bit offsets
  TN_CHECK_ARG((double)o.batch * (double)(1ull << c->n) < 9.0e18, "batch * 2^N too large");

  tn_plan *p = new tn_plan();
  p->n = c->n;
  p->batch = o.batch;
  p->n_params = c->n_params;
  p->n_gates = (long long)c->gates.size();
  p->init = c->init;
  p->opts = o;
  p->host_only = (o.flags & TN_PLAN_HOST_ONLY) != 0;
  p->device = -1;
  const int T = std::min(c->n, o.tile_qubits ? o.tile_qubits : 12);
  const int K = std::min(T, 4);
  p->T = T;
  p->K = K;
  std::string err;
  if (o.flags & TN_PLAN_Q428) {
    p->q428 = new std::vector<Q428Gate>();
    q428_build(*c, *p->q428);
    if (!p->host_only) TN_CUDA(cudaGetDevice(&p->device), "cudaGetDevice");
    p->ws_bytes = 0;
    *out = p;
    return TN_OK;
  }
  if (o.flags & TN_PLAN_BLOCKS) {
    p->blocks = new BlockPlan();
    tn_status s2 = plan_blocks(*c, (int)o.block_qubits, o.batch, o.precision, *p->blocks, err);
    if (s2 == TN_OK && !p->host_only) {
      cudaError_t ce = cudaGetDevice(&p->device);
      if (ce != cudaSuccess) {
        err = cudaGetErrorString(ce);
        s2 = TN_ERR_CUDA;
      }
    }
    if (s2 == TN_OK) s2 = upload_blocks(*p->blocks, p->host_only, c->n_params > 0, err);
    if (s2 != TN_OK) {
      set_error("block plan: %s", err.c_str());
      delete p->blocks;
      delete p;
      return s2;
    }
    p->param_dependent = c->n_params > 0;
    p->ws_bytes = p->blocks->ws_bytes;
    *out = p;
    return TN_OK;
  }
  if (o.flags & TN_PLAN_NETWORK) {
    p->net = new NetPlan();
    int lb = 0;
    while ((1ll << lb) < o.amp_batch) ++lb;
    tn_status s2 = build_network(*c, lb, *p->net, err);
    NetPlan unplanned;
    if (s2 == TN_OK && o.order_trials == 0) unplanned = *p->net;
    if (s2 == TN_OK) s2 = plan_network(*p->net, o.max_intermediate_log2, (int)o.order_trials, (int)o.order_search, err);
    if (s2 == TN_OK) s2 = lower_network(*p->net, o.precision, err);
    // A plan that had to slice runs every merge once per slice: searching four times as many
    // orders (kSlicedTrials) there pays back within a call (the 6x6 depth-12 grid under a 2^20 cap:
    // 245 -> 690 amplitudes/s).  The cheaper of the two plans by the order cost is kept.
    if (s2 == TN_OK && o.order_trials == 0 && !p->net->slices.empty()) {
      std::string err2;
      NetPlan alt = unplanned;
      if (plan_network(alt, o.max_intermediate_log2, kSlicedTrials, (int)o.order_search, err2) == TN_OK &&
          lower_network(alt, o.precision, err2) == TN_OK && alt.cost < p->net->cost)
        *p->net = std::move(alt);
    }
    if (s2 == TN_OK && !p->host_only) {
      TN_CUDA(cudaGetDevice(&p->device), "cudaGetDevice");
      s2 = upload_network(*p->net, err);
    }
    if (s2 != TN_OK) {
      set_error("network plan: %s", err.c_str());
      if (p->net) free_network(*p->net);
      delete p->net;
      delete p;
      return s2;
    }
    p->ws_bytes = p->net->ws_bytes;
    *out = p;
    return TN_OK;
  }
  // Precontracted blocks cost a per-call FP64 product when the circuit reads parameters; below
  // kFuseMinQubitsParam qubits that costs more than the smaller state saves in the passes.
  const bool fuse = !(o.flags & TN_PLAN_NO_FUSION) && (c->n_params == 0 || c->n >= kFuseMinQubitsParam);
  const tn_circuit fwd_circ = push_phases(fuse ? fuse_pairs(*c, p->fused) : *c, p->fused);
  for (const TnGate &g : fwd_circ.gates) p->n_fused += g.kind == KIND_F2 ? 1 : 0;
  tn_status st = build_pass_plan(fwd_circ, T, K, false, p->slots, p->fwd, err);
  // the adjoint sweep stages two tiles (psi, lambda), double-buffered: at most 2^11 amplitudes each
  const int T_bwd = std::min(T, 11);
  if (st == TN_OK && o.target == TN_TARGET_EXPECTATION)
    st = build_pass_plan(*c, T_bwd, std::min(T_bwd, 4), true, p->slots, p->bwd, err);
  if (st != TN_OK) {
    set_error("planner: %s", err.c_str());
    delete p;
    return st;
  }
  p->mstride = 0;
  if (!p->slots.empty()) {
    const MatSlot &l = p->slots.back();
    p->mstride = l.offset + shape_units(l.shape);
  }
  p->mstride = (p->mstride + 1) & ~1;
  p->param_dependent = c->n_params > 0;

  // workspace layout
  size_t off = 0;
  const size_t state_bytes = ((size_t)sizeof(float2) << c->n) * (size_t)o.batch;
  if (p->param_dependent) {
    p->ws_mats = off;
    off = align_up(off + (size_t)p->mstride * sizeof(float2) * (size_t)o.batch);
  }
  if (o.target != TN_TARGET_STATE) {
    p->ws_psi = off;
    off = align_up(off + state_bytes);
  }
  if (o.target == TN_TARGET_EXPECTATION) {
    p->ws_lam = off;
    off = align_up(off + state_bytes);
    p->ws_part = off;
    off = align_up(off + (size_t)o.batch * kMaxRedPasses * 512 * sizeof(double));
  }
  p->ws_bytes = off;

  if (p->host_only && getenv("TNQ_JIT_COMPILE_CHECK") && !(o.flags & TN_PLAN_NO_SPECIALIZE) && jit_supported(*p)) {
    // generate and compile the specialised kernels without loading them (no GPU needed)
    std::vector<int> kinds(p->fwd.ops.size());
    for (size_t i = 0; i < kinds.size(); ++i) kinds[i] = fwd_circ.gates[(size_t)p->fwd.op_gate[i]].kind;
    std::string jerr;
    tn_status u = jit_build(*p, kinds, false, true, jerr);
    if (u == TN_OK && jit_bwd_supported(*p)) {
      std::vector<int> bk(p->bwd.ops.size());
      for (size_t i = 0; i < bk.size(); ++i) bk[i] = c->gates[(size_t)p->bwd.op_gate[i]].kind;
      u = jit_build(*p, bk, true, true, jerr);
    }
    if (u != TN_OK) {
      set_error("plan-specialised kernels: %s", jerr.c_str());
      delete p;
      return u;
    }
  }
  if (!p->host_only) {
    TN_CUDA(cudaGetDevice(&p->device), "cudaGetDevice");
    tn_status u = TN_OK;
    if (u == TN_OK) {  // device copy in the order the materialisation kernel reads (fused blocks first)
      std::vector<MatSlot> ordered = p->slots;
      p->n_fused_slots = order_slots_fused_first(ordered);
      u = upload(ordered, &p->d_slots);
    }
    if (u == TN_OK && !p->fused.empty()) u = upload(p->fused, &p->d_fused);
    if (u == TN_OK) u = upload(p->fwd.passes, &p->d_fwd_pass);
    if (u == TN_OK) u = upload(p->fwd.phases, &p->d_fwd_phase);
    if (u == TN_OK) u = upload(p->fwd.ops, &p->d_fwd_ops);
    if (u == TN_OK) u = upload(p->bwd.passes, &p->d_bwd_pass);
    if (u == TN_OK) u = upload(p->bwd.phases, &p->d_bwd_phase);
    if (u == TN_OK) u = upload(p->bwd.ops, &p->d_bwd_ops);
    if (u == TN_OK) u = upload(p->bwd.grads, &p->d_bwd_grads);
    if (u == TN_OK && !p->param_dependent && p->mstride > 0) {
      cudaError_t e = cudaMalloc((void **)&p->d_fixed_mats, (size_t)p->mstride * sizeof(float2));
      if (e != cudaSuccess) {
        set_error("cudaMalloc of the fixed gate table: %s", cudaGetErrorString(e));
        u = TN_ERR_OOM;
      } else {
        e = launch_materialize(p->d_slots, (int)p->slots.size(), p->n_fused_slots, p->d_fused, nullptr, 0, 1, p->mstride,
                               reinterpret_cast<float2 *>(p->d_fixed_mats), 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) u = cuda_fail(e, "fixed gate table");
      }
    }
    if (u == TN_OK && !(o.flags & TN_PLAN_NO_SPECIALIZE) && jit_supported(*p)) {
      std::vector<int> kinds(p->fwd.ops.size());
      for (size_t i = 0; i < kinds.size(); ++i) kinds[i] = fwd_circ.gates[(size_t)p->fwd.op_gate[i]].kind;
      std::string jerr;
      u = jit_build(*p, kinds, false, false, jerr);
      if (u == TN_OK && !p->param_dependent && p->d_fixed_mats) {
        // fixed angles: each pass's constant table is filled once
        for (size_t i = 0; i < p->jit_cm_ptr.size() && u == TN_OK; ++i)
          if (p->jit_cm_ptr[i] && p->jit_cm_bytes[i]) {
            cudaError_t e = cudaMemcpy(p->jit_cm_ptr[i], p->d_fixed_mats + 2 * (size_t)p->fwd.passes[i].mat_begin,
                                       p->jit_cm_bytes[i], cudaMemcpyDeviceToDevice);
            if (e != cudaSuccess) u = cuda_fail(e, "generated kernels' matrix tables");
          }
      }
      if (u == TN_OK && jit_bwd_supported(*p)) {
        std::vector<int> bk(p->bwd.ops.size());
        for (size_t i = 0; i < bk.size(); ++i) bk[i] = c->gates[(size_t)p->bwd.op_gate[i]].kind;
        u = jit_build(*p, bk, true, false, jerr);
      }
      if (u != TN_OK) set_error("plan-specialised kernels: %s", jerr.c_str());
    }
    if (u != TN_OK) {
      jit_release(*p);
      free_plan_device(p);
      delete p;
      return u;
    }
  }
  *out = p;
  return TN_OK;
}

tn_status tn_plan_contraction_tuned(const tn_circuit *c, const tn_plan_opts *opts, const tn_tune_opts *tune,
                                   tn_stream_t s, tn_plan **out, int32_t *tile_out) {
  TN_CHECK_ARG(c != nullptr && out != nullptr, "NULL argument");
  *out = nullptr;
  tn_plan_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  TN_CHECK_ARG(!(o.flags & (TN_PLAN_NETWORK | TN_PLAN_Q428 | TN_PLAN_BLOCKS | TN_PLAN_HOST_ONLY)),
               "the tile autotuner takes state / expectation plans that run on the GPU");
  TN_CHECK_ARG(o.tile_qubits == 0, "tile_qubits is what the autotuner chooses: leave it 0");
  tn_tune_opts t;
  std::memset(&t, 0, sizeof(t));
  if (tune) t = *tune;
  std::vector<int> cands;
  for (int i = 0; i < 8 && t.candidates[i] != 0; ++i) {
    TN_CHECK_ARG(t.candidates[i] >= kLowBits + 2 && t.candidates[i] <= kMaxTile, "candidate tile %d not in [6, %d]",
                 t.candidates[i], kMaxTile);
    cands.push_back(t.candidates[i]);
  }
  if (cands.empty()) cands = {10, 11, 12, 13};
  TN_CHECK_ARG(t.reps >= 0 && t.reps <= 100, "reps=%d out of range", t.reps);
  TN_CHECK_ARG(t.flags == 0, "flags must be zero");
  for (int i = 0; i < 4; ++i) TN_CHECK_ARG(t.reserved[i] == 0, "reserved fields must be zero");
  return plan_tuned(c, o, cands, t.reps > 0 ? t.reps : 3, reinterpret_cast<cudaStream_t>(s), out, tile_out);
}

tn_status tn_plan_workspace_bytes(const tn_plan *p, size_t *bytes) {
  TN_CHECK_ARG(p != nullptr && bytes != nullptr, "NULL argument");
  *bytes = p->ws_bytes;
  return TN_OK;
}

tn_status tn_plan_get_stats(const tn_plan *p, tn_plan_stats *st) {
  TN_CHECK_ARG(p != nullptr && st != nullptr, "NULL argument");
  std::memset(st, 0, sizeof(*st));
  st->n_qubits = p->n;
  st->n_params = p->n_params;
  st->n_gates = p->n_gates;
  st->n_passes = (int)p->fwd.passes.size();
  st->n_phases = (int)p->fwd.phases.size();
  st->n_ops = (long long)p->fwd.ops.size();
  st->n_fused = p->n_fused;
  if (p->q428) {  // one launch per gate, each reading and writing every amplitude (int32 pairs)
    st->n_passes = (int)p->q428->size();
    st->hbm_bytes = 8.0 * std::ldexp(1.0, p->n) * (1.0 + 2.0 * (double)p->q428->size());
    return TN_OK;
  }
  st->tile_qubits = p->T;
  st->reg_qubits = p->K;
  st->flops = p->fwd.flops;
  double bytes = 0;
  for (const PassDesc &pd : p->fwd.passes) bytes += (pd.init_mode ? 8.0 : 16.0) * (double)(1ull << p->n);
  st->hbm_bytes = bytes;
  st->n_bwd_passes = (int)p->bwd.passes.size();
  st->bwd_flops = 2.0 * p->bwd.flops + p->bwd.grad_flops;
  st->specialized = p->jit_kernels.empty() ? 0 : 1;
  if (p->blocks) {
    const BlockPlan &bp = *p->blocks;
    st->n_passes = (int)bp.qubits.size() - 1;
    st->n_phases = 0;
    st->n_ops = (long long)bp.gates.size();
    st->n_fused = (int)bp.qubits.size();
    st->tile_qubits = bp.k;
    st->reg_qubits = 0;
    st->flops = bp.flops;
    st->hbm_bytes = bp.bytes;
    st->specialized = 0;
  }
  if (p->net) {
    st->n_passes = 0;
    st->net_merges = (int)p->net->launches.size();
    st->net_folded_merges = p->net->folded_merges;
    st->net_max_log2 = p->net->max_log2;
    st->net_sliced = (int)p->net->slices.size();
    st->net_batch_log2 = p->net->log2_batch;
    st->net_cost = p->net->cost;
    st->net_bytes = p->net->bytes;
    st->flops = p->net->flops;
    int tc = 0;
    for (const NetLaunch &L : p->net->launches) tc += L.precision != TN_PREC_FP32;
    st->net_tensor_merges = tc;
  }
  return TN_OK;
}

void tn_free_plan(tn_plan *p) {
  if (!p) return;
  delete p->q428;
  p->q428 = nullptr;
  if (p->blocks) {
    if (!p->host_only) free_blocks(*p->blocks);
    delete p->blocks;
    delete p;
    return;
  }
  if (p->net) {
    if (!p->host_only) free_network(*p->net);
    delete p->net;
    delete p;
    return;
  }
  jit_release(*p);
  if (!p->host_only) free_plan_device(p);
  delete p;
}

tn_status tn_build_observable(int32_t n_qubits, const tn_pauli_sum *H, tn_observable **out) {
  TN_CHECK_ARG(out != nullptr && H != nullptr, "NULL argument");
  *out = nullptr;
  TN_CHECK_ARG(n_qubits >= 1 && n_qubits <= kMaxQubits, "n_qubits=%d out of range", n_qubits);
  TN_CHECK_ARG(H->n_terms >= 0 && H->n_terms <= (1 << 20), "n_terms=%d out of range", H->n_terms);
  TN_CHECK_ARG(H->n_terms == 0 || (H->coef != nullptr && H->paulis != nullptr), "coef/paulis NULL");
  tn_observable *o = new tn_observable();
  o->n = n_qubits;
  o->n_terms = H->n_terms;
  const int T = std::min(n_qubits, 12);
  o->T = T;
  struct HostTerm {
    double coef;
    uint64_t xm, zm;
    int ny;
  };
  std::vector<HostTerm> diag, offd;
  for (int t = 0; t < H->n_terms; ++t) {
    HostTerm h{H->coef[t], 0, 0, 0};
    for (int q = 0; q < n_qubits; ++q) {
      const uint8_t pc = H->paulis[(size_t)t * n_qubits + q];
      if (pc > 3) {
        delete o;
        set_error("term %d qubit %d: Pauli code %u not in {0,1,2,3}", t, q, (unsigned)pc);
        return TN_ERR_INVALID_ARG;
      }
      const uint64_t bit = 1ull << (n_qubits - 1 - q);
      if (pc == 1 || pc == 2) h.xm |= bit;
      if (pc == 2 || pc == 3) h.zm |= bit;
      if (pc == 2) h.ny++;
    }
    (h.xm == 0 ? diag : offd).push_back(h);
  }
  const uint64_t low = (1ull << std::min(kLowBits, n_qubits)) - 1;
  auto make_pass = [&](uint64_t S, int tb, int te) {
    RedPass rp;
    std::memset(&rp, 0, sizeof(rp));
    int tl = 0, ol = 0;
    for (int b = 0; b < n_qubits; ++b) {
      if ((S >> b) & 1) rp.tile_pos[tl++] = (uint8_t)b;
      else rp.outer_pos[ol++] = (uint8_t)b;
    }
    rp.T = tl;
    rp.n_outer = ol;
    rp.term_begin = tb;
    rp.term_end = te;
    return rp;
  };
  auto push_term = [&](const HostTerm &h, uint64_t S) {
    DevTerm d;
    std::memset(&d, 0, sizeof(d));
    d.coef = h.coef;
    d.xm = h.xm;
    d.zm = h.zm;
    d.ny = h.ny;
    int l = 0, xl = 0;
    for (int b = 0; b < n_qubits; ++b)
      if ((S >> b) & 1) {
        if ((h.xm >> b) & 1) xl |= 1 << l;
        ++l;
      }
    d.xl = xl;
    o->terms.push_back(d);
  };
  // greedy passes: each starts from the low bits and takes every remaining term whose flip
  // bits still fit in T tile bits; diagonal terms ride along in the first pass
  std::vector<char> used(offd.size(), 0);
  size_t left = offd.size();
  bool first = true;
  while (first || left > 0) {
    uint64_t S = low;
    int nS = __builtin_popcountll(S);
    std::vector<size_t> take;
    for (size_t i = 0; i < offd.size(); ++i) {
      if (used[i]) continue;
      const uint64_t need = offd[i].xm & ~S;
      const int add = __builtin_popcountll(need);
      if (nS + add <= T) {
        S |= need;
        nS += add;
        take.push_back(i);
      }
    }
    if (!first && take.empty()) {
      delete o;
      set_error("a Pauli term flips more than %d qubits outside the lowest %d; not supported", T - kLowBits, kLowBits);
      return TN_ERR_UNSUPPORTED;
    }
    for (int b = 0; b < n_qubits && nS < T; ++b)
      if (!((S >> b) & 1)) { S |= 1ull << b; ++nS; }
    const int tb = (int)o->terms.size();
    if (first)
      for (const HostTerm &h : diag) push_term(h, S);
    for (size_t i : take) {
      push_term(offd[i], S);
      used[i] = 1;
      --left;
    }
    o->passes.push_back(make_pass(S, tb, (int)o->terms.size()));
    first = false;
  }
  if ((int)o->passes.size() > kMaxRedPasses) {
    delete o;
    set_error("observable needs %zu reduction passes (at most %d supported)", o->passes.size(), kMaxRedPasses);
    return TN_ERR_UNSUPPORTED;
  }
  cudaError_t e = cudaGetDevice(&o->device);
  if (e != cudaSuccess) {
    delete o;
    return cuda_fail(e, "cudaGetDevice");
  }
  tn_status u = upload(o->terms, &o->d_terms);
  if (u == TN_OK) u = upload(o->passes, &o->d_passes);
  if (u != TN_OK) {
    cudaFree(o->d_terms);
    cudaFree(o->d_passes);
    delete o;
    return u;
  }
  *out = o;
  return TN_OK;
}

void tn_free_observable(tn_observable *o) {
  if (!o) return;
  cudaFree(o->d_terms);
  cudaFree(o->d_passes);
  delete o;
}

tn_status tn_contract_state(const tn_plan *p, const double *params_dev, void *state_dev, void *workspace_dev,
                            tn_stream_t s) {
  tn_status st = common_checks(p);
  if (st != TN_OK) return st;
  TN_CHECK_ARG(state_dev != nullptr, "state_dev is NULL");
  TN_CHECK_ARG(((uintptr_t)state_dev & 15) == 0, "state_dev must be 16-byte aligned");
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(s);
  if (p->blocks) {
    TN_CHECK_ARG(p->n_params == 0 || params_dev != nullptr,
                 "this circuit reads %d parameters: params_dev must not be NULL", p->n_params);
    TN_CHECK_ARG(workspace_dev != nullptr, "workspace_dev is NULL (plan needs %zu bytes)", p->ws_bytes);
    TN_CUDA(run_blocks(*p->blocks, params_dev, p->n_params, static_cast<float2 *>(state_dev), workspace_dev, cs),
            "block contraction");
    return TN_OK;
  }
  const float2 *mats = nullptr;
  long long mstride = 0;
  st = call_mats(p, params_dev, workspace_dev, cs, &mats, &mstride);
  if (st != TN_OK) return st;
  TN_CUDA(launch_forward(p, mats, mstride, static_cast<float2 *>(state_dev), cs), "gate-apply kernel");
  return TN_OK;
}

tn_status tn_contract_amplitudes(const tn_plan *p, const double *params_dev, const uint64_t *bitstrings_dev,
                                 int64_t n_bitstrings, void *amps_dev, void *workspace_dev, tn_stream_t s) {
  tn_status st = common_checks(p);
  if (st != TN_OK) return st;
  TN_CHECK_ARG(p->opts.target != TN_TARGET_STATE, "plan target must be AMPLITUDES or EXPECTATION");
  TN_CHECK_ARG(n_bitstrings >= 0, "n_bitstrings < 0");
  TN_CHECK_ARG(n_bitstrings == 0 || (bitstrings_dev != nullptr && amps_dev != nullptr), "NULL device pointer");
  TN_CHECK_ARG(workspace_dev != nullptr, "workspace_dev is NULL");
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(s);
  const float2 *mats = nullptr;
  long long mstride = 0;
  st = call_mats(p, params_dev, workspace_dev, cs, &mats, &mstride);
  if (st != TN_OK) return st;
  if (p->net) {
    const long long cap = 1ll << p->net->call_log2;
    TN_CHECK_ARG(n_bitstrings <= cap, "this network plan takes at most %lld bitstrings per call", cap);
    if (n_bitstrings == 0) return TN_OK;
    TN_CUDA(run_network(*p->net, bitstrings_dev, n_bitstrings, static_cast<float2 *>(amps_dev), workspace_dev, cs),
            "network contraction");
    return TN_OK;
  }
  float2 *psi = reinterpret_cast<float2 *>(static_cast<char *>(workspace_dev) + p->ws_psi);
  TN_CUDA(launch_forward(p, mats, mstride, psi, cs), "gate-apply kernel");
  TN_CUDA(launch_gather(psi, p->n, p->batch, bitstrings_dev, n_bitstrings, static_cast<float2 *>(amps_dev), cs),
          "gather kernel");
  return TN_OK;
}

tn_status tn_contract_state_q428(const tn_plan *p, int32_t *state_dev, tn_stream_t s) {
  TN_CHECK_ARG(p != nullptr, "plan is NULL");
  TN_CHECK_ARG(p->q428 != nullptr, "the plan was not built with TN_PLAN_Q428");
  TN_CHECK_ARG(!p->host_only, "plan was built with TN_PLAN_HOST_ONLY and cannot run");
  TN_CHECK_ARG(state_dev != nullptr, "state_dev is NULL");
  TN_CHECK_ARG(((uintptr_t)state_dev & 7) == 0, "state_dev must be 8-byte aligned");
  tn_status st = check_device(p->device);
  if (st != TN_OK) return st;
  TN_CUDA(launch_q428(*p->q428, p->n, p->init, state_dev, reinterpret_cast<cudaStream_t>(s)), "fixed-point kernels");
  return TN_OK;
}

tn_status tn_expectation(const tn_plan *p, const tn_observable *H, const double *params_dev, double *out_dev,
                         void *workspace_dev, tn_stream_t s) {
  tn_status st = common_checks(p);
  if (st != TN_OK) return st;
  TN_CHECK_ARG(H != nullptr && out_dev != nullptr && workspace_dev != nullptr, "NULL argument");
  TN_CHECK_ARG(p->opts.target == TN_TARGET_EXPECTATION, "plan target must be EXPECTATION");
  TN_CHECK_ARG(H->n == p->n, "observable has %d qubits, circuit %d", H->n, p->n);
  st = check_device(H->device);
  if (st != TN_OK) return st;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(s);
  const float2 *mats = nullptr;
  long long mstride = 0;
  st = call_mats(p, params_dev, workspace_dev, cs, &mats, &mstride);
  if (st != TN_OK) return st;
  char *ws = static_cast<char *>(workspace_dev);
  float2 *psi = reinterpret_cast<float2 *>(ws + p->ws_psi);
  TN_CUDA(launch_forward(p, mats, mstride, psi, cs), "gate-apply kernel");
  TN_CUDA(launch_expectation(H, p->batch, psi, reinterpret_cast<double *>(ws + p->ws_part), out_dev, cs),
          "expectation kernel");
  return TN_OK;
}

tn_status tn_expectation_backward(const tn_plan *p, const tn_observable *H, const double *params_dev,
                                  const double *grad_out_dev, double *grad_params_dev, void *workspace_dev,
                                  tn_stream_t s) {
  tn_status st = common_checks(p);
  if (st != TN_OK) return st;
  TN_CHECK_ARG(H != nullptr && workspace_dev != nullptr, "NULL argument");
  TN_CHECK_ARG(p->opts.target == TN_TARGET_EXPECTATION, "plan target must be EXPECTATION");
  TN_CHECK_ARG(H->n == p->n, "observable has %d qubits, circuit %d", H->n, p->n);
  TN_CHECK_ARG(p->n_params == 0 || grad_params_dev != nullptr, "grad_params_dev is NULL");
  st = check_device(H->device);
  if (st != TN_OK) return st;
  if (p->n_params == 0) return TN_OK;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(s);
  const float2 *mats = nullptr;
  long long mstride = 0;
  st = call_mats(p, params_dev, workspace_dev, cs, &mats, &mstride);
  if (st != TN_OK) return st;
  char *ws = static_cast<char *>(workspace_dev);
  float2 *psi = reinterpret_cast<float2 *>(ws + p->ws_psi);
  float2 *lam = reinterpret_cast<float2 *>(ws + p->ws_lam);
  TN_CUDA(launch_forward(p, mats, mstride, psi, cs), "gate-apply kernel");
  TN_CUDA(launch_apply_hamiltonian(H, p->batch, psi, lam, cs), "H psi kernel");
  TN_CUDA(cudaMemsetAsync(grad_params_dev, 0, sizeof(double) * (size_t)p->batch * p->n_params, cs), "memset grad");
  TN_CUDA(launch_backward(p, mats, mstride, psi, lam, grad_params_dev, cs), "adjoint kernel");
  TN_CUDA(launch_scale_grad(grad_params_dev, grad_out_dev, p->batch, p->n_params, cs), "grad scale kernel");
  return TN_OK;
}

tn_status tn_expectation_value_and_grad(const tn_plan *p, const tn_observable *H, const double *params_dev,
                                        double *out_dev, double *grad_params_dev, void *workspace_dev,
                                        tn_stream_t s) {
  tn_status st = common_checks(p);
  if (st != TN_OK) return st;
  TN_CHECK_ARG(H != nullptr && out_dev != nullptr && workspace_dev != nullptr, "NULL argument");
  TN_CHECK_ARG(p->opts.target == TN_TARGET_EXPECTATION, "plan target must be EXPECTATION");
  TN_CHECK_ARG(H->n == p->n, "observable has %d qubits, circuit %d", H->n, p->n);
  TN_CHECK_ARG(p->n_params == 0 || grad_params_dev != nullptr, "grad_params_dev is NULL");
  st = check_device(H->device);
  if (st != TN_OK) return st;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(s);
  const float2 *mats = nullptr;
  long long mstride = 0;
  st = call_mats(p, params_dev, workspace_dev, cs, &mats, &mstride);
  if (st != TN_OK) return st;
  char *ws = static_cast<char *>(workspace_dev);
  float2 *psi = reinterpret_cast<float2 *>(ws + p->ws_psi);
  float2 *lam = reinterpret_cast<float2 *>(ws + p->ws_lam);
  TN_CUDA(launch_forward(p, mats, mstride, psi, cs), "gate-apply kernel");
  double *part = reinterpret_cast<double *>(ws + p->ws_part);
  if (p->n_params == 0) {
    TN_CUDA(launch_expectation(H, p->batch, psi, part, out_dev, cs), "expectation kernel");
    return TN_OK;
  }
  // lam = H psi, and the energy <psi|lam> from the last pass over lam (no separate reduction)
  TN_CUDA(launch_apply_hamiltonian(H, p->batch, psi, lam, cs, part, out_dev), "H psi kernel");
  TN_CUDA(cudaMemsetAsync(grad_params_dev, 0, sizeof(double) * (size_t)p->batch * p->n_params, cs), "memset grad");
  TN_CUDA(launch_backward(p, mats, mstride, psi, lam, grad_params_dev, cs), "adjoint kernel");
  return TN_OK;
}

tn_status tn_state_expectation_workspace_bytes(const tn_observable *H, int32_t batch, size_t *bytes) {
  TN_CHECK_ARG(H != nullptr && bytes != nullptr, "NULL argument");
  TN_CHECK_ARG(batch >= 1, "batch < 1");
  *bytes = observable_partials(H, batch) * sizeof(double);
  return TN_OK;
}

tn_status tn_state_expectation(const tn_observable *H, int32_t batch, const void *state_dev, double *out_dev,
                               void *workspace_dev, size_t workspace_bytes, tn_stream_t s) {
  TN_CHECK_ARG(H != nullptr && state_dev != nullptr && out_dev != nullptr, "NULL argument");
  TN_CHECK_ARG(batch >= 1, "batch < 1");
  TN_CHECK_ARG(((uintptr_t)state_dev & 15) == 0, "state_dev must be 16-byte aligned");
  const size_t need = observable_partials(H, batch) * sizeof(double);
  TN_CHECK_ARG(workspace_dev != nullptr && workspace_bytes >= need, "workspace needs %zu bytes, got %zu", need,
               workspace_bytes);
  tn_status st = check_device(H->device);
  if (st != TN_OK) return st;
  TN_CUDA(launch_expectation(H, batch, static_cast<const float2 *>(state_dev), static_cast<double *>(workspace_dev),
                             out_dev, reinterpret_cast<cudaStream_t>(s)),
          "expectation kernel");
  return TN_OK;
}

tn_status tn_permute(int32_t n_legs, const int32_t *perm, int64_t batch, const void *in_dev, void *out_dev,
                     tn_stream_t s) {
  TN_CHECK_ARG(n_legs >= 1 && n_legs <= kMaxQubits, "n_legs=%d out of range", n_legs);
  TN_CHECK_ARG(perm != nullptr && in_dev != nullptr && out_dev != nullptr, "NULL argument");
  TN_CHECK_ARG(batch >= 0, "batch < 0");
  unsigned long long seen = 0;
  for (int j = 0; j < n_legs; ++j) {
    TN_CHECK_ARG(perm[j] >= 0 && perm[j] < n_legs, "perm[%d]=%d out of range", j, perm[j]);
    TN_CHECK_ARG(!((seen >> perm[j]) & 1), "perm is not a permutation");
    seen |= 1ull << perm[j];
  }
  TN_CHECK_ARG(((uintptr_t)in_dev & 15) == 0 && ((uintptr_t)out_dev & 15) == 0, "buffers must be 16-byte aligned");
  const size_t bytes = ((size_t)sizeof(float2) << n_legs) * (size_t)batch;
  const char *a = static_cast<const char *>(in_dev);
  const char *b = static_cast<const char *>(out_dev);
  TN_CHECK_ARG(a + bytes <= b || b + bytes <= a, "in_dev and out_dev overlap");
  if (batch == 0) return TN_OK;
  TN_CUDA(launch_permute(n_legs, perm, batch, static_cast<const float2 *>(in_dev), static_cast<float2 *>(out_dev),
                         reinterpret_cast<cudaStream_t>(s)),
          "permute kernel");
  return TN_OK;
}

tn_status tn_cgemm_workspace_bytes(int32_t precision, int64_t batch, int64_t M, int64_t N, int64_t K, size_t *bytes) {
  TN_CHECK_ARG(bytes != nullptr, "NULL argument");
  TN_CHECK_ARG(precision >= TN_PREC_FP32 && precision <= TN_PREC_SPLIT_BF16, "bad precision %d", precision);
  TN_CHECK_ARG(batch >= 0 && M >= 0 && N >= 0 && K >= 0, "negative size");
  *bytes = cgemm_workspace(precision, batch, M, N, K);
  return TN_OK;
}

tn_status tn_cgemm_batched(int32_t precision, int64_t batch, int64_t M, int64_t N, int64_t K, const void *A_dev,
                           const void *B_dev, void *C_dev, void *workspace_dev, size_t workspace_bytes,
                           tn_stream_t s) {
  TN_CHECK_ARG(precision >= TN_PREC_FP32 && precision <= TN_PREC_SPLIT_BF16, "bad precision %d", precision);
  TN_CHECK_ARG(batch >= 0 && M >= 0 && N >= 0 && K >= 0, "negative size");
  if (batch == 0 || M == 0 || N == 0) return TN_OK;
  TN_CHECK_ARG(C_dev != nullptr && (K == 0 || (A_dev != nullptr && B_dev != nullptr)), "NULL argument");
  TN_CHECK_ARG(((uintptr_t)A_dev & 15) == 0 && ((uintptr_t)B_dev & 15) == 0 && ((uintptr_t)C_dev & 15) == 0,
               "operands must be 16-byte aligned");
  const size_t need = cgemm_workspace(precision, batch, M, N, K);
  TN_CHECK_ARG(need == 0 || (workspace_dev != nullptr && workspace_bytes >= need), "workspace needs %zu bytes", need);
  cudaError_t e = launch_cgemm(precision, batch, M, N, K, static_cast<const float2 *>(A_dev),
                               static_cast<const float2 *>(B_dev), static_cast<float2 *>(C_dev), workspace_dev,
                               workspace_bytes, reinterpret_cast<cudaStream_t>(s));
  if (e == cudaErrorNotSupported) {
    set_error("cgemm: shape (M=%lld N=%lld K=%lld) not supported in this precision", (long long)M, (long long)N,
              (long long)K);
    return TN_ERR_UNSUPPORTED;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cgemm kernel");
  return TN_OK;
}

tn_status tn_batch_build(const tn_plan *const *plans, int32_t n_plans, tn_batch **out) {
  TN_CHECK_ARG(out != nullptr && (n_plans == 0 || plans != nullptr), "NULL argument");
  TN_CHECK_ARG(n_plans >= 1 && n_plans <= (1 << 20), "n_plans=%d out of range", n_plans);
  *out = nullptr;
  for (int i = 0; i < n_plans; ++i) {
    TN_CHECK_ARG(plans[i] != nullptr, "plan %d is NULL", i);
    tn_status st = check_device(plans[i]->device);
    if (st != TN_OK) return st;
  }
  return batch_build(plans, n_plans, out);
}

tn_status tn_batch_sizes(const tn_batch *b, int64_t *state_elems, size_t *workspace_bytes) {
  TN_CHECK_ARG(b != nullptr && state_elems != nullptr && workspace_bytes != nullptr, "NULL argument");
  long long e = 0;
  size_t w = 0;
  batch_sizes(b, &e, &w);
  *state_elems = e;
  *workspace_bytes = w;
  return TN_OK;
}

tn_status tn_batch_state_offsets(const tn_batch *b, int64_t *offsets) {
  TN_CHECK_ARG(b != nullptr && offsets != nullptr, "NULL argument");
  return batch_offsets(b, reinterpret_cast<long long *>(offsets));
}

tn_status tn_batch_run(const tn_batch *b, void *states_dev, void *workspace_dev, tn_stream_t s) {
  TN_CHECK_ARG(b != nullptr, "NULL argument");
  TN_CHECK_ARG(batch_num_params(b, nullptr) == 0,
               "the batch has parameterised circuits (%d parameters): use tn_batch_run_params",
               batch_num_params(b, nullptr));
  return tn_batch_run_params(b, nullptr, states_dev, workspace_dev, s);
}

tn_status tn_batch_run_params(const tn_batch *b, const double *params_dev, void *states_dev, void *workspace_dev,
                              tn_stream_t s) {
  TN_CHECK_ARG(b != nullptr && states_dev != nullptr && workspace_dev != nullptr, "NULL argument");
  TN_CHECK_ARG(((uintptr_t)states_dev & 15) == 0, "states_dev must be 16-byte aligned");
  TN_CHECK_ARG(batch_num_params(b, nullptr) == 0 || params_dev != nullptr,
               "the batch's circuits read %d parameters: params_dev must not be NULL", batch_num_params(b, nullptr));
  tn_status st = check_device(batch_device(b));
  if (st != TN_OK) return st;
  TN_CUDA(batch_run(b, params_dev, static_cast<float2 *>(states_dev), workspace_dev, reinterpret_cast<cudaStream_t>(s)),
          "batched executor");
  return TN_OK;
}

tn_status tn_batch_params(const tn_batch *b, int32_t *n_params, int64_t *param_offsets) {
  TN_CHECK_ARG(b != nullptr && n_params != nullptr, "NULL argument");
  *n_params = batch_num_params(b, reinterpret_cast<long long *>(param_offsets));
  return TN_OK;
}

tn_status tn_batch_build_tuned(const tn_circuit *const *circuits, int32_t n_circuits, const tn_tune_opts *opts,
                               tn_stream_t s, tn_batch **out, int32_t *tiles_out) {
  TN_CHECK_ARG(out != nullptr && circuits != nullptr, "NULL argument");
  TN_CHECK_ARG(n_circuits >= 1 && n_circuits <= (1 << 20), "n_circuits=%d out of range", n_circuits);
  *out = nullptr;
  tn_tune_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  for (int i = 0; i < 8 && o.candidates[i] != 0; ++i)
    TN_CHECK_ARG(o.candidates[i] >= kLowBits + 2 && o.candidates[i] <= 12, "candidate tile %d not in [6, 12]",
                 o.candidates[i]);
  TN_CHECK_ARG(o.reps >= 0 && o.reps <= 100, "reps=%d out of range", o.reps);
  TN_CHECK_ARG(o.flags == 0, "flags must be zero");
  for (int i = 0; i < 4; ++i) TN_CHECK_ARG(o.reserved[i] == 0, "reserved fields must be zero");
  for (int i = 0; i < n_circuits; ++i) {
    TN_CHECK_ARG(circuits[i] != nullptr, "circuit %d is NULL", i);
    TN_CHECK_ARG(circuits[i]->n_params == 0, "circuit %d has parameters (the executor takes fixed angles)", i);
    TN_CHECK_ARG(circuits[i]->n >= 1 && circuits[i]->n <= kMaxQubits, "circuit %d: %d qubits", i, circuits[i]->n);
  }
  return batch_build_tuned(circuits, n_circuits, o, reinterpret_cast<cudaStream_t>(s), out, tiles_out);
}

void tn_free_batch(tn_batch *b) { batch_free(b); }

tn_status tn_probe_fma_rate(double *tflops, double *seconds) {
  TN_CHECK_ARG(tflops != nullptr, "NULL argument");
  return probe_fma_rate(tflops, seconds);
}

tn_status tn_batch_test_stall(tn_batch *b, int32_t circ, int32_t pass, int64_t wait_limit_ns) {
  TN_CHECK_ARG(b != nullptr, "NULL argument");
  tn_status st = check_device(batch_device(b));
  if (st != TN_OK) return st;
  return batch_test_stall(b, circ, pass, (long long)wait_limit_ns);
}

tn_status tn_sync_status(tn_stream_t s) {
  int v = 0;
  cudaError_t e = read_and_clear_status(&v, reinterpret_cast<cudaStream_t>(s));
  if (e != cudaSuccess) return cuda_fail(e, "tn_sync_status");
  if (v == TN_ERR_TIMEOUT) {
    set_error("a device-side wait ran out of its iteration budget");
    return TN_ERR_TIMEOUT;
  }
  if (v != 0) {
    set_error("device status word = %d", v);
    return (tn_status)v;
  }
  return TN_OK;
}

}  // extern "C"
