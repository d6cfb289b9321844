// Tile autotuner of the batched executor.
//
// The contraction order of every circuit is fixed by its plan (Sec. 2.2.3: chosen before
// evaluation); what remains free is how the order is cut into work: the tile size T (qubits
// per tile) decides how many passes a circuit takes, how many independent tiles each pass
// offers the persistent executor, and whether a small circuit runs as one item.  No cost
// model predicts the interleaving of hundreds of uneven circuits on 152 SMs well, so the
// tuner measures: circuits are grouped by qubit count, classes are visited in order of
// decreasing work (amplitudes x gates), and for each class every candidate T is tried with
// the other classes held at their current choice; the whole batch is launched and timed
// with CUDA events on the caller's stream, and the fastest T is kept (one coordinate-descent
// sweep).  Planning here is host work; the timed launches are the real executor.  Circuits of
// kBatchDirectMinQubits qubits and more get plan-specialised kernels at the default tile instead
// (compiled on a pool of host threads, one circuit per thread), which the batch runs on its side
// streams; they take part in every timed launch, so the small classes are tuned beside them.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "kernels.h"
#include "tnq_internal.h"

namespace tnq {

namespace {

struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  cudaError_t reserve(size_t n) {
    if (n <= bytes) return cudaSuccess;
    cudaFree(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&p, n);
    if (e == cudaSuccess) bytes = n;
    return e;
  }
  ~DevBuf() { cudaFree(p); }
};

}  // namespace

tn_status batch_build_tuned(const tn_circuit *const *circuits, int n, const tn_tune_opts &o, cudaStream_t s,
                            tn_batch **out, int32_t *tiles_out) {
  std::vector<int> cands;
  for (int i = 0; i < 8 && o.candidates[i] != 0; ++i) cands.push_back(o.candidates[i]);
  if (cands.empty()) cands = {8, 9, 10, 11, 12};
  const int reps = o.reps > 0 ? o.reps : 3;

  // plans per (circuit, T), made on demand; the chosen ones end up owned by the batch
  std::map<std::pair<int, int>, tn_plan *> plans;
  auto release_all = [&](const std::vector<int> *keep) {
    for (auto &kv : plans)
      if (!keep || (*keep)[(size_t)kv.first.first] != kv.first.second) tn_free_plan(kv.second);
    plans.clear();
  };
  auto plan_of = [&](int i, int T, tn_status *st) -> tn_plan * {
    auto it = plans.find({i, T});
    if (it != plans.end()) return it->second;
    tn_plan_opts po;
    std::memset(&po, 0, sizeof(po));
    po.target = TN_TARGET_STATE;
    po.batch = 1;
    po.tile_qubits = T;
    po.flags = TN_PLAN_NO_SPECIALIZE;  // the executor runs the plan's tables, not generated kernels
    tn_plan *p = nullptr;
    *st = tn_plan_contraction(circuits[i], &po, &p);
    if (*st == TN_OK) plans[{i, T}] = p;
    return p;
  };

  std::vector<int> T((size_t)n);
  for (int i = 0; i < n; ++i) T[(size_t)i] = std::min(circuits[i]->n, 12);

  // wide circuits: specialised plans at the default tile, built in parallel (each thread on the
  // caller's device)
  {
    std::vector<int> wide;
    for (int i = 0; i < n; ++i)
      if (circuits[i]->n >= kBatchDirectMinQubits) wide.push_back(i);
    std::vector<tn_plan *> made(wide.size(), nullptr);
    std::vector<tn_status> sts(wide.size(), TN_OK);
    std::vector<std::string> errs(wide.size());
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return cuda_fail(ce, "autotune device");
    std::atomic<size_t> next(0);
    auto worker = [&]() {
      if (cudaSetDevice(dev) != cudaSuccess) return;
      for (size_t k = next++; k < wide.size(); k = next++) {
        tn_plan_opts po;
        std::memset(&po, 0, sizeof(po));
        po.target = TN_TARGET_STATE;
        po.batch = 1;
        sts[k] = tn_plan_contraction(circuits[wide[k]], &po, &made[k]);
        if (sts[k] != TN_OK) errs[k] = tn_last_error();
      }
    };
    const unsigned hw = std::thread::hardware_concurrency();
    const size_t nthreads = std::min<size_t>(wide.size(), std::max(1u, std::min(hw, 16u)));
    std::vector<std::thread> pool;
    for (size_t t = 0; t < nthreads; ++t) pool.emplace_back(worker);
    for (auto &th : pool) th.join();
    tn_status bad = TN_OK;
    std::string bad_err;
    for (size_t k = 0; k < wide.size(); ++k) {
      if (made[k] == nullptr && sts[k] == TN_OK) {  // the worker could not select the device
        sts[k] = TN_ERR_CUDA;
        errs[k] = "autotune: selecting the device on a planning thread failed";
      }
      if (sts[k] != TN_OK && bad == TN_OK) {
        bad = sts[k];
        bad_err = errs[k];
      }
    }
    if (bad != TN_OK) {
      for (tn_plan *p : made)
        if (p) tn_free_plan(p);
      set_error("%s", bad_err.c_str());
      return bad;
    }
    for (size_t k = 0; k < wide.size(); ++k) {
      T[(size_t)wide[k]] = made[k]->T;
      plans[{wide[k], made[k]->T}] = made[k];
    }
  }

  // classes by qubit count (the executor's circuits), most work first
  std::map<int, std::vector<int>> by_n;
  std::map<int, double> work;
  for (int i = 0; i < n; ++i) {
    if (circuits[i]->n >= kBatchDirectMinQubits && plans.count({i, T[(size_t)i]})) continue;
    by_n[circuits[i]->n].push_back(i);
    work[circuits[i]->n] += std::ldexp(1.0, circuits[i]->n) * (double)(circuits[i]->gates.size() + 1);
  }
  std::vector<int> order;
  for (auto &kv : by_n) order.push_back(kv.first);
  std::sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });

  DevBuf states, ws;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(ce, "autotune events");
  }
  // time the batch for the current choice T (fastest of reps launches, ms)
  auto measure = [&](double *ms) -> tn_status {
    std::vector<const tn_plan *> ps((size_t)n);
    for (int i = 0; i < n; ++i) {
      tn_status st = TN_OK;
      ps[(size_t)i] = plan_of(i, T[(size_t)i], &st);
      if (st != TN_OK) return st;
    }
    tn_batch *b = nullptr;
    tn_status st = batch_build(ps.data(), n, &b);
    if (st != TN_OK) return st;
    long long elems = 0;
    size_t wsb = 0;
    batch_sizes(b, &elems, &wsb);
    cudaError_t e = states.reserve((size_t)elems * sizeof(float2));
    if (e == cudaSuccess) e = ws.reserve(wsb);
    float best = 1e30f;
    for (int r = 0; e == cudaSuccess && r <= reps; ++r) {  // launch 0 warms up
      e = cudaEventRecord(e0, s);
      if (e == cudaSuccess) e = batch_run(b, nullptr, static_cast<float2 *>(states.p), ws.p, s);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float t = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
      if (e == cudaSuccess && r > 0) best = std::min(best, t);
    }
    batch_free(b);
    if (e != cudaSuccess) return cuda_fail(e, "autotune launch");
    int dev_status = TN_OK;
    e = read_and_clear_status(&dev_status, s);
    if (e != cudaSuccess) return cuda_fail(e, "autotune status");
    if (dev_status != TN_OK) {
      set_error("autotune: executor reported status %d", dev_status);
      return (tn_status)dev_status;
    }
    *ms = best;
    return TN_OK;
  };

  double cur = 0;
  tn_status st = measure(&cur);
  for (size_t ci = 0; st == TN_OK && ci < order.size(); ++ci) {
    const int nq = order[ci];
    const std::vector<int> &members = by_n[nq];
    std::vector<int> opts;
    for (int c : cands)
      if (c >= kLowBits + 2 && c <= std::min(nq, 12)) opts.push_back(c);
    if (nq <= 12) opts.push_back(nq);  // the whole circuit as one tile
    std::sort(opts.begin(), opts.end());
    opts.erase(std::unique(opts.begin(), opts.end()), opts.end());
    const int start = T[(size_t)members.front()];
    int best_t = start;
    double best_ms = cur;
    for (int t : opts) {
      if (t == start) continue;
      for (int i : members) T[(size_t)i] = t;
      double ms = 0;
      tn_status s2 = measure(&ms);
      if (s2 == TN_ERR_CUDA || s2 == TN_ERR_TIMEOUT) {
        st = s2;
        break;
      }
      if (s2 == TN_OK && ms < best_ms) {
        best_ms = ms;
        best_t = t;
      }
    }
    for (int i : members) T[(size_t)i] = best_t;
    cur = best_ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != TN_OK) {
    release_all(nullptr);
    return st;
  }
  // final batch over the chosen plans, which it adopts
  std::vector<const tn_plan *> ps((size_t)n);
  std::vector<tn_plan *> owned((size_t)n);
  for (int i = 0; i < n; ++i) {
    tn_status s2 = TN_OK;
    owned[(size_t)i] = plan_of(i, T[(size_t)i], &s2);
    ps[(size_t)i] = owned[(size_t)i];
    if (s2 != TN_OK) {
      release_all(nullptr);
      return s2;
    }
  }
  tn_batch *b = nullptr;
  st = batch_build(ps.data(), n, &b);
  if (st != TN_OK) {
    release_all(nullptr);
    return st;
  }
  release_all(&T);  // frees every plan that was not chosen
  batch_adopt_plans(b, owned);
  if (tiles_out)
    for (int i = 0; i < n; ++i) tiles_out[i] = T[(size_t)i];
  *out = b;
  return TN_OK;
}

}  // namespace tnq

namespace tnq {

// Tile autotuner of one state / expectation plan: the circuit is planned at every candidate tile
// size (qubits per on-chip tile: passes, phases and generated kernels all change with it), each
// plan's forward contraction is timed on the caller's stream (CUDA events, one warm-up call, the
// fastest of reps calls; parameters all zero: the kernels' work does not depend on their values),
// and the fastest plan is returned; the others are freed.
tn_status plan_tuned(const tn_circuit *c, const tn_plan_opts &base, const std::vector<int> &cands, int reps,
                     cudaStream_t s, tn_plan **out, int32_t *tile_out) {
  DevBuf state, ws, params;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaError_t e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  if (e != cudaSuccess) return cuda_fail(e, "autotuner events");
  tn_plan *best = nullptr;
  float best_ms = 0.f;
  int best_T = 0;
  tn_status st = TN_OK;
  for (int T : cands) {
    if (T > c->n && T != cands.front()) continue;  // larger tiles than the register are all the same plan
    tn_plan_opts po = base;
    po.tile_qubits = std::min(T, c->n) >= kLowBits + 2 ? std::min(T, c->n) : 0;
    tn_plan *p = nullptr;
    st = tn_plan_contraction(c, &po, &p);
    if (st != TN_OK) break;
    const size_t sbytes = ((size_t)sizeof(float2) << c->n) * (size_t)po.batch;
    e = state.reserve(sbytes);
    if (e == cudaSuccess) e = ws.reserve(std::max<size_t>(p->ws_bytes, 16));
    if (e == cudaSuccess && c->n_params > 0) {
      e = params.reserve((size_t)c->n_params * (size_t)po.batch * sizeof(double));
      if (e == cudaSuccess) e = cudaMemsetAsync(params.p, 0, (size_t)c->n_params * po.batch * sizeof(double), s);
    }
    if (e != cudaSuccess) {
      tn_free_plan(p);
      st = cuda_fail(e, "autotuner scratch");
      break;
    }
    float ms_min = 0.f;
    for (int r = 0; r <= reps && st == TN_OK; ++r) {
      if (r > 0) e = cudaEventRecord(t0, s);
      if (e == cudaSuccess)
        st = tn_contract_state(p, c->n_params > 0 ? static_cast<const double *>(params.p) : nullptr, state.p, ws.p,
                               reinterpret_cast<tn_stream_t>(s));
      if (st != TN_OK) break;
      if (r > 0) {
        e = cudaEventRecord(t1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e == cudaSuccess && (r == 1 || ms < ms_min)) ms_min = ms;
      }
      if (e != cudaSuccess) st = cuda_fail(e, "autotuner timing");
    }
    if (st != TN_OK) {
      tn_free_plan(p);
      break;
    }
    if (best == nullptr || ms_min < best_ms) {
      if (best) tn_free_plan(best);
      best = p;
      best_ms = ms_min;
      best_T = p->T;
    } else {
      tn_free_plan(p);
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (st != TN_OK) {
    if (best) tn_free_plan(best);
    return st;
  }
  *out = best;
  if (tile_out) *tile_out = best_T;
  return TN_OK;
}

}  // namespace tnq
