// Persistent batched executor: the passes of many circuits of uneven size in one launch.
//
// Every circuit's contraction is a chain of passes (rank-growing contractions grouped by
// the planner, Sec. 2.2.3: the order is fixed before evaluation); a pass is a set of
// independent tiles.  The executor lays all (circuit, pass, tile) work items out in one
// list, pass-major across circuits, and each CTA of a grid sized to full co-residency
// claims the next item with one atomic counter.  A tile of pass p of a circuit may start
// only once every tile of pass p-1 of that circuit has been stored; since items are claimed
// in list order and every earlier item is held by a resident CTA, the wait always ends
// (it is nevertheless bounded: after ~2 s the executor records TN_ERR_TIMEOUT, raises a
// global abort flag that every CTA checks, and returns).  Circuits that fit in one tile
// run all of their passes inside one item without going back to HBM.
//
// Wide circuits whose plans carry generated pass kernels (kBatchDirectMinQubits qubits and more:
// at least 128 tiles per pass) do not go through the interpreting executor: a run launches
// their own pass kernels on a few side streams, forked from the caller's stream after the
// gate tables are built and joined back after the persistent launch, so that they share the
// GPU with the executor's small circuits (one graph when captured).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "apply_common.cuh"
#include "kernels.h"

namespace tnq {

struct alignas(16) BatchCirc {
  long long state_off;  // complex64 offset of the circuit's state in the output buffer
  unsigned long long init;
  const PhaseDesc *phases;
  const OpDesc *ops;
  const float2 *mats;   // fixed angles: the plan's table; NULL: the run's table at mats_off
  long long mats_off;   // parameterised circuits: complex64 offset in the run's gate table
  int N;
  int pad;
};

struct alignas(16) BatchTask {
  long long item_begin;  // first global item index of this task
  int circ;
  int pass;  // index into the batch's PassDesc array
  int prev;  // task that must complete first, -1 if none
  int n_tiles;
  int need_extra;  // tiles of prev awaited beyond its count: 0 (1 only under tn_batch_test_stall)
};

namespace {

constexpr int kBatchThreads = 256;  // 2^(12 - 4): the largest tile (12 qubits) with 4 register qubits
constexpr int kBatchT = 12;
constexpr size_t kBatchStageMax = 32 * 1024;  // shared memory for a pass's staged records
constexpr unsigned long long kWaitNs = 2000000000ull;  // default bound of a dependency wait
constexpr int kSideStreams = 4;  // side streams of the wide circuits (measured: 4 beat 1 and 8)

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// three resident CTAs per SM (the work items are latency-bound: more CTAs to overlap tile loads,
// barriers and the dependency waits measured faster than the register spill this costs)
__global__ void __launch_bounds__(kBatchThreads, 3) k_batch_exec(const BatchTask *__restrict__ tasks, int n_tasks,
                                                              const BatchCirc *__restrict__ circs,
                                                              const PassDesc *__restrict__ passes,
                                                              float2 *__restrict__ states, int *done,
                                                              unsigned long long *next_item, int *abort_flag,
                                                              long long total_items, int *status, int stage_cap,
                                                              unsigned long long wait_ns,
                                                              const float2 *__restrict__ run_mats) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ PassDesc pd;
  __shared__ long long s_item;
  __shared__ int s_task, s_go;
  constexpr int K = 4;
  float2 *sm = reinterpret_cast<float2 *>(smem_raw);
  long long *run_off = reinterpret_cast<long long *>(smem_raw + ((size_t)sizeof(float2) << kBatchT));
  const uint32_t full = 0xFFFFu;
  // thread 0 claims the next item while the current tile is stored (the claim's round trip
  // off the path between items); a claimed item only waits on lower items, so holding one
  // while finishing another cannot deadlock
  unsigned long long claimed = threadIdx.x == 0 ? atomicAdd(next_item, 1ull) : 0ull;

  for (;;) {
    if (threadIdx.x == 0) {
      s_item = (long long)claimed;
      s_go = (s_item < total_items && ld_acquire(abort_flag) == 0) ? 1 : 0;
      if (s_go) {
        int lo = 0, hi = n_tasks - 1;  // last task with item_begin <= item
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (tasks[mid].item_begin <= s_item) lo = mid;
          else hi = mid - 1;
        }
        s_task = lo;
        const int prev = tasks[lo].prev;
        if (prev >= 0) {
          const int need = tasks[prev].n_tiles + tasks[lo].need_extra;
          if (ld_acquire(done + prev) < need) {
            const unsigned long long t0 = now_ns();
            for (;;) {
              if (ld_acquire(done + prev) >= need) break;
              if (ld_acquire(abort_flag) != 0 || now_ns() - t0 > wait_ns) {
                atomicCAS(status, 0, (int)TN_ERR_TIMEOUT);
                atomicExch(abort_flag, 1);
                s_go = 0;
                break;
              }
              __nanosleep(200);
            }
          }
        }
      }
    }
    __syncthreads();
    if (!s_go) break;
    const BatchTask task = tasks[s_task];
    BatchCirc circ = circs[task.circ];
    if (circ.mats == nullptr) circ.mats = run_mats + circ.mats_off;
    for (int i = threadIdx.x; i < (int)(sizeof(PassDesc) / 4); i += blockDim.x)
      reinterpret_cast<int *>(&pd)[i] = reinterpret_cast<const int *>(passes + task.pass)[i];
    __syncthreads();
    const int T = pd.T;
    const int L = T < kLowBits ? T : kLowBits;
    const int tile = 1 << T;
    const int lowmask = (1 << L) - 1;
    for (int r = threadIdx.x; r < (1 << (T - L)); r += blockDim.x) {
      long long off = 0;
      for (int j = 0; j < T - L; ++j)
        if ((r >> j) & 1) off |= 1ll << pd.tile_pos[L + j];
      run_off[r] = off;
    }
    // the pass's phase and op records and matrix entries: staged in shared memory when they fit
    // (the gate loop then never waits on a dependent global load)
    const int n_ph = pd.phase_end - pd.phase_begin, n_ops = pd.op_end - pd.op_begin;
    const int n_mat = pd.mat_end - pd.mat_begin;
    const int need = n_ph * (int)sizeof(PhaseDesc) + n_ops * (int)sizeof(OpDesc) + n_mat * (int)sizeof(float2);
    const PhaseDesc *phs = circ.phases;
    const OpDesc *ops = circ.ops;
    const float2 *mats = circ.mats;
    if (need <= stage_cap) {
      PhaseDesc *s_ph = reinterpret_cast<PhaseDesc *>(run_off + (1 << (kBatchT - kLowBits)));
      OpDesc *s_ops = reinterpret_cast<OpDesc *>(s_ph + n_ph);
      float2 *s_mat = reinterpret_cast<float2 *>(s_ops + n_ops);
      stage_int4(reinterpret_cast<int4 *>(s_ph), reinterpret_cast<const int4 *>(circ.phases + pd.phase_begin),
                 n_ph * (int)(sizeof(PhaseDesc) / 16));
      stage_int4(reinterpret_cast<int4 *>(s_ops), reinterpret_cast<const int4 *>(circ.ops + pd.op_begin), n_ops);
      for (int i = threadIdx.x; i < n_mat; i += blockDim.x) s_mat[i] = circ.mats[pd.mat_begin + i];
      phs = s_ph - pd.phase_begin;
      ops = s_ops - pd.op_begin;
      mats = s_mat - pd.mat_begin;
    }
    const long long t = s_item - task.item_begin;
    unsigned long long base = 0, outer_mask = 0;
    for (int j = 0; j < pd.n_outer; ++j) {
      base |= (unsigned long long)((t >> j) & 1) << pd.outer_pos[j];
      outer_mask |= 1ull << pd.outer_pos[j];
    }
    float2 *st = states + circ.state_off;
    __syncthreads();
    if (pd.init_mode && (circ.init & outer_mask) != base) {
      // a basis state is zero outside the one tile that holds it: store zeros, skip the phases
      if (threadIdx.x == 0) claimed = atomicAdd(next_item, 1ull);
      for (int c = threadIdx.x; c < (tile >> 1); c += blockDim.x) {
        const int i = c << 1;
        const long long g = (long long)base + run_off[i >> L] + (i & lowmask);
        *reinterpret_cast<float4 *>(st + g) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(done + s_task, 1);
      }
      continue;
    }
    if (pd.init_mode) {
      for (int i = threadIdx.x; i < tile; i += blockDim.x) sm[swz(i)] = make_float2(0.f, 0.f);
      __syncthreads();
      if (threadIdx.x == 0 && (circ.init & outer_mask) == base) {
        int li = 0;
        for (int j = 0; j < T; ++j) li |= (int)((circ.init >> pd.tile_pos[j]) & 1ull) << j;
        sm[swz(li)] = make_float2(1.f, 0.f);
      }
    } else {
      // written by other CTAs during the previous pass: read through L2, never a stale L1 line
      for (int c = threadIdx.x; c < (tile >> 1); c += blockDim.x) {
        const int i = c << 1;
        const long long g = (long long)base + run_off[i >> L] + (i & lowmask);
        const float4 v = __ldcg(reinterpret_cast<const float4 *>(st + g));
        sm[swz(i)] = make_float2(v.x, v.y);
        sm[swz(i + 1)] = make_float2(v.z, v.w);
      }
    }
    __syncthreads();
    const bool active = threadIdx.x < (1 << (T - K));
    for (int p = pd.phase_begin; p < pd.phase_end; ++p) {
      if (active) {
        const PhaseDesc &ph = phs[p];
        BitCtx ctx;
        ctx.tb = deposit(threadIdx.x, ph.thr_pos, T - K);
        ctx.base = base;
        ctx.full = full;
        const int pb = swz(ctx.tb);
        int ro[1 << K];
        ro[0] = 0;
#pragma unroll
        for (int r = 0; r < K; ++r) {
          const int d = swz(1 << ph.reg_pos[r]);
#pragma unroll
          for (int j = 0; j < (1 << r); ++j) ro[j | (1 << r)] = ro[j] ^ d;
        }
        float2 a[1 << K];
#pragma unroll
        for (int j = 0; j < (1 << K); ++j) a[j] = sm[pb ^ ro[j]];
        uint32_t neg = 0;
        for (int o = ph.op_begin; o < ph.op_end; ++o) {
          OpDesc op;
          *reinterpret_cast<int4 *>(&op) = *reinterpret_cast<const int4 *>(ops + o);
          apply_op<K, false>(a, op, ctx, mats, neg);  // SWAP as a dense 4x4: 80 registers, 3 CTAs per SM
        }
        if (neg) reg_flush_sign<K>(a, neg);
#pragma unroll
        for (int j = 0; j < (1 << K); ++j) sm[pb ^ ro[j]] = a[j];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) claimed = atomicAdd(next_item, 1ull);
    for (int c = threadIdx.x; c < (tile >> 1); c += blockDim.x) {
      const int i = c << 1;
      const long long g = (long long)base + run_off[i >> L] + (i & lowmask);
      const float2 x = sm[swz(i)], y = sm[swz(i + 1)];
      *reinterpret_cast<float4 *>(st + g) = make_float4(x.x, x.y, y.x, y.y);
    }
    // the barrier orders every thread's stores before thread 0's device-scope fence (which is
    // cumulative), so the tile is visible device-wide before it is counted
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(done + s_task, 1);
    }
  }
}

}  // namespace

}  // namespace tnq

// ------------------------------------------------------------------------------ host side

struct tn_batch {
  int n;
  int device;
  std::vector<long long> offsets;
  long long total_elems = 0;
  long long total_items = 0;
  int n_tasks = 0;
  tnq::BatchTask *d_tasks = nullptr;
  tnq::BatchCirc *d_circs = nullptr;
  tnq::PassDesc *d_passes = nullptr;
  size_t ws_bytes = 0;
  int stage_cap = 0;             // shared-memory bytes for a pass's records (largest pass, capped)
  std::vector<tn_plan *> owned;  // plans made for this batch (tile autotuner)
  std::vector<tnq::BatchTask> h_tasks;            // host copy of the task list
  // parameterised circuits: their gate tables are materialised per run (one kernel, all circuits)
  int n_params = 0;                                // parameters of all circuits, back to back
  std::vector<long long> param_offsets;            // first parameter of each circuit
  int n_slots = 0;                                 // matrix slots of the parameterised circuits
  int n_fused_slots = 0;                           //   of which fused blocks (listed first)
  long long run_mats_elems = 0;                    // complex64 entries of the per-run table
  size_t ws_mats = 0;                              // byte offset of that table in the workspace
  tnq::MatSlot *d_slots = nullptr;
  tnq::FusedMember *d_fused = nullptr;
  std::vector<std::vector<int>> circ_tasks;       // tasks of each circuit, pass order
  unsigned long long wait_ns = 2000000000ull;     // dependency-wait bound passed to the kernel
  int stalled_task = -1;                          // task altered by tn_batch_test_stall, -1 if none
  // circuits run by their own generated pass kernels on side streams (most work first)
  std::vector<int> direct;
  std::vector<int> direct_stream;                  // side stream of each
  std::vector<const tn_plan *> plan_ptrs;          // every circuit's plan
  std::vector<long long> mats_off;                 // parameterised circuits: offset in the per-run table
  std::vector<cudaStream_t> side;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
};

namespace tnq {

tn_status batch_build(const tn_plan *const *plans, int n, tn_batch **out) {
  std::vector<BatchCirc> circs((size_t)n);
  std::vector<PassDesc> passes;
  std::vector<std::vector<int>> circ_pass((size_t)n);  // batch pass indices per circuit
  std::vector<MatSlot> all_slots;                       // parameterised circuits' forward slots
  std::vector<FusedMember> all_fused;
  long long run_mats = 0;
  tn_batch *b = new tn_batch();
  b->n = n;
  b->offsets.resize((size_t)n);
  long long off = 0;
  for (int i = 0; i < n; ++i) {
    const tn_plan *p = plans[i];
    if (p == nullptr || p->host_only) {
      delete b;
      set_error("plan %d is NULL or host-only", i);
      return TN_ERR_INVALID_ARG;
    }
    if (p->batch != 1) {
      delete b;
      set_error("plan %d: the batched executor takes plans of batch 1 (one parameter set per circuit)", i);
      return TN_ERR_UNSUPPORTED;
    }
    const bool direct = !p->jit_kernels.empty() && p->n >= kBatchDirectMinQubits;
    if (!direct && (p->K != 4 || p->T > kBatchT || p->T < kLowBits + 2)) {
      delete b;
      set_error("plan %d: the batched executor needs 6 <= tile qubits <= 12 (circuit of %d qubits)", i, p->n);
      return TN_ERR_UNSUPPORTED;
    }
    b->plan_ptrs.push_back(p);
    b->mats_off.push_back(-1);
    if (direct) b->direct.push_back(i);
    BatchCirc &c = circs[(size_t)i];
    std::memset(&c, 0, sizeof(c));
    c.state_off = off;
    c.init = p->init;
    c.phases = p->d_fwd_phase;
    c.ops = p->d_fwd_ops;
    c.mats = reinterpret_cast<const float2 *>(p->d_fixed_mats);
    c.mats_off = 0;
    c.N = p->n;
    b->param_offsets.push_back(b->n_params);
    if (p->param_dependent) {
      // its slots join the batch's per-run table: entry offsets, fused members and parameter
      // indices shifted to the circuit's place in the combined tables
      c.mats = nullptr;
      c.mats_off = run_mats;
      b->mats_off[(size_t)i] = run_mats;
      const int fbase = (int)all_fused.size();
      for (const FusedMember &f : p->fused) {
        FusedMember g = f;
        for (int a = 0; a < 3; ++a)
          for (int k = 0; k < 2; ++k)
            if (g.pidx[a][k] >= 0) g.pidx[a][k] += b->n_params;
        all_fused.push_back(g);
      }
      for (const MatSlot &sl : p->slots) {
        if (sl.form != FORM_U) continue;  // forward entries only (the executor runs no adjoint)
        MatSlot t = sl;
        t.offset += (int)run_mats;
        if (t.kind == KIND_F2) t.fuse_begin += fbase;
        for (int a = 0; a < 3; ++a)
          for (int k = 0; k < 2; ++k)
            if (t.pidx[a][k] >= 0) t.pidx[a][k] += b->n_params;
        all_slots.push_back(t);
      }
      run_mats += (p->mstride + 1) & ~1ll;
      b->n_params += p->n_params;
    }
    b->offsets[(size_t)i] = off;
    off += 1ll << p->n;
    off = (off + 1) & ~1ll;  // keep every state 16-byte aligned
    if (direct) continue;  // no work items: its own kernels run it
    const bool one_tile = p->fwd.passes.front().n_outer == 0;
    if (one_tile) {  // the whole state is one tile: every pass runs in the same item
      PassDesc m = p->fwd.passes.front();
      m.phase_end = p->fwd.passes.back().phase_end;
      m.op_end = p->fwd.passes.back().op_end;
      m.mat_end = p->fwd.passes.back().mat_end;
      circ_pass[(size_t)i].push_back((int)passes.size());
      passes.push_back(m);
    } else {
      for (const PassDesc &pd : p->fwd.passes) {
        circ_pass[(size_t)i].push_back((int)passes.size());
        passes.push_back(pd);
      }
    }
  }
  b->total_elems = off;
  // side streams of the direct circuits: most work first, each to the least-loaded stream; the
  // uses of one parameterised plan share a stream (its per-call constant tables are rewritten
  // before each launch)
  if (!b->direct.empty()) {
    auto work = [&](int i) { return b->plan_ptrs[(size_t)i]->fwd.passes.size() * std::ldexp(1.0, b->plan_ptrs[(size_t)i]->n); };
    std::stable_sort(b->direct.begin(), b->direct.end(), [&](int x, int y) { return work(x) > work(y); });
    const int ns = std::min<int>(kSideStreams, (int)b->direct.size());
    std::vector<double> load((size_t)ns, 0.0);
    std::vector<std::pair<const tn_plan *, int>> owner;
    for (int i : b->direct) {
      const tn_plan *p = b->plan_ptrs[(size_t)i];
      int k = -1;
      if (p->param_dependent)
        for (auto &o : owner)
          if (o.first == p) k = o.second;
      if (k < 0) {
        k = 0;
        for (int j = 1; j < ns; ++j)
          if (load[(size_t)j] < load[(size_t)k]) k = j;
        if (p->param_dependent) owner.push_back({p, k});
      }
      load[(size_t)k] += work(i);
      b->direct_stream.push_back(k);
    }
    cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    b->side.assign((size_t)ns, nullptr);
    b->join.assign((size_t)ns, nullptr);
    for (int k = 0; e == cudaSuccess && k < ns; ++k) {
      e = cudaStreamCreateWithFlags(&b->side[(size_t)k], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[(size_t)k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
      batch_free(b);
      return cuda_fail(e, "batch side streams");
    }
  }
  // staging budget: the largest pass's phase/op records and matrix entries, up to 32 KB
  size_t stage = 0;
  for (const PassDesc &pd : passes)
    stage = std::max(stage, (size_t)(pd.phase_end - pd.phase_begin) * sizeof(PhaseDesc) +
                                (size_t)(pd.op_end - pd.op_begin) * sizeof(OpDesc) +
                                (size_t)(pd.mat_end - pd.mat_begin) * sizeof(float2));
  b->stage_cap = (int)std::min<size_t>((stage + 15) & ~(size_t)15, kBatchStageMax);
  // pass-major task list
  std::vector<BatchTask> tasks;
  std::vector<int> last_task((size_t)n, -1);
  size_t max_p = 0;
  for (auto &v : circ_pass) max_p = std::max(max_p, v.size());
  long long items = 0;
  for (size_t pi = 0; pi < max_p; ++pi)
    for (int i = 0; i < n; ++i) {
      if (pi >= circ_pass[(size_t)i].size()) continue;
      BatchTask t;
      std::memset(&t, 0, sizeof(t));
      t.item_begin = items;
      t.circ = i;
      t.pass = circ_pass[(size_t)i][pi];
      t.prev = last_task[(size_t)i];
      t.n_tiles = 1 << passes[(size_t)t.pass].n_outer;
      items += t.n_tiles;
      last_task[(size_t)i] = (int)tasks.size();
      tasks.push_back(t);
    }
  b->circ_tasks.assign((size_t)n, {});
  for (size_t k = 0; k < tasks.size(); ++k) b->circ_tasks[(size_t)tasks[k].circ].push_back((int)k);
  b->h_tasks = tasks;
  b->total_items = items;
  b->n_tasks = (int)tasks.size();
  b->ws_bytes = ((size_t)b->n_tasks * sizeof(int) + 255) / 256 * 256 + 256;
  b->n_slots = (int)all_slots.size();
  b->run_mats_elems = run_mats;
  b->ws_mats = b->ws_bytes;
  b->ws_bytes += ((size_t)run_mats * sizeof(float2) + 255) / 256 * 256;
  cudaError_t e = cudaGetDevice(&b->device);
  auto up = [&](const void *src, size_t bytes, void **dst) {
    if (e != cudaSuccess) return;
    e = cudaMalloc(dst, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
  };
  up(tasks.data(), sizeof(BatchTask) * tasks.size(), (void **)&b->d_tasks);
  up(circs.data(), sizeof(BatchCirc) * circs.size(), (void **)&b->d_circs);
  up(passes.data(), sizeof(PassDesc) * passes.size(), (void **)&b->d_passes);
  b->n_fused_slots = order_slots_fused_first(all_slots);
  if (!all_slots.empty()) up(all_slots.data(), sizeof(MatSlot) * all_slots.size(), (void **)&b->d_slots);
  if (!all_fused.empty()) up(all_fused.data(), sizeof(FusedMember) * all_fused.size(), (void **)&b->d_fused);
  if (e != cudaSuccess) {
    batch_free(b);  // the tables allocated so far, the side streams and their events
    return cuda_fail(e, "batched executor tables");
  }
  *out = b;
  return TN_OK;
}

cudaError_t batch_run(const tn_batch *b, const double *params, float2 *states, void *ws, cudaStream_t s) {
  // workspace: [done counters per task][next item (u64)][abort flag][per-run gate table]
  char *w = static_cast<char *>(ws);
  int *done = reinterpret_cast<int *>(w);
  const size_t counters = ((size_t)b->n_tasks * sizeof(int) + 255) / 256 * 256;
  unsigned long long *next = reinterpret_cast<unsigned long long *>(w + counters);
  int *abort_flag = reinterpret_cast<int *>(w + counters + 8);
  float2 *run_mats = reinterpret_cast<float2 *>(w + b->ws_mats);
  cudaError_t e = cudaMemsetAsync(ws, 0, b->ws_mats, s);
  if (e != cudaSuccess) return e;
  if (b->n_slots > 0) {  // every parameterised circuit's gate table, one kernel
    e = launch_materialize(b->d_slots, b->n_slots, b->n_fused_slots, b->d_fused, params, b->n_params, 1, 0, run_mats, s);
    if (e != cudaSuccess) return e;
  }
  // wide circuits: their own pass kernels on the side streams (forked after the gate tables)
  const int ns = (int)b->side.size();
  if (ns > 0) {
    e = cudaEventRecord(b->fork, s);
    for (int k = 0; e == cudaSuccess && k < ns; ++k) e = cudaStreamWaitEvent(b->side[(size_t)k], b->fork, 0);
    for (size_t j = 0; e == cudaSuccess && j < b->direct.size(); ++j) {
      const int i = b->direct[j];
      const tn_plan *p = b->plan_ptrs[(size_t)i];
      const float2 *m = p->param_dependent ? run_mats + b->mats_off[(size_t)i] : reinterpret_cast<const float2 *>(p->d_fixed_mats);
      e = launch_forward(p, m, p->mstride, states + b->offsets[(size_t)i], b->side[(size_t)b->direct_stream[j]],
                         false);  // ordinary launches: the GPU is shared with the other streams
    }
    if (e != cudaSuccess) return e;
  }
  if (b->total_items > 0) {
    const size_t smem = ((size_t)sizeof(float2) << kBatchT) +
                        ((size_t)1 << (kBatchT - kLowBits)) * sizeof(long long) + (size_t)b->stage_cap;
    e = ensure_smem(reinterpret_cast<const void *>(k_batch_exec), smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_exec, kBatchThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    // never more CTAs than can be resident at once: a CTA may wait for items held by others
    long long grid = (long long)num_sms() * per_sm;
    if (grid > b->total_items) grid = b->total_items;
    k_batch_exec<<<(unsigned)grid, kBatchThreads, smem, s>>>(b->d_tasks, b->n_tasks, b->d_circs, b->d_passes, states,
                                                             done, next, abort_flag, b->total_items,
                                                             static_cast<int *>(status_word_ptr()), b->stage_cap,
                                                             b->wait_ns, run_mats);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // join the side streams back into the caller's stream
  for (int k = 0; e == cudaSuccess && k < ns; ++k) {
    e = cudaEventRecord(b->join[(size_t)k], b->side[(size_t)k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->join[(size_t)k], 0);
  }
  return e;
}

tn_status batch_sizes(const tn_batch *b, long long *elems, size_t *ws) {
  *elems = b->total_elems;
  *ws = b->ws_bytes;
  return TN_OK;
}

tn_status batch_offsets(const tn_batch *b, long long *offsets) {
  for (int i = 0; i < b->n; ++i) offsets[i] = b->offsets[(size_t)i];
  return TN_OK;
}

int batch_device(const tn_batch *b) { return b->device; }

tn_status batch_test_stall(tn_batch *b, int circ, int pass, long long wait_ns) {
  auto upload = [&](int k) -> cudaError_t {
    return cudaMemcpy(b->d_tasks + k, &b->h_tasks[(size_t)k], sizeof(BatchTask), cudaMemcpyHostToDevice);
  };
  // restore the table and the default bound first
  if (b->stalled_task >= 0) {
    b->h_tasks[(size_t)b->stalled_task].need_extra = 0;
    const cudaError_t e = upload(b->stalled_task);
    if (e != cudaSuccess) return cuda_fail(e, "batch task table");
    b->stalled_task = -1;
  }
  b->wait_ns = kWaitNs;
  if (circ < 0) return TN_OK;
  if (circ >= b->n) {
    set_error("circuit %d out of range (batch of %d)", circ, b->n);
    return TN_ERR_INVALID_ARG;
  }
  const std::vector<int> &ts = b->circ_tasks[(size_t)circ];
  if (pass < 1 || pass >= (int)ts.size()) {
    set_error("circuit %d has %d work-list passes; a stall needs 1 <= pass < %d", circ, (int)ts.size(),
              (int)ts.size());
    return TN_ERR_INVALID_ARG;
  }
  if (wait_ns < 1000000ll || wait_ns > 10000000000ll) {
    set_error("wait_limit_ns must be within [1e6, 1e10]");
    return TN_ERR_INVALID_ARG;
  }
  const int k = ts[(size_t)pass];
  b->h_tasks[(size_t)k].need_extra = 1;
  const cudaError_t e = upload(k);
  if (e != cudaSuccess) return cuda_fail(e, "batch task table");
  b->stalled_task = k;
  b->wait_ns = (unsigned long long)wait_ns;
  return TN_OK;
}

int batch_num_params(const tn_batch *b, long long *offsets) {
  if (offsets)
    for (int i = 0; i < b->n; ++i) offsets[i] = b->param_offsets[(size_t)i];
  return b->n_params;
}

void batch_free(tn_batch *b) {
  if (!b) return;
  cudaFree(b->d_slots);
  cudaFree(b->d_fused);
  cudaFree(b->d_tasks);
  cudaFree(b->d_circs);
  cudaFree(b->d_passes);
  for (cudaStream_t t : b->side)
    if (t) cudaStreamDestroy(t);
  for (cudaEvent_t ev : b->join)
    if (ev) cudaEventDestroy(ev);
  if (b->fork) cudaEventDestroy(b->fork);
  for (tn_plan *p : b->owned) tn_free_plan(p);
  delete b;
}

void batch_adopt_plans(tn_batch *b, const std::vector<tn_plan *> &plans) {
  b->owned.insert(b->owned.end(), plans.begin(), plans.end());
}

}  // namespace tnq
