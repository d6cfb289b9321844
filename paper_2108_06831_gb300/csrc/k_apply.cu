// Kernel (a): fused gate-apply over the state tensor.
//
// Each gate of the circuit is a small tensor merged into the state by a tensor product
// and a contraction over the gate's input legs (Sec. 2.2.1); applied to the whole state
// that is psi' = (I (x) U (x) I) psi (Sec. 2.1).  One launch ("pass") applies a planned
// group of gates: every CTA repeatedly takes one tile of 2^T amplitudes, stages it in
// shared memory with coalesced 128-bit loads (the low four index bits are always inside
// the tile, so every global access is a 128-byte run), runs the pass's phases (each
// maps K tile bits to registers and applies its ops there) and writes the tile back.
// Tiles are independent, so the grid is persistent: one wave of CTAs sized from the
// occupancy calculator, striding over batch x 2^(N-T) tiles.
#include "apply_common.cuh"
#include "kernels.h"

namespace tnq {

template <int K>
__global__ void __launch_bounds__(512) k_fwd_pass(const PassDesc *__restrict__ pdesc,
                                                   const PhaseDesc *__restrict__ phases,
                                                   const OpDesc *__restrict__ ops_g,
                                                   const float2 *__restrict__ mats_g, long long mstride,
                                                   float2 *__restrict__ state, int N, int batch,
                                                   unsigned long long init_basis, int staged) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ PassDesc pd;
  for (int i = threadIdx.x; i < (int)(sizeof(PassDesc) / 4); i += blockDim.x)
    reinterpret_cast<int *>(&pd)[i] = reinterpret_cast<const int *>(pdesc)[i];
  __syncthreads();
  const int T = pd.T;
  const int L = T < kLowBits ? T : kLowBits;
  const int tile = 1 << T;
  const int nthr = blockDim.x;
  float2 *sm = reinterpret_cast<float2 *>(smem_raw);
  long long *run_off = reinterpret_cast<long long *>(smem_raw + (size_t)tile * sizeof(float2));
  for (int r = threadIdx.x; r < (1 << (T - L)); r += nthr) {
    long long off = 0;
    for (int j = 0; j < T - L; ++j)
      if ((r >> j) & 1) off |= 1ll << pd.tile_pos[L + j];
    run_off[r] = off;
  }
  unsigned long long outer_mask = 0;
  for (int j = 0; j < pd.n_outer; ++j) outer_mask |= 1ull << pd.outer_pos[j];
  // the pass's op records and matrix entries are read by every tile: stage them once
  const int n_ops = pd.op_end - pd.op_begin;
  const int n_mat = pd.mat_end - pd.mat_begin;
  const int n_runs = (1 << (T - L)) < 2 ? 2 : (1 << (T - L));  // 16-byte aligned run table
  OpDesc *s_ops = reinterpret_cast<OpDesc *>(run_off + n_runs);
  float2 *s_mat = reinterpret_cast<float2 *>(s_ops + n_ops);
  const OpDesc *ops = ops_g;
  if (staged) {
    stage_int4(reinterpret_cast<int4 *>(s_ops), reinterpret_cast<const int4 *>(ops_g + pd.op_begin), n_ops);
    ops = s_ops - pd.op_begin;
  }
  long long cur_b = -1;
  __syncthreads();

  const long long n_tiles = 1ll << pd.n_outer;
  const long long work = n_tiles * batch;
  const uint32_t full = (K >= 5) ? 0xFFFFFFFFu : ((1u << (1 << K)) - 1u);
  const int lowmask = (1 << L) - 1;

  for (long long w = blockIdx.x; w < work; w += gridDim.x) {
    const long long b = w >> pd.n_outer;
    const long long t = w & (n_tiles - 1);
    unsigned long long base = 0;
    for (int j = 0; j < pd.n_outer; ++j) base |= (unsigned long long)((t >> j) & 1) << pd.outer_pos[j];
    float2 *st = state + ((long long)b << N);
    const float2 *mb = mats_g + b * mstride;
    if (staged) {
      if (b != cur_b) {
        if (cur_b >= 0) __syncthreads();
        stage_int4(reinterpret_cast<int4 *>(s_mat), reinterpret_cast<const int4 *>(mb + pd.mat_begin), n_mat >> 1);
        cur_b = b;
      }
      mb = s_mat - pd.mat_begin;
    }

    if (pd.init_mode) {
      for (int i = threadIdx.x; i < tile; i += nthr) sm[swz(i)] = make_float2(0.f, 0.f);
      __syncthreads();
      if (threadIdx.x == 0 && (init_basis & outer_mask) == base) {
        int li = 0;
        for (int j = 0; j < T; ++j) li |= (int)((init_basis >> pd.tile_pos[j]) & 1ull) << j;
        sm[swz(li)] = make_float2(1.f, 0.f);
      }
    } else {
      for (int c = threadIdx.x; c < (tile >> 1); c += nthr) {
        const int i = c << 1;
        const long long g = (long long)base + run_off[i >> L] + (i & lowmask);
        const float4 v = *reinterpret_cast<const float4 *>(st + g);
        sm[swz(i)] = make_float2(v.x, v.y);
        sm[swz(i + 1)] = make_float2(v.z, v.w);
      }
    }
    __syncthreads();

    for (int p = pd.phase_begin; p < pd.phase_end; ++p) {
      const PhaseDesc &ph = phases[p];
      const int nthrbits = T - K;
      BitCtx ctx;
      ctx.tb = deposit(threadIdx.x, ph.thr_pos, nthrbits);
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
        const int4 raw = *reinterpret_cast<const int4 *>(ops + o);
        OpDesc op;
        *reinterpret_cast<int4 *>(&op) = raw;
        apply_op<K>(a, op, ctx, mb, neg);
      }
      if (neg) reg_flush_sign<K>(a, neg);
#pragma unroll
      for (int j = 0; j < (1 << K); ++j) sm[pb ^ ro[j]] = a[j];
      __syncthreads();
    }

    for (int c = threadIdx.x; c < (tile >> 1); c += nthr) {
      const int i = c << 1;
      const long long g = (long long)base + run_off[i >> L] + (i & lowmask);
      const float2 x = sm[swz(i)], y = sm[swz(i + 1)];
      *reinterpret_cast<float4 *>(st + g) = make_float4(x.x, x.y, y.x, y.y);
    }
    __syncthreads();
  }
}

namespace {
constexpr size_t kStageBytes = 48 * 1024;  // ops + matrices staged in shared memory when they fit

template <int K>
cudaError_t launch_fwd_k(const PassDesc &h, const PassDesc *d_pass, const PhaseDesc *d_phases, const OpDesc *d_ops,
                         const float2 *mats, long long mstride, float2 *state, int N, int batch,
                         unsigned long long init, cudaStream_t s) {
  const int T = h.T;
  const int L = T < kLowBits ? T : kLowBits;
  const int threads = 1 << (T - K);
  const size_t n_runs = ((size_t)1 << (T - L)) < 2 ? 2 : ((size_t)1 << (T - L));
  size_t smem = ((size_t)1 << T) * sizeof(float2) + n_runs * sizeof(long long);
  const size_t stage = (size_t)(h.op_end - h.op_begin) * sizeof(OpDesc) + (size_t)(h.mat_end - h.mat_begin) * sizeof(float2);
  const int staged = stage <= kStageBytes ? 1 : 0;
  if (staged) smem += stage;
  cudaError_t e = ensure_smem(reinterpret_cast<const void *>(k_fwd_pass<K>), smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fwd_pass<K>, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const long long work = (long long)batch << h.n_outer;
  long long grid = (long long)num_sms() * per_sm;
  if (grid > work) grid = work;
  k_fwd_pass<K><<<(unsigned)grid, threads, smem, s>>>(d_pass, d_phases, d_ops, mats, mstride, state, N, batch, init,
                                                       staged);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_forward(const tn_plan *p, const float2 *mats, long long mstride, float2 *state, cudaStream_t s,
                           bool pdl) {
  if (!p->jit_kernels.empty()) {
    for (size_t i = 0; i < p->fwd.passes.size(); ++i) {
      const PassDesc &h = p->fwd.passes[i];
      const int threads = p->jit_threads[i];
      const size_t smem = p->jit_smem[i];
      const int per_sm = i < p->jit_grid.size() ? p->jit_grid[i] : 1;  // resident CTAs per SM (load time)
      cudaError_t e = cudaSuccess;
      long long work = (long long)p->batch << h.n_outer;
      long long grid = (long long)num_sms() * per_sm;
      if (grid > work) grid = work;
      const float2 *m = mats;
      unsigned long long init = p->init;
      // per-call tables (parameterised, batch 1): this pass's entries into its constant table
      if (p->param_dependent && i < p->jit_cm_ptr.size() && p->jit_cm_ptr[i] && p->jit_cm_bytes[i]) {
        e = cudaMemcpyAsync(p->jit_cm_ptr[i], mats + h.mat_begin, p->jit_cm_bytes[i], cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
      }
      void *args[] = {(void *)&m, (void *)&mstride, (void *)&state, (void *)&work, (void *)&init};
      e = pdl ? launch_pdl_func((const void *)p->jit_kernels[i], dim3((unsigned)grid), dim3(threads), args, smem, s)
              : cudaLaunchKernel((const void *)p->jit_kernels[i], dim3((unsigned)grid), dim3(threads), args, smem, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  for (size_t i = 0; i < p->fwd.passes.size(); ++i) {
    const PassDesc &h = p->fwd.passes[i];
    cudaError_t e = cudaSuccess;
    switch (h.K) {
      case 1: e = launch_fwd_k<1>(h, p->d_fwd_pass + i, p->d_fwd_phase, p->d_fwd_ops, mats, mstride, state, p->n, p->batch, p->init, s); break;
      case 2: e = launch_fwd_k<2>(h, p->d_fwd_pass + i, p->d_fwd_phase, p->d_fwd_ops, mats, mstride, state, p->n, p->batch, p->init, s); break;
      case 3: e = launch_fwd_k<3>(h, p->d_fwd_pass + i, p->d_fwd_phase, p->d_fwd_ops, mats, mstride, state, p->n, p->batch, p->init, s); break;
      case 4: e = launch_fwd_k<4>(h, p->d_fwd_pass + i, p->d_fwd_phase, p->d_fwd_ops, mats, mstride, state, p->n, p->batch, p->init, s); break;
      default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace tnq
