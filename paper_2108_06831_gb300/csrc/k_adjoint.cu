// Adjoint sweep for d<H>/d(theta).
//
// With psi_k = U_k ... U_1 |x0> and lambda_k = U_{k+1}^dag ... U_G^dag H psi_G, the
// derivative of <H> = <psi_G|H|psi_G> w.r.t. an angle a of gate k is
// 2 Re <lambda_k| dU_k/da |psi_{k-1}>.  The sweep walks the gates backwards carrying both
// states: psi_{k-1} = U_k^dag psi_k, the derivative dot, lambda_{k-1} = U_k^dag lambda_k.
// It reuses the forward kernel's tiling: the adjoint plan is the reversed gate list with
// conjugate-transposed tables, grouped into passes and register phases the same way,
// with two tiles (psi, lambda) staged per CTA.  Derivative dots are reduced in FP32 per
// warp, accumulated per CTA in FP64 in shared memory, and added to grad once per CTA.
#include "apply_common.cuh"
#include "kernels.h"

namespace tnq {

namespace {

__device__ __forceinline__ float re_conj_mul(float2 l, float2 v) { return fmaf(l.x, v.x, l.y * v.y); }

template <int K, int R>
__device__ __forceinline__ float grad_dot_g1(const float2 (&a)[1 << K], const float2 (&l)[1 << K], float2 d00,
                                             float2 d01, float2 d10, float2 d11) {
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < (1 << K); ++j) {
    if (j & (1 << R)) continue;
    const int j1 = j | (1 << R);
    const float2 x = a[j], y = a[j1];
    acc += re_conj_mul(l[j], cmul2(d00, x, d01, y));
    acc += re_conj_mul(l[j1], cmul2(d10, x, d11, y));
  }
  return acc;
}

// 2 sum_j Re(conj(l_j) (D a)_j) for the derivative D of op (entries at dm).
template <int K>
__device__ __forceinline__ float grad_dot(const float2 (&a)[1 << K], const float2 (&l)[1 << K], const OpDesc &op,
                                          const BitCtx &c, const float2 *dm) {
  float acc = 0.f;
  if (op.type == OP_G1) {
    const float4 m01 = ld4(dm);
    const float4 m23 = ld4(dm + 2);
    const float2 d00 = make_float2(m01.x, m01.y), d01 = make_float2(m01.z, m01.w);
    const float2 d10 = make_float2(m23.x, m23.y), d11 = make_float2(m23.z, m23.w);
    switch (op.a_pos) {
      case 0: acc = grad_dot_g1<K, 0>(a, l, d00, d01, d10, d11); break;
      case 1: if constexpr (K > 1) acc = grad_dot_g1<K, 1>(a, l, d00, d01, d10, d11); break;
      case 2: if constexpr (K > 2) acc = grad_dot_g1<K, 2>(a, l, d00, d01, d10, d11); break;
      case 3: if constexpr (K > 3) acc = grad_dot_g1<K, 3>(a, l, d00, d01, d10, d11); break;
      case 4: if constexpr (K > 4) acc = grad_dot_g1<K, 4>(a, l, d00, d01, d10, d11); break;
    }
  } else if (op.type == OP_D1) {
    const float4 d = ld4(dm);
    const float2 d0 = make_float2(d.x, d.y), d1 = make_float2(d.z, d.w);
    const uint32_t m = src_mask(c, op.a_kind, op.a_pos);
#pragma unroll
    for (int j = 0; j < (1 << K); ++j) acc += re_conj_mul(l[j], cmul(a[j], csel((m >> j) & 1u, d1, d0)));
  } else if (op.type == OP_DP) {
    const float2 e = ldg_c(dm);
    const uint32_t m = src_mask(c, op.a_kind, op.a_pos) & src_mask(c, op.b_kind, op.b_pos);
#pragma unroll
    for (int j = 0; j < (1 << K); ++j)
      if ((m >> j) & 1u) acc += re_conj_mul(l[j], cmul(a[j], e));
  }
  return 2.f * acc;
}

}  // namespace

template <int K>
__global__ void __launch_bounds__(512) k_bwd_pass(const PassDesc *__restrict__ pdesc,
                                                   const PhaseDesc *__restrict__ phases,
                                                   const OpDesc *__restrict__ ops,
                                                   const GradRec *__restrict__ grads,
                                                   const float2 *__restrict__ mats, long long mstride,
                                                   float2 *__restrict__ psi, float2 *__restrict__ lam,
                                                   double *__restrict__ grad, int n_params, int N) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ PassDesc pd;
  for (int i = threadIdx.x; i < (int)(sizeof(PassDesc) / 4); i += blockDim.x)
    reinterpret_cast<int *>(&pd)[i] = reinterpret_cast<const int *>(pdesc)[i];
  __syncthreads();
  const int T = pd.T;
  const int L = T < kLowBits ? T : kLowBits;
  const int tile = 1 << T;
  const int nthr = blockDim.x;
  const int nwarps = (nthr + 31) >> 5;
  float2 *sp = reinterpret_cast<float2 *>(smem_raw);
  float2 *sl = sp + tile;
  long long *run_off = reinterpret_cast<long long *>(sl + tile);
  double *gacc = reinterpret_cast<double *>(run_off + (1 << (T - L)));  // [grad_slots]
  float *wacc = reinterpret_cast<float *>(gacc + pd.grad_slots);        // [grad_slots][nwarps]
  for (int r = threadIdx.x; r < (1 << (T - L)); r += nthr) {
    long long off = 0;
    for (int j = 0; j < T - L; ++j)
      if ((r >> j) & 1) off |= 1ll << pd.tile_pos[L + j];
    run_off[r] = off;
  }
  for (int s = threadIdx.x; s < pd.grad_slots; s += nthr) gacc[s] = 0.0;
  __syncthreads();

  const long long n_tiles = 1ll << pd.n_outer;
  const int b = blockIdx.y;
  const uint32_t full = (K >= 5) ? 0xFFFFFFFFu : ((1u << (1 << K)) - 1u);
  const int lowmask = (1 << L) - 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned wmask = nthr >= 32 ? 0xFFFFFFFFu : ((1u << nthr) - 1u);
  float2 *gp = psi + ((long long)b << N);
  float2 *gl = lam + ((long long)b << N);
  const float2 *mb = mats + (long long)b * mstride;

  for (long long t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    unsigned long long base = 0;
    for (int j = 0; j < pd.n_outer; ++j) base |= (unsigned long long)((t >> j) & 1) << pd.outer_pos[j];
    for (int c = threadIdx.x; c < (tile >> 1); c += nthr) {
      const int i = c << 1;
      const long long g = (long long)base + run_off[i >> L] + (i & lowmask);
      const float4 v = *reinterpret_cast<const float4 *>(gp + g);
      const float4 w = *reinterpret_cast<const float4 *>(gl + g);
      sp[swz(i)] = make_float2(v.x, v.y);
      sp[swz(i + 1)] = make_float2(v.z, v.w);
      sl[swz(i)] = make_float2(w.x, w.y);
      sl[swz(i + 1)] = make_float2(w.z, w.w);
    }
    for (int s = threadIdx.x; s < pd.grad_slots * nwarps; s += nthr) wacc[s] = 0.f;
    __syncthreads();

    for (int p = pd.phase_begin; p < pd.phase_end; ++p) {
      const PhaseDesc &ph = phases[p];
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
      float2 a[1 << K], l[1 << K];
#pragma unroll
      for (int j = 0; j < (1 << K); ++j) {
        a[j] = sp[pb ^ ro[j]];
        l[j] = sl[pb ^ ro[j]];
      }
      uint32_t neg = 0;
      for (int o = ph.op_begin; o < ph.op_end; ++o) {
        const int4 raw = __ldg(reinterpret_cast<const int4 *>(ops + o));
        OpDesc op;
        *reinterpret_cast<int4 *>(&op) = raw;
        if (op.has_grad) {
          reg_flush_sign<K>(a, neg);
          reg_flush_sign<K>(l, neg);
          neg = 0;
          uint32_t dummy = 0;
          apply_op<K>(a, op, ctx, mb, dummy);  // psi_{k-1} = U^dag psi_k
          for (int gi = 0; gi < op.n_grad; ++gi) {
            const GradRec gr = grads[op.aux + gi];
            float v = grad_dot<K>(a, l, op, ctx, mb + gr.mat);
            for (int off = (nthr >= 32 ? 16 : nthr >> 1); off > 0; off >>= 1) v += __shfl_xor_sync(wmask, v, off);
            if (lane == 0) wacc[gr.slot * nwarps + warp] += v;
          }
          apply_op<K>(l, op, ctx, mb, dummy);  // lambda_{k-1} = U^dag lambda_k
        } else {
          uint32_t neg_l = neg;
          apply_op<K>(a, op, ctx, mb, neg);
          apply_op<K>(l, op, ctx, mb, neg_l);
        }
      }
      reg_flush_sign<K>(a, neg);
      reg_flush_sign<K>(l, neg);
#pragma unroll
      for (int j = 0; j < (1 << K); ++j) {
        sp[pb ^ ro[j]] = a[j];
        sl[pb ^ ro[j]] = l[j];
      }
      __syncthreads();
    }

    for (int c = threadIdx.x; c < (tile >> 1); c += nthr) {
      const int i = c << 1;
      const long long g = (long long)base + run_off[i >> L] + (i & lowmask);
      const float2 x = sp[swz(i)], y = sp[swz(i + 1)];
      const float2 u = sl[swz(i)], v = sl[swz(i + 1)];
      *reinterpret_cast<float4 *>(gp + g) = make_float4(x.x, x.y, y.x, y.y);
      *reinterpret_cast<float4 *>(gl + g) = make_float4(u.x, u.y, v.x, v.y);
    }
    for (int s = threadIdx.x; s < pd.grad_slots; s += nthr) {
      float v = 0.f;
      for (int w = 0; w < nwarps; ++w) v += wacc[s * nwarps + w];
      gacc[s] += (double)v;
    }
    __syncthreads();
  }
  // one FP64 add per slot and CTA (slot -> parameter through the pass's records)
  const int rec0 = pd.grad_begin;  // first GradRec of this pass; slot s is record rec0 + s
  for (int s = threadIdx.x; s < pd.grad_slots; s += nthr) {
    const GradRec gr = grads[rec0 + s];
    atomicAdd(grad + (long long)b * n_params + gr.param, gacc[s]);
  }
}

namespace {
template <int K>
cudaError_t launch_bwd_k(const PassDesc &h, const PassDesc *d_pass, const tn_plan *p, const float2 *mats,
                         long long mstride, float2 *psi, float2 *lam, double *grad, cudaStream_t s) {
  const int T = h.T;
  const int L = T < kLowBits ? T : kLowBits;
  const int threads = 1 << (T - K);
  const int nwarps = (threads + 31) / 32;
  const size_t smem = 2 * ((size_t)1 << T) * sizeof(float2) + ((size_t)1 << (T - L)) * sizeof(long long) +
                      (size_t)h.grad_slots * sizeof(double) + (size_t)h.grad_slots * nwarps * sizeof(float);
  cudaError_t e = ensure_smem(reinterpret_cast<const void *>(k_bwd_pass<K>), smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bwd_pass<K>, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const long long n_tiles = 1ll << h.n_outer;
  long long gx = ((long long)num_sms() * per_sm + p->batch - 1) / p->batch;
  if (gx > n_tiles) gx = n_tiles;
  if (gx < 1) gx = 1;
  dim3 grid((unsigned)gx, (unsigned)p->batch);
  k_bwd_pass<K><<<grid, threads, smem, s>>>(d_pass, p->d_bwd_phase, p->d_bwd_ops, p->d_bwd_grads, mats, mstride, psi,
                                            lam, grad, p->n_params, p->n);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_backward(const tn_plan *p, const float2 *mats, long long mstride, float2 *psi, float2 *lam,
                            double *grad, cudaStream_t s) {
  if (!p->jit_bwd_kernels.empty()) {
    for (size_t i = 0; i < p->bwd.passes.size(); ++i) {
      const PassDesc &h = p->bwd.passes[i];
      const int threads = p->jit_bwd_threads[i];
      const size_t smem = p->jit_bwd_smem[i];
      const int per_sm = i < p->jit_bwd_grid.size() ? p->jit_bwd_grid[i] : 1;  // queried at load time
      cudaError_t e = cudaSuccess;
      const long long n_tiles = 1ll << h.n_outer;
      long long gx = ((long long)num_sms() * per_sm + p->batch - 1) / p->batch;
      if (gx > n_tiles) gx = n_tiles;
      if (gx < 1) gx = 1;
      const float2 *m = mats;
      int np = p->n_params;
      void *args[] = {(void *)&m, (void *)&mstride, (void *)&psi, (void *)&lam, (void *)&grad, (void *)&np};
      e = launch_pdl_func((const void *)p->jit_bwd_kernels[i], dim3((unsigned)gx, (unsigned)p->batch), dim3(threads),
                          args, smem, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  for (size_t i = 0; i < p->bwd.passes.size(); ++i) {
    const PassDesc &h = p->bwd.passes[i];
    cudaError_t e = cudaSuccess;
    switch (h.K) {
      case 1: e = launch_bwd_k<1>(h, p->d_bwd_pass + i, p, mats, mstride, psi, lam, grad, s); break;
      case 2: e = launch_bwd_k<2>(h, p->d_bwd_pass + i, p, mats, mstride, psi, lam, grad, s); break;
      case 3: e = launch_bwd_k<3>(h, p->d_bwd_pass + i, p, mats, mstride, psi, lam, grad, s); break;
      case 4: e = launch_bwd_k<4>(h, p->d_bwd_pass + i, p, mats, mstride, psi, lam, grad, s); break;
      default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace tnq
