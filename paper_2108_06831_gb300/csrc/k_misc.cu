// Small kernels of libtnq: per-call gate-matrix tables, amplitude gather, gradient
// scaling, device status word.
#include <algorithm>
#include <vector>

#include "apply_common.cuh"
#include "kernels.h"

namespace tnq {

// Gate tensors are built once per call from the parameters (angles in FP64, entries stored as
// complex64).  The slot array lists the fused blocks (KIND_F2) first.  Few fused blocks (small
// batches): each block and batch element takes one warp -- lane m evaluates member m's matrix
// embedded as a 4x4, then lanes 0..15 form the product one entry each, member by member.  Many
// (kFusedPerThread or more): one thread each, members applied in turn to a 4x4 held by the thread
// (all lanes busy; FP64 throughput is what bounds this on GB300).  Either way the product is
// stored in the packed layout (SHAPE_M4X).  Every other slot and batch element takes one thread.
constexpr int kMatWarps = 4;
constexpr long long kFusedPerThread = 1024;  // fused blocks x batch from which each takes one thread

// One regular slot (one gate's matrix) for one batch element; prow: its parameters (may be NULL).
__device__ void materialize_one(const MatSlot &s, const double *prow, float2 *table) {
  double ang[3] = {s.angle[0], s.angle[1], s.angle[2]};
  for (int a = 0; a < 3; ++a)
    for (int q = 0; q < 2; ++q)
      if (s.pidx[a][q] >= 0) ang[a] += prow[s.pidx[a][q]];
  double tmp[32];
  float ent[32];
  const int n = slot_entries(s, ang, tmp, ent);
  float2 *dst = table + s.offset;
  for (int i = 0; i < n; ++i) dst[i] = make_float2(ent[2 * i], ent[2 * i + 1]);
}

__global__ void __launch_bounds__(32 * kMatWarps) k_materialize(const MatSlot *__restrict__ slots, int n_slots,
                                                               int n_fused_slots,
                                                               const FusedMember *__restrict__ fused,
                                                               const double *__restrict__ params, int n_params,
                                                               int batch, long long mstride, float2 *__restrict__ out,
                                                               int fused_per_thread) {
  __shared__ double emb[kMatWarps][kMaxFusedMembers][32];
  __shared__ double acc[kMatWarps][2][32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long gw = (long long)blockIdx.x * kMatWarps + w;  // global warp
  if (fused_per_thread) {
    // many fused blocks (large batches): one thread each, every lane busy in FP64
    const long long n_ft = (long long)n_fused_slots * batch;
    const long long n_fwt = (n_ft + 31) / 32;                    // warps of the fused blocks
    if (gw < n_fwt) {
      const long long t = gw * 32 + lane;
      if (t >= n_ft) return;
      const int b = (int)(t / n_fused_slots);
      const MatSlot &s = slots[t % n_fused_slots];
      const double *prow = params ? params + (long long)b * n_params : nullptr;
      double M[32];
      for (int i = 0; i < 32; ++i) M[i] = (i & 1) == 0 && ((i >> 1) % 5) == 0 ? 1.0 : 0.0;
      for (int m = 0; m < s.fuse_count; ++m) fused_apply_member(fused[s.fuse_begin + m], prow, M);
      float2 *dst = out + (long long)b * mstride + s.offset;
      for (int k = 0; k < 16; ++k) {
        const float re = (float)M[2 * k], im = (float)M[2 * k + 1];
        dst[2 * k] = make_float2(re, re);
        dst[2 * k + 1] = make_float2(-im, im);
      }
      return;
    }
    const int n_reg = n_slots - n_fused_slots;
    const long long t = (gw - n_fwt) * 32 + lane;
    if (t >= (long long)n_reg * batch) return;
    const int b = (int)(t / n_reg);
    materialize_one(slots[n_fused_slots + t % n_reg], params ? params + (long long)b * n_params : nullptr,
                    out + (long long)b * mstride);
    return;
  }
  const long long n_fw = (long long)n_fused_slots * batch;      // warps of the fused blocks
  if (gw < n_fw) {
    const int b = (int)(gw / n_fused_slots);
    const MatSlot &s = slots[gw % n_fused_slots];
    float2 *dst = out + (long long)b * mstride + s.offset;
    const double *prow = params ? params + (long long)b * n_params : nullptr;
    const int cnt = s.fuse_count;
    if (lane < cnt) fused_embed(fused[s.fuse_begin + lane], prow, emb[w][lane]);
    acc[w][0][lane] = (lane & 1) == 0 && ((lane >> 1) % 5) == 0 ? 1.0 : 0.0;  // identity
    __syncwarp();
    int cur = 0;
    for (int m = 0; m < cnt; ++m) {  // acc <- emb[m] * acc
      if (lane < 16) {
        const int i = lane >> 2, j = lane & 3;
        double re = 0.0, im = 0.0;
        for (int q = 0; q < 4; ++q) {
          const double xr = emb[w][m][2 * (4 * i + q)], xi = emb[w][m][2 * (4 * i + q) + 1];
          const double yr = acc[w][cur][2 * (4 * q + j)], yi = acc[w][cur][2 * (4 * q + j) + 1];
          re += xr * yr - xi * yi;
          im += xr * yi + xi * yr;
        }
        acc[w][cur ^ 1][2 * lane] = re;
        acc[w][cur ^ 1][2 * lane + 1] = im;
      }
      __syncwarp();
      cur ^= 1;
    }
    if (lane < 16) {  // packed entry (re, re, -im, im)
      const float re = (float)acc[w][cur][2 * lane], im = (float)acc[w][cur][2 * lane + 1];
      dst[2 * lane] = make_float2(re, re);
      dst[2 * lane + 1] = make_float2(-im, im);
    }
    return;
  }
  const int n_reg = n_slots - n_fused_slots;
  if (n_reg == 0) return;
  const long long t = (gw - n_fw) * 32 + lane;
  if (t >= (long long)n_reg * batch) return;
  const int b = (int)(t / n_reg);
  materialize_one(slots[n_fused_slots + t % n_reg], params ? params + (long long)b * n_params : nullptr,
                  out + (long long)b * mstride);
}

cudaError_t launch_materialize(const MatSlot *d_slots, int n_slots, int n_fused_slots, const FusedMember *d_fused,
                               const double *params, int n_params, int batch, long long mstride, float2 *out,
                               cudaStream_t s) {
  const long long nf = (long long)n_fused_slots * batch, nr = (long long)(n_slots - n_fused_slots) * batch;
  const int per_thread = nf >= kFusedPerThread ? 1 : 0;
  const long long warps = (per_thread ? (nf + 31) / 32 : nf) + (nr + 31) / 32;
  if (warps == 0) return cudaSuccess;
  k_materialize<<<(unsigned)((warps + kMatWarps - 1) / kMatWarps), 32 * kMatWarps, 0, s>>>(
      d_slots, n_slots, n_fused_slots, d_fused, params, n_params, batch, mstride, out, per_thread);
  return cudaGetLastError();
}

// Slot order the materialisation kernel expects: the fused blocks first.
int order_slots_fused_first(std::vector<MatSlot> &slots) {
  std::stable_partition(slots.begin(), slots.end(), [](const MatSlot &m) { return m.kind == KIND_F2; });
  int n = 0;
  for (const MatSlot &m : slots) n += m.kind == KIND_F2 ? 1 : 0;
  return n;
}

// Closing the output legs with <x| (Sec. 2.2.3) on a contracted state is a gather.
__global__ void k_gather(const float2 *__restrict__ state, int N, int batch, const uint64_t *__restrict__ xs,
                         long long nx, float2 *__restrict__ amps) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx * batch) return;
  const long long b = i / nx, k = i % nx;
  amps[i] = state[((long long)b << N) + (long long)xs[k]];
}

cudaError_t launch_gather(const float2 *state, int N, int batch, const uint64_t *xs, long long nx, float2 *amps,
                          cudaStream_t s) {
  const long long total = nx * batch;
  if (total == 0) return cudaSuccess;
  k_gather<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(state, N, batch, xs, nx, amps);
  return cudaGetLastError();
}

__global__ void k_scale_grad(double *grad, const double *gout, int batch, int P) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)batch * P) return;
  grad[i] *= gout[i / P];
}

cudaError_t launch_scale_grad(double *grad, const double *gout, int batch, int P, cudaStream_t s) {
  if (gout == nullptr || (long long)batch * P == 0) return cudaSuccess;
  const long long total = (long long)batch * P;
  k_scale_grad<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(grad, gout, batch, P);
  return cudaGetLastError();
}

cudaError_t launch_zero(void *p, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return cudaSuccess;
  return cudaMemsetAsync(p, 0, bytes, s);
}

// ---------------------------------------------------------------------------------------
// Device status word: kernels with bounded waits or finiteness checks record the first
// failure here (atomicCAS from 0); tn_sync_status reads and clears it.
// ---------------------------------------------------------------------------------------
__device__ int g_tn_status = 0;

void *status_word_ptr() {
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_tn_status) != cudaSuccess) return nullptr;
  return p;
}

cudaError_t read_and_clear_status(int *value, cudaStream_t s) {
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  int v = 0;
  e = cudaMemcpyFromSymbol(&v, g_tn_status, sizeof(int));
  if (e != cudaSuccess) return e;
  if (v != 0) {
    const int zero = 0;
    e = cudaMemcpyToSymbol(g_tn_status, &zero, sizeof(int));
    if (e != cudaSuccess) return e;
  }
  *value = v;
  return cudaSuccess;
}

}  // namespace tnq
