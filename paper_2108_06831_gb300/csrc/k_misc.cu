// Small kernels of libtnq: per-call gate-matrix tables, amplitude gather, gradient
// scaling, device status word.
#include <algorithm>
#include <vector>

#include "apply_common.cuh"
#include "kernels.h"

namespace tnq {

// Gate tensors are built once per call from the parameters (angles in FP64, entries stored as
// complex64).  The slot array lists the fused blocks (KIND_F2) first: each fused block and batch
// element takes one warp -- lane m evaluates member m's matrix embedded as a 4x4, then lanes
// 0..15 form the product one entry each, member by member, and store it in the packed layout
// (SHAPE_M4X); every other slot and batch element takes one thread (one gate's matrix).
constexpr int kMatWarps = 4;

__global__ void __launch_bounds__(32 * kMatWarps) k_materialize(const MatSlot *__restrict__ slots, int n_slots,
                                                               int n_fused_slots,
                                                               const FusedMember *__restrict__ fused,
                                                               const double *__restrict__ params, int n_params,
                                                               int batch, long long mstride, float2 *__restrict__ out) {
  __shared__ double emb[kMatWarps][kMaxFusedMembers][32];
  __shared__ double acc[kMatWarps][2][32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long gw = (long long)blockIdx.x * kMatWarps + w;  // global warp
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
  const MatSlot &s = slots[n_fused_slots + t % n_reg];
  float2 *dst = out + (long long)b * mstride + s.offset;
  double ang[3] = {s.angle[0], s.angle[1], s.angle[2]};
  for (int a = 0; a < 3; ++a)
    for (int q = 0; q < 2; ++q)
      if (s.pidx[a][q] >= 0) ang[a] += params[(long long)b * n_params + s.pidx[a][q]];
  double tmp[32];
  float ent[32];
  const int n = slot_entries(s, ang, tmp, ent);
  for (int i = 0; i < n; ++i) dst[i] = make_float2(ent[2 * i], ent[2 * i + 1]);
}

cudaError_t launch_materialize(const MatSlot *d_slots, int n_slots, int n_fused_slots, const FusedMember *d_fused,
                               const double *params, int n_params, int batch, long long mstride, float2 *out,
                               cudaStream_t s) {
  const long long warps = (long long)n_fused_slots * batch + ((long long)(n_slots - n_fused_slots) * batch + 31) / 32;
  if (warps == 0) return cudaSuccess;
  k_materialize<<<(unsigned)((warps + kMatWarps - 1) / kMatWarps), 32 * kMatWarps, 0, s>>>(
      d_slots, n_slots, n_fused_slots, d_fused, params, n_params, batch, mstride, out);
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
