// Small kernels of libtnq: per-call gate-matrix tables, amplitude gather, gradient
// scaling, device status word.
#include "apply_common.cuh"
#include "kernels.h"

namespace tnq {

// Gate tensors are built once per call from the parameters (one thread per slot and
// batch element; angles in FP64, entries stored as complex64).  A fused block (KIND_F2) is the
// FP64 product of its member gates, stored in the packed layout (SHAPE_M4X).
__global__ void k_materialize(const MatSlot *__restrict__ slots, int n_slots, const FusedMember *__restrict__ fused,
                              const double *__restrict__ params, int n_params, int batch, long long mstride,
                              float2 *__restrict__ out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n_slots * batch) return;
  const int b = (int)(idx / n_slots);
  const int k = (int)(idx % n_slots);
  const MatSlot &s = slots[k];
  float2 *dst = out + (long long)b * mstride + s.offset;
  if (s.kind == KIND_F2) {
    double m[32];
    float ent[64];
    fused_matrix(fused + s.fuse_begin, s.fuse_count, params ? params + (long long)b * n_params : nullptr, m);
    packed_m4x(m, ent);
    for (int i = 0; i < 32; ++i) dst[i] = make_float2(ent[2 * i], ent[2 * i + 1]);
    return;
  }
  double ang[3] = {s.angle[0], s.angle[1], s.angle[2]};
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < 2; ++k)
      if (s.pidx[a][k] >= 0) ang[a] += params[(long long)b * n_params + s.pidx[a][k]];
  double tmp[32];
  float ent[32];
  const int n = slot_entries(s, ang, tmp, ent);
  for (int i = 0; i < n; ++i) dst[i] = make_float2(ent[2 * i], ent[2 * i + 1]);
}

cudaError_t launch_materialize(const MatSlot *d_slots, int n_slots, const FusedMember *d_fused, const double *params,
                               int n_params, int batch, long long mstride, float2 *out, cudaStream_t s) {
  const long long total = (long long)n_slots * batch;
  if (total == 0) return cudaSuccess;
  const int threads = 128;
  k_materialize<<<(unsigned)((total + threads - 1) / threads), threads, 0, s>>>(d_slots, n_slots, d_fused, params,
                                                                               n_params, batch, mstride, out);
  return cudaGetLastError();
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
