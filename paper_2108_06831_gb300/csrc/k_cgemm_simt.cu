// Kernel (c), plain FP32 form: batched complex GEMM on the CUDA cores.
//
// A pairwise merge of two tensors, once their legs are grouped into row, contracted and
// column indices, is the matrix product of Eq. 2.2: C[m][n] = sum_k A[m][k] B[n][k]
// (both operands stored with the contracted index contiguous).  This kernel is the FP32
// reference the tensor-core forms are measured against: 64x64 output tiles, 16-deep K
// slices staged in shared memory, 4x4 complex outputs per thread, FFMA accumulation.
#include "kernels.h"

namespace tnq {

namespace {
constexpr int BM = 64, BN = 64, BK = 16;

__global__ void __launch_bounds__(256) k_cgemm_fp32(long long M, long long N, long long K, const float2 *__restrict__ A,
                                                    const float2 *__restrict__ B, float2 *__restrict__ C) {
  __shared__ float2 As[BK][BM + 1];
  __shared__ float2 Bs[BK][BN + 1];
  const long long b = blockIdx.z;
  const long long m0 = (long long)blockIdx.y * BM, n0 = (long long)blockIdx.x * BN;
  const float2 *Ab = A + b * M * K;
  const float2 *Bb = B + b * N * K;
  float2 *Cb = C + b * M * N;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  for (long long k0 = 0; k0 < K; k0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      const int r = e / BK, c = e % BK;
      const long long gm = m0 + r, gk = k0 + c;
      As[c][r] = (gm < M && gk < K) ? Ab[gm * K + gk] : make_float2(0.f, 0.f);
      const long long gn = n0 + r;
      Bs[c][r] = (gn < N && gk < K) ? Bb[gn * K + gk] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float2 a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fmaf(a[i].x, bb[j].x, acc[i][j].x);
          acc[i][j].x = fmaf(-a[i].y, bb[j].y, acc[i][j].x);
          acc[i][j].y = fmaf(a[i].x, bb[j].y, acc[i][j].y);
          acc[i][j].y = fmaf(a[i].y, bb[j].x, acc[i][j].y);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long long gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
      if (gm < M && gn < N) Cb[gm * N + gn] = acc[i][j];
    }
}
}  // namespace

cudaError_t launch_cgemm_fp32(long long batch, long long M, long long N, long long K, const float2 *A, const float2 *B,
                              float2 *C, cudaStream_t s) {
  if (batch > 65535) return cudaErrorNotSupported;
  dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM), (unsigned)batch);
  if (grid.y > 65535) return cudaErrorNotSupported;
  k_cgemm_fp32<<<grid, 256, 0, s>>>(M, N, K, A, B, C);
  return cudaGetLastError();
}

}  // namespace tnq
