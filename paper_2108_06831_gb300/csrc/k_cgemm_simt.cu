// Kernel (c), plain FP32 form: batched complex GEMM on the CUDA cores.
//
// A pairwise merge of two tensors, once their legs are grouped into row, contracted and
// column indices, is the matrix product of Eq. 2.2: C[m][n] = sum_k A[m][k] B[n][k]
// (both operands stored with the contracted index contiguous).  This kernel is the FP32
// reference the tensor-core forms are measured against, and the form used for merges too
// narrow for the tensor-core tiles.  One template covers the shapes a network contraction
// produces: a CTA of 256 threads computes a BM x BN tile in TM x TN complex blocks per
// thread, streaming BK-deep slices of both operands through shared memory (stored
// transposed, so a warp's reads along rows are conflict-free), with FFMA accumulation.
// The tile is fitted to the operand shape: narrow N (down to 8 columns) takes tall tiles so
// that no column work is wasted, and short K (8) takes an 8-deep slice.
#include "kernels.h"

namespace tnq {

namespace {

constexpr int kThreads = 256;

template <int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__(kThreads, 2) k_cgemm_fp32(long long M, long long N, long long K,
                                                         const float2 *__restrict__ A, const float2 *__restrict__ B,
                                                         float2 *__restrict__ C) {
  static_assert((BM / TM) * (BN / TN) == kThreads, "one thread per TM x TN block");
  __shared__ float2 As[BK][BM + 1];
  __shared__ float2 Bs[BK][BN + 1];
  const long long b = blockIdx.z;
  const long long m0 = (long long)blockIdx.y * BM, n0 = (long long)blockIdx.x * BN;
  const float2 *Ab = A + b * M * K;
  const float2 *Bb = B + b * N * K;
  float2 *Cb = C + b * M * N;
  constexpr int NX = BN / TN;  // threads along n
  const int tx = threadIdx.x % NX, ty = threadIdx.x / NX;
  float2 acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = make_float2(0.f, 0.f);
  // K-contiguous operands: pairs of complex numbers (16 bytes) per load when K is even
  const bool vec = (K % 2) == 0;
  for (long long k0 = 0; k0 < K; k0 += BK) {
    if (vec) {
      for (int e = threadIdx.x; e < BM * (BK / 2); e += kThreads) {
        const int r = e / (BK / 2), c = 2 * (e % (BK / 2));
        const long long gm = m0 + r, gk = k0 + c;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gm < M && gk < K) v = *reinterpret_cast<const float4 *>(Ab + gm * K + gk);
        As[c][r] = make_float2(v.x, v.y);
        As[c + 1][r] = make_float2(v.z, v.w);
      }
      for (int e = threadIdx.x; e < BN * (BK / 2); e += kThreads) {
        const int r = e / (BK / 2), c = 2 * (e % (BK / 2));
        const long long gn = n0 + r, gk = k0 + c;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gn < N && gk < K) v = *reinterpret_cast<const float4 *>(Bb + gn * K + gk);
        Bs[c][r] = make_float2(v.x, v.y);
        Bs[c + 1][r] = make_float2(v.z, v.w);
      }
    } else {
      for (int e = threadIdx.x; e < BM * BK; e += kThreads) {
        const int r = e / BK, c = e % BK;
        const long long gm = m0 + r, gk = k0 + c;
        As[c][r] = (gm < M && gk < K) ? Ab[gm * K + gk] : make_float2(0.f, 0.f);
      }
      for (int e = threadIdx.x; e < BN * BK; e += kThreads) {
        const int r = e / BK, c = e % BK;
        const long long gn = n0 + r, gk = k0 + c;
        Bs[c][r] = (gn < N && gk < K) ? Bb[gn * K + gk] : make_float2(0.f, 0.f);
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float2 a[TM], bb[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + (BM / TM) * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) bb[j] = Bs[kk][tx + NX * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          acc[i][j].x = fmaf(a[i].x, bb[j].x, acc[i][j].x);
          acc[i][j].x = fmaf(-a[i].y, bb[j].y, acc[i][j].x);
          acc[i][j].y = fmaf(a[i].x, bb[j].y, acc[i][j].y);
          acc[i][j].y = fmaf(a[i].y, bb[j].x, acc[i][j].y);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const long long gm = m0 + ty + (BM / TM) * i, gn = n0 + tx + NX * j;
      if (gm < M && gn < N) Cb[gm * N + gn] = acc[i][j];
    }
}

template <int BM, int BN, int BK, int TM, int TN>
cudaError_t launch_shape(long long batch, long long M, long long N, long long K, const float2 *A, const float2 *B,
                         float2 *C, cudaStream_t s) {
  dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM), (unsigned)batch);
  if ((N + BN - 1) / BN > 0x7fffffffll || grid.y > 65535) return cudaErrorNotSupported;
  k_cgemm_fp32<BM, BN, BK, TM, TN><<<grid, kThreads, 0, s>>>(M, N, K, A, B, C);
  return cudaGetLastError();
}

template <int BK>
cudaError_t launch_k(long long batch, long long M, long long N, long long K, const float2 *A, const float2 *B,
                     float2 *C, cudaStream_t s) {
  if (N <= 8) return launch_shape<256, 8, BK, 4, 2>(batch, M, N, K, A, B, C, s);
  if (N <= 16) return launch_shape<128, 16, BK, 4, 2>(batch, M, N, K, A, B, C, s);
  if (N <= 32) return launch_shape<128, 32, BK, 4, 4>(batch, M, N, K, A, B, C, s);
  return launch_shape<64, 64, BK, 4, 4>(batch, M, N, K, A, B, C, s);
}

}  // namespace

cudaError_t launch_cgemm_fp32(long long batch, long long M, long long N, long long K, const float2 *A, const float2 *B,
                              float2 *C, cudaStream_t s) {
  if (batch > 65535) return cudaErrorNotSupported;
  if (K <= 8) return launch_k<8>(batch, M, N, K, A, B, C, s);
  return launch_k<16>(batch, M, N, K, A, B, C, s);
}

}  // namespace tnq
