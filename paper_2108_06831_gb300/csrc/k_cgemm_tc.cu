// Kernel (c), tensor-core forms: batched complex GEMM on tcgen05 with TMEM accumulators.
#include "kernels.h"

namespace tnq {

cudaError_t launch_cgemm_fp32(long long batch, long long M, long long N, long long K, const float2 *A, const float2 *B,
                              float2 *C, cudaStream_t s);

size_t cgemm_workspace(int precision, long long batch, long long M, long long N, long long K) {
  (void)precision; (void)batch; (void)M; (void)N; (void)K;
  return 0;
}

cudaError_t launch_cgemm(int precision, long long batch, long long M, long long N, long long K, const float2 *A,
                         const float2 *B, float2 *C, void *ws, size_t ws_bytes, cudaStream_t s) {
  (void)ws; (void)ws_bytes;
  if (precision == TN_PREC_FP32) return launch_cgemm_fp32(batch, M, N, K, A, B, C, s);
  return cudaErrorNotSupported;
}

}  // namespace tnq
