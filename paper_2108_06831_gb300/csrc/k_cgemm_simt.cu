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
#include <algorithm>
#include <cstring>
#include <vector>

#include "kernels.h"

namespace tnq {

namespace {

constexpr int kThreads = 256;

// An output map with the tables of its permuted epilogue for one tile shape.
struct StagedMap {
  OutMap map;
  int lgn, L, nlo, pairs;
  int s_lo[64], s_hi[64];       // staging offsets (complex)
  long long g_lo[64], g_hi[64];  // stored offsets (complex)
};
void build_staged(StagedMap &sm, const OutMap &om, long long M, long long N, int BM, int BN);

// Output index of natural flat index bits [lo, nbits) of f under the map (0 for identity).
__device__ __forceinline__ long long map_bits(const OutMap &om, long long f, int lo) {
  long long r = 0;
  for (int i = lo; i < om.nbits; ++i)
    if ((f >> i) & 1) r |= 1ll << om.pos[i];
  return r;
}

template <int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__(kThreads, 2) k_cgemm_fp32(long long M, long long N, long long K,
                                                         const float2 *__restrict__ A, const float2 *__restrict__ B,
                                                         float2 *__restrict__ C, const __grid_constant__ StagedMap om) {
  static_assert((BM / TM) * (BN / TN) == kThreads, "one thread per TM x TN block");
  // operand slices during the K loop; the C tile (row stride BN + 1) in the permuted epilogue
  constexpr int kAB = BK * (BM + 1) + BK * (BN + 1), kTile = BM * (BN + 1);
  __shared__ float2 smem[kAB > kTile ? kAB : kTile];
  float2(*As)[BM + 1] = reinterpret_cast<float2(*)[BM + 1]>(smem);
  float2(*Bs)[BN + 1] = reinterpret_cast<float2(*)[BN + 1]>(smem + BK * (BM + 1));
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
  if (om.map.identity) {
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const long long gm = m0 + ty + (BM / TM) * i, gn = n0 + tx + NX * j;
        if (gm < M && gn < N) Cb[gm * N + gn] = acc[i][j];
      }
  } else {
    // Permuted output: the tile is staged in shared memory and written back in stored-index
    // order, u -> (staging offset, stored offset) from the host-built tables (copied to shared
    // memory: lanes index them divergently).
    __shared__ int s_lo[64], s_hi[64];
    __shared__ long long g_lo[64], g_hi[64];
    if (threadIdx.x < 64) {
      s_lo[threadIdx.x] = om.s_lo[threadIdx.x];
      g_lo[threadIdx.x] = om.g_lo[threadIdx.x];
    } else if (threadIdx.x < 128) {
      s_hi[threadIdx.x - 64] = om.s_hi[threadIdx.x - 64];
      g_hi[threadIdx.x - 64] = om.g_hi[threadIdx.x - 64];
    }
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) smem[(ty + (BM / TM) * i) * (BN + 1) + tx + NX * j] = acc[i][j];
    __syncthreads();
    const long long gbase = map_bits(om.map, ((b * M + m0) << om.lgn) | n0, 0);
    const int L = om.L, nlo = om.nlo, lo_mask = (1 << om.nlo) - 1;
    if (L == 0) {
      if (threadIdx.x == 0) C[gbase] = smem[0];
    } else if (om.pairs) {  // u, u + 1 adjacent in memory: 16-byte stores
      for (int u = 2 * threadIdx.x; u < (1 << L); u += 2 * kThreads) {
        const float2 x0 = smem[s_lo[u & lo_mask] + s_hi[u >> nlo]];
        const float2 x1 = smem[s_lo[(u + 1) & lo_mask] + s_hi[(u + 1) >> nlo]];
        *reinterpret_cast<float4 *>(C + gbase + g_lo[u & lo_mask] + g_hi[u >> nlo]) =
            make_float4(x0.x, x0.y, x1.x, x1.y);
      }
    } else {
      for (int u = threadIdx.x; u < (1 << L); u += kThreads)
        C[gbase + g_lo[u & lo_mask] + g_hi[u >> nlo]] = smem[s_lo[u & lo_mask] + s_hi[u >> nlo]];
    }
  }
}

// Tables of the permuted epilogue for one tile shape (built on the host once per launch).
// The tile's valid local bits (vc column bits, then vr row bits) are enumerated by increasing
// stored position; u's low nlo bits and high L - nlo bits index the tables.
void build_staged(StagedMap &sm, const OutMap &om, long long M, long long N, int BM, int BN) {
  sm.map = om;
  int lgn = 0, lgm = 0, lbn = 0, lbm = 0;
  while ((1ll << lgn) < N) ++lgn;
  while ((1ll << lgm) < M) ++lgm;
  while ((1 << lbn) < BN) ++lbn;
  while ((1 << lbm) < BM) ++lbm;
  const int vc = std::min(lbn, lgn), vr = std::min(lbm, lgm), L = vc + vr;
  sm.lgn = lgn;
  sm.L = L;
  sm.nlo = std::min(L, 6);
  std::vector<int> order((size_t)L);
  for (int k = 0; k < L; ++k) order[(size_t)k] = k;
  auto spos = [&](int k) { return (int)(k < vc ? om.pos[k] : om.pos[lgn + k - vc]); };
  auto sm_of = [&](int k) { return k < vc ? (1 << k) : ((BN + 1) << (k - vc)); };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return spos(a) < spos(b); });
  for (int half = 0; half < 2; ++half) {
    const int nb = half ? L - sm.nlo : sm.nlo, k0 = half ? sm.nlo : 0;
    for (int u = 0; u < (1 << nb); ++u) {
      int so = 0;
      long long go = 0;
      for (int k = 0; k < nb; ++k)
        if ((u >> k) & 1) {
          so += sm_of(order[(size_t)(k0 + k)]);
          go += 1ll << spos(order[(size_t)(k0 + k)]);
        }
      (half ? sm.s_hi : sm.s_lo)[u] = so;
      (half ? sm.g_hi : sm.g_lo)[u] = go;
    }
  }
  sm.pairs = L > 0 && spos(order[0]) == 0;
}

template <int BM, int BN, int BK, int TM, int TN>
cudaError_t launch_shape(long long batch, long long M, long long N, long long K, const float2 *A, const float2 *B,
                         float2 *C, const OutMap &om, cudaStream_t s) {
  dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM), (unsigned)batch);
  if ((N + BN - 1) / BN > 0x7fffffffll || grid.y > 65535) return cudaErrorNotSupported;
  StagedMap sm;
  std::memset(&sm, 0, sizeof(sm));
  sm.map = om;
  if (!om.identity) build_staged(sm, om, M, N, BM, BN);
  k_cgemm_fp32<BM, BN, BK, TM, TN><<<grid, kThreads, 0, s>>>(M, N, K, A, B, C, sm);
  return cudaGetLastError();
}

template <int BK>
cudaError_t launch_k(long long batch, long long M, long long N, long long K, const float2 *A, const float2 *B,
                     float2 *C, const OutMap &om, cudaStream_t s) {
  if (N <= 8) return launch_shape<256, 8, BK, 4, 2>(batch, M, N, K, A, B, C, om, s);
  if (N <= 16) return launch_shape<128, 16, BK, 4, 2>(batch, M, N, K, A, B, C, om, s);
  if (N <= 32) return launch_shape<128, 32, BK, 4, 4>(batch, M, N, K, A, B, C, om, s);
  return launch_shape<64, 64, BK, 4, 4>(batch, M, N, K, A, B, C, om, s);
}

}  // namespace

cudaError_t launch_cgemm_fp32(long long batch, long long M, long long N, long long K, const float2 *A, const float2 *B,
                              float2 *C, cudaStream_t s, const OutMap *om) {
  if (batch > 65535) return cudaErrorNotSupported;
  const OutMap ident;
  const OutMap &m = om ? *om : ident;
  if (K <= 8) return launch_k<8>(batch, M, N, K, A, B, C, m, s);
  return launch_k<16>(batch, M, N, K, A, B, C, m, s);
}

}  // namespace tnq
