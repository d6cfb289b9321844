// Kernel (c), plain FP32 form: batched complex GEMM on the CUDA cores.
//
// A pairwise merge of two tensors, once their legs are grouped into row, contracted and
// column indices, is the matrix product of Eq. 2.2: C[m][n] = sum_k A[m][k] B[n][k]
// (both operands stored with the contracted index contiguous).  This kernel is the FP32
// reference the tensor-core forms are measured against, and the form used for merges too
// narrow for the tensor-core tiles.  One template covers the shapes a network contraction
// produces: a CTA of 256 threads computes a BM x BN tile in TM x TN complex blocks per
// thread, streaming BK-deep slices of both operands through shared memory (two slices in
// flight, copied asynchronously; rows padded so a warp's reads fall in distinct banks), with
// FFMA accumulation.
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

__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__(kThreads, 2) k_cgemm_fp32(long long M, long long N, long long K, long long k_len,
                                                         const float2 *__restrict__ A, const float2 *__restrict__ B,
                                                         float2 *__restrict__ C, float2 *__restrict__ P,
                                                         const __grid_constant__ StagedMap om) {
  static_assert((BM / TM) * (BN / TN) == kThreads, "one thread per TM x TN block");
  pdl_wait();
  pdl_trigger();
  // two K slices of both operands in flight (row-major, row stride BK + 1: a warp's reads across
  // rows fall in distinct banks); the C tile (row stride BN + 1) in the permuted epilogue
  constexpr int kLd = BK + 1;
  constexpr int kSlice = (BM + BN) * kLd, kTile = BM * (BN + 1);
  __shared__ float2 smem[2 * kSlice > kTile ? 2 * kSlice : kTile];
  // tiles of one batch element along x, n fastest (M may need more than 65535 row tiles)
  const long long tiles_n = (N + BN - 1) / BN;
  const long long b = blockIdx.z;
  const long long m0 = ((long long)blockIdx.x / tiles_n) * BM, n0 = ((long long)blockIdx.x % tiles_n) * BN;
  const float2 *Ab = A + b * M * K;
  const float2 *Bb = B + b * N * K;
  float2 *Cb = C + b * M * N;
  // split K (P != nullptr): this CTA sums k in [kb, ke) and stores its partial tile to P
  const long long kb = (long long)blockIdx.y * k_len, ke = kb + k_len < K ? kb + k_len : K;
  constexpr int NX = BN / TN;  // threads along n
  const int tx = threadIdx.x % NX, ty = threadIdx.x / NX;
  float2 acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = make_float2(0.f, 0.f);
  // slice k0 of A (BM rows) and B (BN rows) into buffer sb: asynchronous copies of the
  // elements in range, zeros for the ragged edges
  auto load_slice = [&](int sb, long long k0) {
    float2 *as = smem + sb * kSlice, *bs = as + BM * kLd;
    for (int e = threadIdx.x; e < (BM + BN) * BK; e += kThreads) {
      const int r = e / BK, c = e % BK;
      const long long gk = k0 + c;
      if (r < BM) {
        const long long gm = m0 + r;
        if (gm < M && gk < ke) cp_async8(as + r * kLd + c, Ab + gm * K + gk);
        else as[r * kLd + c] = make_float2(0.f, 0.f);
      } else {
        const long long gn = n0 + (r - BM);
        if (gn < N && gk < ke) cp_async8(bs + (r - BM) * kLd + c, Bb + gn * K + gk);
        else bs[(r - BM) * kLd + c] = make_float2(0.f, 0.f);
      }
    }
    cp_async_commit();
  };
  int sb = 0;
  if (ke > kb) load_slice(0, kb);
  for (long long k0 = kb; k0 < ke; k0 += BK) {
    if (k0 + BK < ke) {
      load_slice(sb ^ 1, k0 + BK);
      cp_async_wait<1>();  // the current slice has landed (the next may still be in flight)
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float2 *as = smem + sb * kSlice, *bs = as + BM * kLd;
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float2 a[TM], bb[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = as[(ty + (BM / TM) * i) * kLd + kk];
#pragma unroll
      for (int j = 0; j < TN; ++j) bb[j] = bs[(tx + NX * j) * kLd + kk];
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
    __syncthreads();  // the buffer is free for the slice after next
    sb ^= 1;
  }
  if (P != nullptr || om.map.identity) {
    float2 *Ob = P != nullptr ? P + ((long long)blockIdx.y * gridDim.z + b) * M * N : Cb;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const long long gm = m0 + ty + (BM / TM) * i, gn = n0 + tx + NX * j;
        if (gm < M && gn < N) Ob[gm * N + gn] = acc[i][j];
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

// Small merges (at most 2^18 complex multiply-adds, K <= 64; most merges of small circuits):
// one thread per output element reads its K-contiguous rows of A and B straight from global
// memory (cache-resident at this size) and stores through the output map, without tile
// staging.  The accumulation over k is the tiled kernel's (same order, same fused
// multiply-adds), so both give the same bits.
__global__ void __launch_bounds__(256) k_cgemm_small(long long M, long long N, long long K, long long total,
                                                     const float2 *__restrict__ A, const float2 *__restrict__ B,
                                                     float2 *__restrict__ C, const __grid_constant__ OutMap om) {
  pdl_wait();
  pdl_trigger();
  for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < total;
       f += (long long)gridDim.x * blockDim.x) {
    const long long n = f % N, bm = f / N;  // bm = b M + m
    const long long b = bm / M;
    const float2 *a = A + bm * K;
    const float2 *w = B + (b * N + n) * K;
    float2 acc = make_float2(0.f, 0.f);
    for (long long k = 0; k < K; ++k) {
      const float2 x = a[k], y = w[k];
      acc.x = fmaf(x.x, y.x, acc.x);
      acc.x = fmaf(-x.y, y.y, acc.x);
      acc.y = fmaf(x.x, y.y, acc.y);
      acc.y = fmaf(x.y, y.x, acc.y);
    }
    C[om.identity ? f : map_bits(om, f, 0)] = acc;
  }
}
constexpr long long kSmallWork = 1ll << 18;

// Sum of the split-K partials (in split order) of every output element, stored through the
// output map: C[map(f)] = sum_s P[s][f], f the natural index (b M + m) N + n.
__global__ void k_splitk_reduce(const float2 *__restrict__ P, int splits, long long total, float2 *__restrict__ C,
                                const __grid_constant__ OutMap om) {
  pdl_wait();
  pdl_trigger();
  for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < total;
       f += (long long)gridDim.x * blockDim.x) {
    float2 acc = P[f];
    for (int s = 1; s < splits; ++s) {
      const float2 v = P[(long long)s * total + f];
      acc.x += v.x;
      acc.y += v.y;
    }
    C[om.identity ? f : map_bits(om, f, 0)] = acc;
  }
}

// The same sum for few outputs: one block of 128 threads per output element strides over the
// splits, then a fixed tree (warp shuffles, then the four warp sums in order).
__global__ void k_splitk_reduce_few(const float2 *__restrict__ P, int splits, long long total, float2 *__restrict__ C,
                                    const __grid_constant__ OutMap om) {
  pdl_wait();
  pdl_trigger();
  const long long f = blockIdx.x;
  float2 acc = make_float2(0.f, 0.f);
  for (int s = threadIdx.x; s < splits; s += blockDim.x) {
    const float2 v = P[(long long)s * total + f];
    acc.x += v.x;
    acc.y += v.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
  }
  __shared__ float2 warp_sum[4];
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float2 r = warp_sum[0];
    for (int w = 1; w < 4; ++w) {
      r.x += warp_sum[w].x;
      r.y += warp_sum[w].y;
    }
    C[om.identity ? f : map_bits(om, f, 0)] = r;
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

// Tile shape (BM x BN) for an output of N columns.
inline void tile_for(long long N, int *bm, int *bn) {
  *bn = N <= 8 ? 8 : N <= 16 ? 16 : N <= 32 ? 32 : 64;
  *bm = *bn == 64 ? 64 : 128;
}

// Split K: an output of few tiles with a long K (a merge that contracts most of two large
// operands into a small result) would leave most SMs idle and one CTA looping over K; K is
// then cut into ranges of at least 256 (a multiple of the K slice) so that about two CTAs
// per SM (152 SMs) run, each storing a partial tile, and k_splitk_reduce adds the partials.
constexpr long long kSplitTargetCtas = 2 * 152;
int split_k(long long batch, long long M, long long N, long long K, long long *k_len) {
  int bm = 0, bn = 0;
  tile_for(N, &bm, &bn);
  const long long tiles = batch * ((M + bm - 1) / bm) * ((N + bn - 1) / bn);
  *k_len = K;
  if (K < 512 || tiles >= kSplitTargetCtas) return 1;
  long long S = std::min<long long>((kSplitTargetCtas + tiles - 1) / tiles, K / 256);
  if (S <= 1) return 1;
  const int bk = K <= 8 ? 8 : 16;
  long long kl = (K + S - 1) / S;
  kl = (kl + bk - 1) / bk * bk;
  *k_len = kl;
  return (int)((K + kl - 1) / kl);
}

template <int BM, int BN, int BK, int TM, int TN>
cudaError_t launch_shape(long long batch, long long M, long long N, long long K, const float2 *A, const float2 *B,
                         float2 *C, float2 *P, const OutMap &om, cudaStream_t s) {
  const long long tiles = ((N + BN - 1) / BN) * ((M + BM - 1) / BM);
  if (tiles > 0x7fffffffll) return cudaErrorNotSupported;
  long long k_len = K;
  const int splits = P != nullptr ? split_k(batch, M, N, K, &k_len) : 1;
  dim3 grid((unsigned)tiles, (unsigned)splits, (unsigned)batch);
  StagedMap sm;
  std::memset(&sm, 0, sizeof(sm));
  sm.map = om;
  if (!om.identity && splits == 1) build_staged(sm, om, M, N, BM, BN);
  cudaError_t e = launch_pdl(k_cgemm_fp32<BM, BN, BK, TM, TN>, grid, dim3(kThreads), 0, s, M, N, K, k_len, A, B, C,
                             splits > 1 ? P : (float2 *)nullptr, sm);
  if (e != cudaSuccess || splits == 1) return e;
  const long long total = batch * M * N;
  if (total <= 4096)
    return launch_pdl(k_splitk_reduce_few, dim3((unsigned)total), dim3(128), 0, s, (const float2 *)P, splits, total, C,
                      om);
  return launch_pdl(k_splitk_reduce, dim3((unsigned)std::min<long long>((total + 255) / 256, 4096)), dim3(256), 0, s,
                    (const float2 *)P, splits, total, C, om);
}

template <int BK>
cudaError_t launch_k(long long batch, long long M, long long N, long long K, const float2 *A, const float2 *B,
                     float2 *C, float2 *P, const OutMap &om, cudaStream_t s) {
  int bm = 0, bn = 0;
  tile_for(N, &bm, &bn);
  if (bn == 8) return launch_shape<128, 8, BK, 2, 2>(batch, M, N, K, A, B, C, P, om, s);
  if (bn == 16) return launch_shape<128, 16, BK, 4, 2>(batch, M, N, K, A, B, C, P, om, s);
  if (bn == 32) return launch_shape<128, 32, BK, 4, 4>(batch, M, N, K, A, B, C, P, om, s);
  return launch_shape<64, 64, BK, 4, 4>(batch, M, N, K, A, B, C, P, om, s);
}

}  // namespace

size_t cgemm_fp32_workspace(long long batch, long long M, long long N, long long K) {
  long long k_len = 0;
  const int splits = split_k(batch, M, N, K, &k_len);
  return splits > 1 ? (size_t)splits * (size_t)(batch * M * N) * sizeof(float2) : 0;
}

double cgemm_fp32_tile_fill(long long M, long long N) {
  int bm = 0, bn = 0;
  tile_for(N, &bm, &bn);
  const double rows = (double)M / (double)(((M + bm - 1) / bm) * bm);
  const double cols = (double)N / (double)(((N + bn - 1) / bn) * bn);
  return rows * cols;
}

cudaError_t launch_cgemm_fp32(long long batch, long long M, long long N, long long K, const float2 *A, const float2 *B,
                              float2 *C, void *ws, size_t ws_bytes, cudaStream_t s, const OutMap *om) {
  if (batch > 65535) return cudaErrorNotSupported;
  const size_t need = cgemm_fp32_workspace(batch, M, N, K);
  if (need > 0 && (ws == nullptr || ws_bytes < need)) return cudaErrorInvalidValue;
  float2 *P = need > 0 ? static_cast<float2 *>(ws) : nullptr;
  const OutMap ident;
  const OutMap &m = om ? *om : ident;
  const long long total = batch * M * N;
  // small merges, and tall narrow ones (at most four output columns, where the tiled kernel's
  // 8-column tiles would mostly compute padding) of any size: one thread per output element
  // (on the Fig. 3.1 amplitude sweep: up to 2 columns 12.1 ms per step, up to 4 12.0, up to 8
  // 13.1, none 22.4)
  if (K <= 64 && ((double)total * (double)K <= (double)kSmallWork || N <= 4)) {
    const long long blocks = std::min<long long>((total + 255) / 256, (long long)num_sms() * 16);
    return launch_pdl(k_cgemm_small, dim3((unsigned)blocks), dim3(256), 0, s, M, N, K, total, A, B, C, m);
  }
  if (K <= 8) return launch_k<8>(batch, M, N, K, A, B, C, P, m, s);
  return launch_k<16>(batch, M, N, K, A, B, C, P, m, s);
}

}  // namespace tnq
