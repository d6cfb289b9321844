// Kernel (b): index permutation over binary legs.
//
// Before two tensors are merged as a matrix product their legs are regrouped so that the
// contracted legs are contiguous (Sec. 3 reshapes every operand into matrices before it is
// deployed).  For a tensor of n legs of size 2, out[y] = in[x] where output leg j holds
// input leg perm[j].  The kernel is a generalised transpose and HBM-bound (8 bytes read and
// 8 written per element):
//   - a tile is 2^R rows of 2^lo input-contiguous elements (lo = 5 low input bits); the
//     first e row bits are the "extra" input bits that feed the lo low output bits, the other
//     R - e are "passive" outer bits (lowest input bits first) that only make the tile large
//     enough (up to 64 rows, 16 KB) to keep the copy engine busy whatever the permutation;
//   - each row is fetched by the bulk-copy (TMA) engine straight into shared memory
//     (cp.async.bulk, completion counted on an mbarrier), two tiles in flight per CTA;
//   - every warp then writes whole 2^lo-element output runs with coalesced stores.
// Every mbarrier wait is bounded: on expiry the kernel records TN_ERR_TIMEOUT in the
// device status word and returns.
#include <cstring>

#include "apply_common.cuh"
#include "kernels.h"

namespace tnq {

namespace {

constexpr int kPermThreads = 256;
constexpr int kPermStages = 2;
constexpr unsigned long long kWaitNs = 2000000000ull;  // bound of every mbarrier wait

constexpr int kPermMaxRowBits = 6;  // at most 64 rows of 32 elements per tile

struct PermParams {
  int n, lo, e, r, n_outer;       // r = row bits of a tile (e extra + r - e passive)
  int row_stride;                 // shared-memory row stride (elements, multiple of 2)
  uint8_t extra_in[8];            // input bit of extra (row) bit q
  uint8_t col_from_k[8];          // for output low bit j: input bit o_in[j]
  uint8_t m_in[8];                // input low bits not feeding output low bits (run-index bits)
  uint8_t m_out[8];               // their output bit positions
  uint8_t pas_in[8], pas_out[8];  // passive row bits: input and output bit positions
  uint8_t outer_in[40], outer_out[40];
  int *status;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait (about two seconds of wall time): false, and the status word set, on expiry.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int *status) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = now_ns();
  for (;;) {
    for (int i = 0; i < 256; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (now_ns() - t0 > kWaitNs) break;
  }
  if (status) atomicCAS(status, 0, (int)TN_ERR_TIMEOUT);
  return false;
}

__global__ void __launch_bounds__(kPermThreads) k_permute(PermParams P, long long batch, const float2 *__restrict__ in,
                                                          float2 *__restrict__ out) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[kPermStages];
  __shared__ int lane_off[32];
  __shared__ int m_off[1 << kPermMaxRowBits];
  __shared__ long long m_out_off[1 << kPermMaxRowBits];
  __shared__ long long row_in_off[1 << kPermMaxRowBits];
  __shared__ int abort_flag;
  const int rows = 1 << P.r;
  const int runlen = 1 << P.lo;
  const int stage_elems = rows * P.row_stride;
  float2 *stage = reinterpret_cast<float2 *>(smem_raw);

  if (threadIdx.x < runlen) {
    const int k = threadIdx.x;
    int row = 0, col = 0;
    for (int j = 0; j < P.lo; ++j) {
      const int ib = P.col_from_k[j];
      const int v = (k >> j) & 1;
      if (ib < P.lo) col |= v << ib;
      else
        for (int q = 0; q < P.e; ++q)
          if (P.extra_in[q] == ib) row |= v << q;
    }
    lane_off[k] = row * P.row_stride + col;
  }
  if (threadIdx.x < rows) {
    // row m of the tile: bits [0, e) extra, bits [e, r) passive.  As a write index, the low
    // e bits of m are the run-index bits m_in instead (same count as the extra bits).
    const int m = threadIdx.x;
    int col = 0;
    long long yo = 0, xo = 0;
    for (int q = 0; q < P.e; ++q) {
      const int v = (m >> q) & 1;
      col |= v << P.m_in[q];
      yo |= (long long)v << P.m_out[q];
      xo |= (long long)v << P.extra_in[q];
    }
    for (int q = P.e; q < P.r; ++q) {
      const int v = (m >> q) & 1;
      yo |= (long long)v << P.pas_out[q - P.e];
      xo |= (long long)v << P.pas_in[q - P.e];
    }
    m_off[m] = col + ((m >> P.e) << P.e) * P.row_stride;
    m_out_off[m] = yo;
    row_in_off[m] = xo;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < kPermStages; ++s) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
  }
  __syncthreads();

  const long long n_tiles = 1ll << P.n_outer;
  const long long work = n_tiles * batch;
  const long long elems = 1ll << P.n;
  const uint32_t row_bytes = (uint32_t)runlen * sizeof(float2);

  auto tile_bases = [&](long long w, long long &ib, long long &ob) {
    const long long b = w >> P.n_outer, t = w & (n_tiles - 1);
    ib = b * elems;
    ob = b * elems;
    for (int q = 0; q < P.n_outer; ++q)
      if ((t >> q) & 1) {
        ib += 1ll << P.outer_in[q];
        ob += 1ll << P.outer_out[q];
      }
  };
  auto issue = [&](long long w, int s) {
    long long ib, ob;
    tile_bases(w, ib, ob);
    if (threadIdx.x == 0) mbar_expect_tx(&bars[s], row_bytes * rows);
    __syncwarp();
    for (int r = threadIdx.x; r < rows; r += 32)
      bulk_g2s(stage + s * stage_elems + r * P.row_stride, in + ib + row_in_off[r], row_bytes, &bars[s]);
  };

  long long w0 = blockIdx.x;
  if (threadIdx.x < 32 && w0 < work) issue(w0, 0);
  uint32_t phase[kPermStages] = {0, 0};
  int s = 0;
  for (long long w = w0; w < work; w += gridDim.x) {
    const long long wn = w + gridDim.x;
    if (threadIdx.x < 32 && wn < work) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(wn, s ^ 1);
    }
    if (!mbar_wait_bounded(&bars[s], phase[s], P.status)) abort_flag = 1;
    phase[s] ^= 1;
    long long ib, ob;
    tile_bases(w, ib, ob);
    const float2 *st = stage + s * stage_elems;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int m = warp; m < rows; m += kPermThreads / 32)
      out[ob + m_out_off[m] + lane] = st[lane_off[lane] + m_off[m]];
    __syncthreads();
    if (abort_flag) {
      // let the copy already issued into the other stage land (bounded) before exiting
      if (wn < work) mbar_wait_bounded(&bars[s ^ 1], phase[s ^ 1], nullptr);
      return;
    }
    s ^= 1;
  }
}

// Short runs (lo < 5, tensors with fewer than 5 legs): direct element mapping.
__global__ void k_permute_small(int n, long long batch, const float2 *in, float2 *out, const PermParams P) {
  const long long total = (1ll << n) * batch;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long b = i >> n;
    const long long y = i & ((1ll << n) - 1);
    long long x = 0;
    for (int j = 0; j < n; ++j) x |= ((y >> j) & 1) << P.outer_in[j];
    out[(b << n) + y] = in[(b << n) + x];
  }
}

}  // namespace

cudaError_t launch_permute(int n, const int32_t *perm, long long batch, const float2 *in, float2 *out, cudaStream_t s) {
  // output bit ob = n-1-j holds input bit ib = n-1-perm[j]
  int in_of_out[64], out_of_in[64];
  for (int j = 0; j < n; ++j) {
    const int ob = n - 1 - j, ib = n - 1 - perm[j];
    in_of_out[ob] = ib;
    out_of_in[ib] = ob;
  }
  PermParams P;
  std::memset(&P, 0, sizeof(P));
  P.n = n;
  P.status = static_cast<int *>(status_word_ptr());
  if (n < 5) {
    for (int ob = 0; ob < n; ++ob) P.outer_in[ob] = (uint8_t)in_of_out[ob];
    const long long total = (1ll << n) * batch;
    const int threads = 256;
    long long blocks = (total + threads - 1) / threads;
    if (blocks > 65535) blocks = 65535;
    k_permute_small<<<(unsigned)blocks, threads, 0, s>>>(n, batch, in, out, P);
    return cudaGetLastError();
  }
  const int lo = 5;
  P.lo = lo;
  bool in_S[64] = {false};
  for (int b = 0; b < lo; ++b) in_S[b] = true;
  int e = 0;
  for (int j = 0; j < lo; ++j) {
    const int ib = in_of_out[j];
    P.col_from_k[j] = (uint8_t)ib;
    if (ib >= lo) {
      in_S[ib] = true;
      P.extra_in[e++] = (uint8_t)ib;
    }
  }
  P.e = e;
  P.r = e;
  // input low bits that do not feed an output low bit index the output runs
  int mq = 0;
  for (int b = 0; b < lo; ++b) {
    bool feeds = false;
    for (int j = 0; j < lo; ++j) feeds |= in_of_out[j] == b;
    if (!feeds) {
      P.m_in[mq] = (uint8_t)b;
      P.m_out[mq] = (uint8_t)out_of_in[b];
      ++mq;
    }
  }
  // passive row bits (lowest remaining input bits) fill the tile up to 64 rows; the rest
  // index tiles
  int no = 0;
  for (int b = 0; b < n; ++b)
    if (!in_S[b]) {
      if (P.r < kPermMaxRowBits) {
        P.pas_in[P.r - e] = (uint8_t)b;
        P.pas_out[P.r - e] = (uint8_t)out_of_in[b];
        ++P.r;
        continue;
      }
      P.outer_in[no] = (uint8_t)b;
      P.outer_out[no] = (uint8_t)out_of_in[b];
      ++no;
    }
  P.n_outer = no;
  P.row_stride = (1 << lo) + 2;
  const size_t smem = (size_t)kPermStages * (1 << P.r) * P.row_stride * sizeof(float2);
  int per_sm = 0;
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_permute, kPermThreads, smem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  const long long work = (1ll << no) * batch;
  long long grid = (long long)num_sms() * per_sm;
  if (grid > work) grid = work;
  k_permute<<<(unsigned)grid, kPermThreads, smem, s>>>(P, batch, in, out);
  return cudaGetLastError();
}

}  // namespace tnq
