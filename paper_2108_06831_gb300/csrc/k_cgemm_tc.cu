// Kernel (c), tensor-core forms: batched complex GEMM on tcgen05 with TMEM accumulators.
//
// A pairwise merge of two tensors is the product of Eq. 2.2, C[m][n] = sum_k A[m][k] B[n][k]
// once the legs are grouped (both operands with the contracted index contiguous).  The
// complex product is computed as one real GEMM: A (complex M x K, interleaved) is already
// the real M x 2K matrix [re im re im ...], and B is replaced by its 2x2 real embedding
// B2 (2N x 2K) with rows 2n = (Br, -Bi) and 2n+1 = (Bi, Br) per k, so that the real
// product A B2^T, read as interleaved pairs, is exactly Cr = ArBr - AiBi, Ci = ArBi + AiBr.
//
// FP32 accuracy on low-precision tensor cores comes from splitting the operands:
//   3XTF32:     x = hi + lo, hi = x rounded to TF32, lo = x - hi (exact);
//               C = hi*hi + hi*lo + lo*hi (kind::tf32, three MMAs per K slice);
//   SPLIT_BF16: x = x0 + x1 + x2 with x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1);
//               C = x0y0 + x0y1 + x1y0 + x0y2 + x1y1 + x2y0 (kind::f16 with bf16 operands).
// The embedding and split of B are written once per call into the workspace by a small prep
// kernel.  For 3XTF32 with at most two column tiles (HBM-bound merges) the A operand is
// split inside the GEMM: its FP32 tile arrives by TMA,
// and four converter warps overwrite it with hi and write lo beside it (same element size and
// swizzle, so the split is elementwise at equal offsets) before the MMAs read the stage; A
// then crosses HBM once, as FP32.  Otherwise A is split by a prep kernel too.  The GEMM
// streams the parts with TMA (128-byte swizzle) through a multi-stage mbarrier pipeline, a
// single thread issues tcgen05.mma into four 128 x BN FP32 accumulators in tensor memory,
// and the four converter/epilogue warps drain them with tcgen05.ld.  Inside the
// MMA an addend loses its low bits against a large accumulator, so, following Ootomo and
// Yokota's error-corrected TF32 GEMM, the correction products are summed apart from the
// leading one, and the leading product itself is spread over three accumulators (K tiles
// round robin); the epilogue adds the four in round-to-nearest FP32.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "kernels.h"

namespace tnq {

cudaError_t launch_cgemm_fp32(long long batch, long long M, long long N, long long K, const float2 *A, const float2 *B,
                              float2 *C, void *ws, size_t ws_bytes, cudaStream_t s, const OutMap *om);
size_t cgemm_fp32_workspace(long long batch, long long M, long long N, long long K);

namespace {

constexpr int BM = 128;          // rows of A per CTA (MMA M)
constexpr int BN = 128;          // real columns of C per CTA (MMA N) = 64 complex columns
constexpr int KBYTES = 128;      // bytes of K per stage and operand row (one 128-byte swizzle span)
// warps 0-3: A split (3XTF32) and epilogue (warp w owns TMEM lanes 32w..32w+31);
// warp 4: TMA producer; warp 5: TMEM allocation and MMA issue
constexpr int kThreads = 192;
constexpr int kConvThreads = 128;
constexpr int kColBits = 6;  // log2 of the complex columns of a tile (BN / 2)
static_assert(BN / 2 == 1 << kColBits, "column table covers one tile");
constexpr int kMain = 3;                      // leading-product accumulators, used round robin by K tile
constexpr int kTmemCols = (kMain + 1) * BN;   // + one correction accumulator = all 512 columns
constexpr unsigned long long kWaitNs = 2000000000ull;  // bound of every mbarrier wait
constexpr int kRasterRows = 8;  // row tiles per group of the tile order (k_cgemm_tc)

enum : int { PREC_TF32 = 1, PREC_BF16 = 2 };

template <int PREC>
struct Cfg;
template <>
struct Cfg<PREC_TF32> {
  static constexpr int kElem = 4, kParts = 2, kProducts = 3, kStages = 3, kMmaK = 8, kFmt = 2;
  __device__ static int pa(int p) { return p == 2 ? 1 : 0; }  // (hi,hi), (hi,lo), (lo,hi)
  __device__ static int pb(int p) { return p == 1 ? 1 : 0; }
};
template <>
struct Cfg<PREC_BF16> {
  static constexpr int kElem = 2, kParts = 3, kProducts = 6, kStages = 2, kMmaK = 16, kFmt = 1;
  // (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
  __device__ static int pa(int p) { return p == 2 ? 1 : p == 4 ? 1 : p == 5 ? 2 : 0; }
  __device__ static int pb(int p) { return p == 1 ? 1 : p == 3 ? 2 : p == 4 ? 1 : 0; }
};

constexpr int kTileA = BM * KBYTES;  // bytes of one A part per stage
constexpr int kTileB = BN * KBYTES;

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, int n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(n));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait (about two seconds of wall time): false, and the device status word set, if
// the phase never completed.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, int *status) {
  if (mbar_try(b, parity)) return true;
  const unsigned long long t0 = now_ns();
  for (;;) {
    for (int i = 0; i < 256; ++i)
      if (mbar_try(b, parity)) return true;
    if (now_ns() - t0 > kWaitNs) break;
  }
  if (status) atomicCAS(status, 0, (int)TN_ERR_TIMEOUT);
  return false;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::
          "r"(saddr(dst)),
      "l"(map), "r"(saddr(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

// Shared-memory matrix descriptor (K-major operand, 128-byte swizzle, 8-row groups 1024 B apart).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);       // start address
  d |= (uint64_t)1 << 16;                        // leading byte offset (unused with this swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;              // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                        // descriptor version
  d |= (uint64_t)2 << 61;                        // 128-byte swizzle
  return d;
}

template <int PREC>
__device__ __forceinline__ constexpr uint32_t instr_desc() {
  return (1u << 4)                                   // D: F32
         | ((uint32_t)Cfg<PREC>::kFmt << 7)          // A format
         | ((uint32_t)Cfg<PREC>::kFmt << 10)         // B format
         | ((uint32_t)(BN >> 3) << 17)               // N
         | ((uint32_t)(BM >> 4) << 24);              // M
}

template <int PREC>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
  constexpr uint32_t idesc = instr_desc<PREC>();
  if constexpr (PREC == PREC_TF32) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  }
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}

// 32 consecutive fp32 columns of this warp's 32 TMEM lanes (one per thread); completes at
// the next tcgen05.wait::ld.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

// Output index of natural flat index bits [lo, nbits) of f under the map.
__device__ __forceinline__ long long map_bits(const OutMap &om, long long f, int lo) {
  long long r = 0;
  for (int i = lo; i < om.nbits; ++i)
    if ((f >> i) & 1) r |= 1ll << om.pos[i];
  return r;
}

// One 32-column chunk (16 complex values, interleaved) of a row of C, either row-major
// (identity map) or at mapped positions: rowaddr = map of the row and column-tile bits,
// ctab[j] = map of the tile-local column bits (j < 64).
__device__ __forceinline__ void store_chunk(const OutMap &om, float *crow, float2 *C2, long long rowaddr,
                                            const long long *ctab, int c, const float (&v)[32]) {
  if (om.identity) {
    float4 *dst = reinterpret_cast<float4 *>(crow + c);
#pragma unroll
    for (int k = 0; k < 8; ++k) dst[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
  } else {
#pragma unroll
    for (int q = 0; q < 16; ++q) C2[rowaddr + ctab[c / 2 + q]] = make_float2(v[2 * q], v[2 * q + 1]);
  }
}

struct TmaMaps {
  CUtensorMap a[3];
  CUtensorMap b[3];
};

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}

// SPLIT_A (3XTF32 only): A arrives as FP32 and is split in shared memory by warps 0-3.
template <int PREC, bool SPLIT_A>
__global__ void __launch_bounds__(kThreads, 1) k_cgemm_tc(const __grid_constant__ TmaMaps maps, int k_tiles,
                                                          long long M, long long N2, float *__restrict__ C,
                                                          int *status, const __grid_constant__ OutMap om) {
  using CF = Cfg<PREC>;
  static_assert(!SPLIT_A || PREC == PREC_TF32, "on-chip split is the TF32 form");
  pdl_wait();  // before any memory access or TMEM allocation: the previous kernel has completed
  pdl_trigger();
  constexpr int S = CF::kStages;
  constexpr int stage_bytes = CF::kParts * (kTileA + kTileB);
  // bytes the TMA delivers per stage: A once as FP32 when it is split here, else its parts
  constexpr uint32_t tx_bytes = (SPLIT_A ? kTileA : CF::kParts * kTileA) + CF::kParts * kTileB;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment of every tile (required by the 128-byte swizzle pattern)
  unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[S], conv[S], empty[S], done;
  __shared__ __align__(8) uint64_t drain;  // abort path: completion of the MMAs already issued
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ int issued_parity[S];  // parity of the last TMA phase issued per stage, -1 if none
  __shared__ long long ctab[BN / 2];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // tile order: CTAs launch in linear order; consecutive CTAs walk kRasterRows row tiles before the
  // next column tile, so the CTAs resident at once read few A and B panels and the panels they share
  // stay in L2 (row-major order would re-read every B panel once per wave of CTAs)
  int n0, m0;
  {
    const int tn = (int)gridDim.x, tm = (int)gridDim.y;
    const int pid = (int)blockIdx.y * tn + (int)blockIdx.x;
    const int group = pid / (kRasterRows * tn);
    const int first = group * kRasterRows;
    const int rows = tm - first < kRasterRows ? tm - first : kRasterRows;
    const int in = pid - group * kRasterRows * tn;
    m0 = (first + in % rows) * BM;
    n0 = (in / rows) * BN;
  }
  const int bz = blockIdx.z;
  if (threadIdx.x < BN / 2) ctab[threadIdx.x] = om.identity ? 0 : map_bits(om, threadIdx.x, 0);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], kConvThreads);
      mbar_init(&empty[s], 1);
      issued_parity[s] = -1;
    }
    mbar_init(&done, 1);
    mbar_init(&drain, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 5) {  // the whole warp allocates the accumulators' columns of tensor memory
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem_d = tmem_base;
  bool mma_issued = false;  // warp 5 lane 0: at least one MMA was issued

  if (warp == 4) {
    if (lane == 0) {  // TMA producer
      for (int kt = 0; kt < k_tiles; ++kt) {
        const int s = kt % S;
        if (kt >= S && !mbar_wait(&empty[s], ((kt / S) - 1) & 1, status)) {
          abort_flag = 1;
          break;
        }
        mbar_expect_tx(&full[s], tx_bytes);
        issued_parity[s] = (kt / S) & 1;
        unsigned char *st = smem + (size_t)s * stage_bytes;
        const int kc = kt * (KBYTES / CF::kElem);
        const int a_loads = SPLIT_A ? 1 : CF::kParts;
        for (int p = 0; p < a_loads; ++p) tma_load_3d(st + p * kTileA, &maps.a[p], &full[s], kc, m0, bz);
        for (int p = 0; p < CF::kParts; ++p)
          tma_load_3d(st + CF::kParts * kTileA + p * kTileB, &maps.b[p], &full[s], kc, n0, bz);
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {  // MMA issuer
      bool ok = true;
      for (int kt = 0; kt < k_tiles; ++kt) {
        const int s = kt % S;
        if (!mbar_wait(SPLIT_A ? &conv[s] : &full[s], (kt / S) & 1, status)) {
          ok = false;
          abort_flag = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t st = saddr(smem + (size_t)s * stage_bytes);
#pragma unroll
        for (int p = 0; p < CF::kProducts; ++p) {
          const uint32_t a_base = st + CF::pa(p) * kTileA;
          const uint32_t b_base = st + CF::kParts * kTileA + CF::pb(p) * kTileB;
#pragma unroll
          for (int kk = 0; kk < KBYTES / (CF::kMmaK * CF::kElem); ++kk) {
            const uint32_t off = kk * CF::kMmaK * CF::kElem;  // 32 bytes per MMA along K
            // product 0 (the leading parts) of K tile kt accumulates in columns [j BN, (j+1) BN),
            // j = kt mod kMain; the correction products in [kMain BN, (kMain+1) BN).  Small terms
            // never meet the large running sum inside the MMA, and each leading accumulator sees
            // a third of the K steps.
            const int j = kt % kMain;
            const uint32_t dst = tmem_d + (uint32_t)((p == 0 ? j : kMain) * BN);
            const bool acc = p == 0 ? (kt >= kMain || kk > 0) : (kt > 0 || kk > 0 || p > 1);
            mma<PREC>(dst, smem_desc(a_base + off), smem_desc(b_base + off), acc ? 1u : 0u);
          }
        }
        mma_issued = true;
        mma_commit(&empty[s]);  // frees the stage once these MMAs have read it
      }
      if (ok) mma_commit(&done);
    }
  } else if constexpr (SPLIT_A) {
    // A split: x -> hi = TF32(x) (in place), lo = x - hi (part 1 of the stage), then make the
    // generic-proxy writes visible to the tensor cores and report the stage converted
    for (int kt = 0; kt < k_tiles; ++kt) {
      const int s = kt % S;
      if (!mbar_wait(&full[s], (kt / S) & 1, status)) {
        abort_flag = 1;
        break;
      }
      float4 *hi = reinterpret_cast<float4 *>(smem + (size_t)s * stage_bytes);
      float4 *lo = reinterpret_cast<float4 *>(smem + (size_t)s * stage_bytes + kTileA);
#pragma unroll 4
      for (int c = threadIdx.x; c < kTileA / 16; c += kConvThreads) {
        const float4 v = hi[c];
        const float4 h = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
        lo[c] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
        hi[c] = h;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&conv[s]);
    }
  }
  __syncwarp();

  // epilogue: warps 0-3 drain their 32 TMEM lanes (= 32 rows of the tile)
  bool have = !abort_flag && mbar_wait(&done, 0, status);
  have = __all_sync(0xFFFFFFFFu, have);  // tcgen05.ld is warp-collective: decide per warp
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (have && warp < 4) {
    const long long row = m0 + warp * 32 + lane;
    float *crow = C + ((long long)bz * M + row) * N2 + n0;
    long long rowaddr = 0;
    if (!om.identity) {
      int lgn = 0;
      while ((2ll << lgn) < N2) ++lgn;  // complex columns = 2^lgn
      rowaddr = map_bits(om, (((long long)bz * M + row) << lgn) | (long long)(n0 / 2), kColBits);
    }
    const int n_main = k_tiles < kMain ? k_tiles : kMain;  // accumulators that were written
    for (int c = 0; c < BN; c += 32) {
      const uint32_t taddr = tmem_d + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
      float v[32];
      {
        uint32_t e[32];
        tmem_ld32(taddr + kMain * BN, e);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(e[i]);
      }
      for (int j = 0; j < n_main; ++j) {  // corrections first, then the leading sums in order
        uint32_t r[32];
        tmem_ld32(taddr + j * BN, r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] += __uint_as_float(r[i]);
      }
      store_chunk(om, crow, reinterpret_cast<float2 *>(C), rowaddr, ctab, c, v);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (abort_flag) {  // uniform: nothing writes the flag after the barrier above
    // let copies already in flight land (the last phase issued into each stage), and let the
    // MMAs already issued finish reading shared memory and writing TMEM, before the CTA
    // releases either
    if (threadIdx.x == 0)
      for (int s = 0; s < S; ++s)
        if (issued_parity[s] >= 0) mbar_wait(&full[s], (uint32_t)issued_parity[s], nullptr);
    if (warp == 5 && lane == 0 && mma_issued) {
      mma_commit(&drain);
      mbar_wait(&drain, 0, nullptr);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (warp == 5) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_d), "r"(kTmemCols));
  }
}

// Persistent form for short, HBM-bound merges (3XTF32 or SPLIT_BF16, A split on chip, at most
// kStreamMaxKTiles K tiles; a network merge has N = K = 64 and thousands of 128-row tiles):
// one CTA per SM walks the tiles (column tile fastest, then row tile, then batch), the TMA
// stage ring runs on across tile boundaries, and the accumulators are double-buffered in
// TMEM (leading + correction product per buffer, 2 x 2 x BN columns), so dedicated epilogue
// warps drain tile i while tile i+1 is loaded, split and multiplied.
// Warps 0-3: A split; warp 4: TMA; warp 5: TMEM allocation and MMA issue; warps 6-9:
// epilogue (warp w owns TMEM lanes 32 (w mod 4)..+31).
constexpr int kStreamThreads = 320;
constexpr int kStreamMaxKTiles = 8;  // a single leading accumulator per tile stays accurate
constexpr int kStgStride = 17;       // staging row stride (complex): rows fall in different banks

// Split of one A stage from FP32 into three BF16 parts, in place: the FP32 tile is two 128-byte
// boxes (K elements 32j..32j+31 of every row, 16-byte chunks swizzled by row mod 8); part p is a
// 128 x 64 BF16 tile at p x 16 KB (chunk d = K elements 8d..8d+7, same swizzle).  Each of the 128
// converter threads first reads its 8 output chunks' sources, then (after a named barrier: the
// parts overwrite the FP32 tile) writes x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1).
__device__ __forceinline__ void split_bf16_in_place(unsigned char *st) {
  float v[8][8];
#pragma unroll
  for (int it = 0; it < 8; ++it) {
    const int item = threadIdx.x + kConvThreads * it, r = item >> 3, d = item & 7;
    const unsigned char *row = st + (d >> 2) * kTileA + r * 128;
    const int c0 = 2 * (d & 3);
    const float4 a = *reinterpret_cast<const float4 *>(row + ((c0 ^ (r & 7)) << 4));
    const float4 b = *reinterpret_cast<const float4 *>(row + (((c0 + 1) ^ (r & 7)) << 4));
    v[it][0] = a.x, v[it][1] = a.y, v[it][2] = a.z, v[it][3] = a.w;
    v[it][4] = b.x, v[it][5] = b.y, v[it][6] = b.z, v[it][7] = b.w;
  }
  asm volatile("bar.sync 1, %0;" ::"n"(kConvThreads) : "memory");
#pragma unroll
  for (int it = 0; it < 8; ++it) {
    const int item = threadIdx.x + kConvThreads * it, r = item >> 3, d = item & 7;
    uint32_t w[3][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t h[3][2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const float x = v[it][2 * q + e];
        const __nv_bfloat16 b0 = __float2bfloat16_rn(x);
        const float r1 = x - __bfloat162float(b0);
        const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
        const __nv_bfloat16 b2 = __float2bfloat16_rn(r1 - __bfloat162float(b1));
        h[0][e] = __bfloat16_as_ushort(b0);
        h[1][e] = __bfloat16_as_ushort(b1);
        h[2][e] = __bfloat16_as_ushort(b2);
      }
#pragma unroll
      for (int p = 0; p < 3; ++p) w[p][q] = h[p][0] | (h[p][1] << 16);
    }
#pragma unroll
    for (int p = 0; p < 3; ++p)
      *reinterpret_cast<uint4 *>(st + p * kTileA + r * 128 + ((d ^ (r & 7)) << 4)) =
          make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
  }
}

template <int PREC>
__global__ void __launch_bounds__(kStreamThreads, 1)
    k_cgemm_tc_stream(const __grid_constant__ TmaMaps maps, int k_tiles, int tiles_n, int tiles_m,
                      long long total_tiles, long long M, long long N2, float *__restrict__ C, int *status,
                      const __grid_constant__ OutMap om) {
  using CF = Cfg<PREC>;
  pdl_wait();  // before any memory access or TMEM allocation: the previous kernel has completed
  pdl_trigger();
  constexpr int S = CF::kStages;
  constexpr int stage_bytes = CF::kParts * (kTileA + kTileB);
  // A arrives as FP32: one 128-byte box per row and K tile for TF32, two for BF16 (64 elements)
  constexpr int a_boxes = PREC == PREC_TF32 ? 1 : 2;
  constexpr uint32_t tx_bytes = a_boxes * kTileA + CF::kParts * kTileB;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[S], conv[S], empty[S], acc_full[2], acc_empty[2], drain;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ int issued_parity[S];  // parity of the last TMA phase issued per stage, -1 if none
  // Permuted epilogue: a warp stages 32 rows x 16 complex columns (one 32-float chunk of its
  // rows) and writes them back in stored-index order.  The chunk's 9 local bits (5 row, 4
  // column) are enumerated by increasing stored position (u); u -> staging offset and u ->
  // stored offset are linear in u's bits, tabulated for u's low 5 and high 4 bits.
  __shared__ float2 stage_c[4][32 * kStgStride];
  __shared__ int sm_lo[32], sm_hi[16];
  __shared__ long long g_lo[32], g_hi[16];
  __shared__ int pairs_contig;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (!om.identity && threadIdx.x == 0) {
    int lgn = 0;
    while ((2ll << lgn) < N2) ++lgn;
    // local bit b: b < 4 column bit b (stored at pos[b]); b >= 4 row bit b - 4 (pos[lgn + b - 4])
    int spos[9], order[9];
    for (int b = 0; b < 9; ++b) {
      spos[b] = b < 4 ? om.pos[b] : om.pos[lgn + b - 4];
      order[b] = b;
    }
    for (int i = 1; i < 9; ++i)  // insertion sort by stored position
      for (int j = i; j > 0 && spos[order[j - 1]] > spos[order[j]]; --j) {
        const int t = order[j];
        order[j] = order[j - 1];
        order[j - 1] = t;
      }
    auto contrib_s = [&](int b) { return b < 4 ? (1 << b) : (kStgStride << (b - 4)); };
    for (int u = 0; u < 32; ++u) {
      int so = 0;
      long long go = 0;
      for (int k = 0; k < 5; ++k)
        if ((u >> k) & 1) {
          so += contrib_s(order[k]);
          go += 1ll << spos[order[k]];
        }
      sm_lo[u] = so;
      g_lo[u] = go;
    }
    for (int u = 0; u < 16; ++u) {
      int so = 0;
      long long go = 0;
      for (int k = 0; k < 4; ++k)
        if ((u >> k) & 1) {
          so += contrib_s(order[5 + k]);
          go += 1ll << spos[order[5 + k]];
        }
      sm_hi[u] = so;
      g_hi[u] = go;
    }
    pairs_contig = spos[order[0]] == 0 ? 1 : 0;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], kConvThreads);
      mbar_init(&empty[s], 1);
      issued_parity[s] = -1;
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 128);
    }
    mbar_init(&drain, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem_d = tmem_base;
  bool mma_issued = false;  // warp 5 lane 0: at least one MMA was issued

  auto aborted = [&]() { return *reinterpret_cast<volatile int *>(&abort_flag) != 0; };
  auto decode = [&](long long t, int &nt, int &mt, int &bz) {
    nt = (int)(t % tiles_n);
    const long long r = t / tiles_n;
    mt = (int)(r % tiles_m);
    bz = (int)(r / tiles_m);
  };

  if (warp == 4) {
    if (lane == 0) {  // TMA producer
      long long g = 0;
      for (long long t = blockIdx.x; t < total_tiles && !aborted(); t += gridDim.x) {
        int nt, mt, bz;
        decode(t, nt, mt, bz);
        for (int kt = 0; kt < k_tiles; ++kt, ++g) {
          const int s = (int)(g % S);
          if (g >= S && !mbar_wait(&empty[s], (uint32_t)(((g / S) - 1) & 1), status)) {
            abort_flag = 1;
            break;
          }
          mbar_expect_tx(&full[s], tx_bytes);
          issued_parity[s] = (int)((g / S) & 1);
          unsigned char *st = smem + (size_t)s * stage_bytes;
          const int kc = kt * (KBYTES / CF::kElem);  // K elements before this tile
          for (int j = 0; j < a_boxes; ++j) tma_load_3d(st + j * kTileA, &maps.a[0], &full[s], kc + 32 * j, mt * BM, bz);
          for (int p = 0; p < CF::kParts; ++p)
            tma_load_3d(st + CF::kParts * kTileA + p * kTileB, &maps.b[p], &full[s], kc, nt * BN, bz);
        }
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {  // MMA issuer
      long long g = 0, li = 0;
      for (long long t = blockIdx.x; t < total_tiles && !aborted(); t += gridDim.x, ++li) {
        const int ab = (int)(li & 1);
        if (li >= 2 && !mbar_wait(&acc_empty[ab], (uint32_t)(((li / 2) - 1) & 1), status)) {
          abort_flag = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t base = tmem_d + (uint32_t)(ab * 2 * BN);
        bool ok = true;
        for (int kt = 0; kt < k_tiles; ++kt, ++g) {
          const int s = (int)(g % S);
          if (!mbar_wait(&conv[s], (uint32_t)((g / S) & 1), status)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t st = saddr(smem + (size_t)s * stage_bytes);
#pragma unroll
          for (int p = 0; p < CF::kProducts; ++p) {
            const uint32_t a_base = st + CF::pa(p) * kTileA;
            const uint32_t b_base = st + CF::kParts * kTileA + CF::pb(p) * kTileB;
#pragma unroll
            for (int kk = 0; kk < KBYTES / (CF::kMmaK * CF::kElem); ++kk) {
              const uint32_t off = kk * CF::kMmaK * CF::kElem;
              const uint32_t dst = p == 0 ? base : base + BN;
              const bool acc = p == 0 ? (kt > 0 || kk > 0) : (kt > 0 || kk > 0 || p > 1);
              mma<PREC>(dst, smem_desc(a_base + off), smem_desc(b_base + off), acc ? 1u : 0u);
            }
          }
          mma_issued = true;
          mma_commit(&empty[s]);
        }
        if (!ok) {
          abort_flag = 1;
          break;
        }
        mma_commit(&acc_full[ab]);
      }
    }
  } else if (warp < 4) {  // A split, as in k_cgemm_tc
    long long g = 0;
    for (long long t = blockIdx.x; t < total_tiles; t += gridDim.x) {
      bool ok = true;
      for (int kt = 0; kt < k_tiles; ++kt, ++g) {
        const int s = (int)(g % S);
        if (!mbar_wait(&full[s], (uint32_t)((g / S) & 1), status)) {
          ok = false;
          break;
        }
        if constexpr (PREC == PREC_TF32) {
          float4 *hi = reinterpret_cast<float4 *>(smem + (size_t)s * stage_bytes);
          float4 *lo = reinterpret_cast<float4 *>(smem + (size_t)s * stage_bytes + kTileA);
#pragma unroll 4
          for (int c = threadIdx.x; c < kTileA / 16; c += kConvThreads) {
            const float4 v = hi[c];
            const float4 h = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
            lo[c] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
            hi[c] = h;
          }
        } else {
          split_bf16_in_place(smem + (size_t)s * stage_bytes);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&conv[s]);
      }
      if (!ok) {
        abort_flag = 1;
        break;
      }
    }
  } else {  // epilogue warps 6-9
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    int lgn = 0;
    while ((2ll << lgn) < N2) ++lgn;  // complex columns = 2^lgn
    long long li = 0;
    for (long long t = blockIdx.x; t < total_tiles; t += gridDim.x, ++li) {
      const int ab = (int)(li & 1);
      bool have = mbar_wait(&acc_full[ab], (uint32_t)((li / 2) & 1), status);
      have = __all_sync(0xFFFFFFFFu, have);
      if (!have) {
        abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int nt, mt, bz;
      decode(t, nt, mt, bz);
      const long long row0 = (long long)bz * M + (long long)mt * BM + q * 32;  // the warp's first row
      const uint32_t base = tmem_d + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * 2 * BN);
      float2 *stg = stage_c[q];
      for (int c = 0; c < BN; c += 32) {
        uint32_t r[32], e[32];
        tmem_ld32(base + BN + c, e);  // corrections
        tmem_ld32(base + c, r);       // leading product
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float v[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(e[k]) + __uint_as_float(r[k]);
        if (om.identity) {
          // row-major: stage, then 8 lanes write each row's 128 bytes (4 rows per store)
#pragma unroll
          for (int k = 0; k < 16; ++k) stg[lane * kStgStride + k] = make_float2(v[2 * k], v[2 * k + 1]);
          __syncwarp();
          const float *cbase = C + ((long long)row0 * N2 + (long long)nt * BN + c);
#pragma unroll
          for (int it = 0; it < 8; ++it) {
            const int pr = it * 32 + lane;  // pair index: row pr / 8, complex pair pr % 8
            const int rr = pr >> 3, cc = 2 * (pr & 7);
            const float2 x0 = stg[rr * kStgStride + cc], x1 = stg[rr * kStgStride + cc + 1];
            *reinterpret_cast<float4 *>(const_cast<float *>(cbase) + (long long)rr * N2 + 2 * cc) =
                make_float4(x0.x, x0.y, x1.x, x1.y);
          }
          __syncwarp();
          continue;
        }
        // stored offset of everything but the chunk's local bits (lane row bits, 4 column bits)
        const long long gbase = map_bits(om, (row0 << lgn) | ((long long)nt * (BN / 2) + c / 2), 0);
#pragma unroll
        for (int k = 0; k < 16; ++k) stg[lane * kStgStride + k] = make_float2(v[2 * k], v[2 * k + 1]);
        __syncwarp();
        float2 *C2 = reinterpret_cast<float2 *>(C);
#pragma unroll
        for (int it = 0; it < 8; ++it) {
          const int u = 64 * it + 2 * lane;  // even: u and u + 1 differ in the lowest sorted bit
          const float2 x0 = stg[sm_lo[u & 31] + sm_hi[u >> 5]];
          const float2 x1 = stg[sm_lo[(u + 1) & 31] + sm_hi[(u + 1) >> 5]];
          const long long g0 = gbase + g_lo[u & 31] + g_hi[u >> 5];
          if (pairs_contig) {
            *reinterpret_cast<float4 *>(C2 + g0) = make_float4(x0.x, x0.y, x1.x, x1.y);
          } else {
            C2[g0] = x0;
            C2[gbase + g_lo[(u + 1) & 31] + g_hi[(u + 1) >> 5]] = x1;
          }
        }
        __syncwarp();
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&acc_empty[ab]);
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (abort_flag) {  // uniform: nothing writes the flag after the barrier above
    // let copies already in flight land, and the MMAs already issued finish, before the CTA
    // releases its shared memory and tensor memory
    if (threadIdx.x == 0)
      for (int s = 0; s < S; ++s)
        if (issued_parity[s] >= 0) mbar_wait(&full[s], (uint32_t)issued_parity[s], nullptr);
    if (warp == 5 && lane == 0 && mma_issued) {
      mma_commit(&drain);
      mbar_wait(&drain, 0, nullptr);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (warp == 5) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_d), "r"(kTmemCols));
  }
}

// ------------------------------------------------------------------------------ prep kernels

// A (real view [rows][cols]) -> parts
template <int PREC>
__global__ void k_split(const float *__restrict__ x, long long n, void *p0, void *p1, void *p2) {
  pdl_wait();
  pdl_trigger();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float v = x[i];
    if constexpr (PREC == PREC_TF32) {
      const float hi = tf32_rna(v);
      static_cast<float *>(p0)[i] = hi;
      static_cast<float *>(p1)[i] = v - hi;
    } else {
      const __nv_bfloat16 b0 = __float2bfloat16_rn(v);
      const float r1 = v - __bfloat162float(b0);
      const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
      const float r2 = r1 - __bfloat162float(b1);
      static_cast<__nv_bfloat16 *>(p0)[i] = b0;
      static_cast<__nv_bfloat16 *>(p1)[i] = b1;
      static_cast<__nv_bfloat16 *>(p2)[i] = __float2bfloat16_rn(r2);
    }
  }
}

// B (complex [N][K]) -> 2x2 real embedding [2N][2K], then split.
template <int PREC>
__global__ void k_embed_split(const float2 *__restrict__ b, long long N, long long K, long long batch, void *p0,
                              void *p1, void *p2) {
  pdl_wait();
  pdl_trigger();
  const long long total = batch * N * K;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long bb = i / (N * K), r = i % (N * K), n = r / K, k = r % K;
    const float2 v = b[i];
    const long long base = bb * (2 * N) * (2 * K);
    const long long i0 = base + (2 * n) * (2 * K) + 2 * k;      // row 2n:   (re, -im)
    const long long i1 = base + (2 * n + 1) * (2 * K) + 2 * k;  // row 2n+1: (im,  re)
    const float e[4] = {v.x, -v.y, v.y, v.x};
    const long long at[4] = {i0, i0 + 1, i1, i1 + 1};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float x = e[q];
      if constexpr (PREC == PREC_TF32) {
        const float hi = tf32_rna(x);
        static_cast<float *>(p0)[at[q]] = hi;
        static_cast<float *>(p1)[at[q]] = x - hi;
      } else {
        const __nv_bfloat16 b0 = __float2bfloat16_rn(x);
        const float r1 = x - __bfloat162float(b0);
        const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(b1);
        static_cast<__nv_bfloat16 *>(p0)[at[q]] = b0;
        static_cast<__nv_bfloat16 *>(p1)[at[q]] = b1;
        static_cast<__nv_bfloat16 *>(p2)[at[q]] = __float2bfloat16_rn(r2);
      }
    }
  }
}

// ------------------------------------------------------------------------------ host side

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

bool make_map(CUtensorMap *m, const void *base, int elem, long long cols, long long rows, long long batch, int box_rows) {
  auto enc = encode_fn();
  if (!enc) return false;
  const CUtensorMapDataType dt = elem == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)cols * elem, (cuuint64_t)cols * rows * elem};
  cuuint32_t box[3] = {(cuuint32_t)(KBYTES / elem), (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return enc(m, dt, 3, const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// K needs no multiple of the K tile: the TMA fills the part of a K tile beyond the operands
// with zeros (exact zero products); only the row stride must be a multiple of 16 bytes.
bool tc_shape_ok(int precision, long long M, long long N, long long K) {
  const long long elem = precision == TN_PREC_3XTF32 ? 4 : 2;
  return M % BM == 0 && (2 * N) % BN == 0 && (2 * K * elem) % 16 == 0 && M > 0 && N > 0 && K > 0 &&
         M * 2 * N < (1ll << 40);
}

int k_tiles_of(int precision, long long K) {
  const long long elem = precision == TN_PREC_3XTF32 ? 4 : 2;
  return (int)((2 * K * elem + KBYTES - 1) / KBYTES);
}

size_t part_bytes(int precision, long long rows, long long cols, long long batch) {
  return (size_t)rows * cols * batch * (precision == TN_PREC_3XTF32 ? 4 : 2);
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// A is split on chip when few CTAs read each A tile (HBM-bound merges: the split copy would
// cost more traffic than the GEMM); with many column tiles the one-pass prep split is
// cheaper than converting every tile again in every CTA.
bool split_a_on_chip(int precision, long long N, long long K) {
  if ((2 * N) / BN > 2) return false;
  if (precision == TN_PREC_3XTF32) return true;
  // BF16 parts are made on chip by the streaming kernel only (short K)
  return precision == TN_PREC_SPLIT_BF16 && k_tiles_of(precision, K) <= kStreamMaxKTiles;
}

template <int PREC, bool SPLIT_A>
cudaError_t run_tc(long long batch, long long M, long long N, long long K, const float2 *A, const float2 *B, float2 *C,
                   void *ws, cudaStream_t s, const OutMap &om) {
  using CF = Cfg<PREC>;
  const int prec_abi = PREC == PREC_TF32 ? TN_PREC_3XTF32 : TN_PREC_SPLIT_BF16;
  const size_t pa = SPLIT_A ? 0 : align256(part_bytes(prec_abi, M, 2 * K, batch));
  const size_t pb = align256(part_bytes(prec_abi, 2 * N, 2 * K, batch));
  char *w = static_cast<char *>(ws);
  void *ap[3] = {w, w + pa, w + 2 * pa};
  char *wb = w + CF::kParts * pa;
  void *bp[3] = {wb, wb + pb, wb + 2 * pb};
  cudaError_t e = cudaSuccess;
  if (SPLIT_A) {
    ap[0] = const_cast<float2 *>(A);  // the GEMM reads A itself (FP32) and splits it on chip
  } else {
    const long long na = batch * M * 2 * K;
    e = launch_pdl(k_split<PREC>, dim3((unsigned)std::min<long long>((na + 255) / 256, 65535)), dim3(256), 0, s,
                   reinterpret_cast<const float *>(A), na, ap[0], ap[1], ap[2]);
    if (e != cudaSuccess) return e;
  }
  const long long nb = batch * N * K;
  e = launch_pdl(k_embed_split<PREC>, dim3((unsigned)std::min<long long>((nb + 255) / 256, 65535)), dim3(256), 0, s,
                 B, N, K, batch, bp[0], bp[1], bp[2]);
  if (e != cudaSuccess) return e;
  TmaMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  for (int p = 0; p < CF::kParts; ++p) {
    // A split on chip arrives as FP32 (4-byte elements) whatever the parts' type
    if ((!SPLIT_A || p == 0) && !make_map(&maps.a[p], ap[p], SPLIT_A ? 4 : CF::kElem, 2 * K, M, batch, BM))
      return cudaErrorInvalidValue;
    if (!make_map(&maps.b[p], bp[p], CF::kElem, 2 * K, 2 * N, batch, BN)) return cudaErrorInvalidValue;
  }
  const size_t smem = (size_t)CF::kStages * CF::kParts * (kTileA + kTileB) + 1024;
  const int k_tiles = k_tiles_of(prec_abi, K);
  if constexpr (SPLIT_A) {
    if (k_tiles <= kStreamMaxKTiles) {  // short merge: persistent CTAs with overlapped epilogue
      e = ensure_smem(reinterpret_cast<const void *>(k_cgemm_tc_stream<PREC>), smem);
      if (e != cudaSuccess) return e;
      const int tiles_n = (int)((2 * N) / BN), tiles_m = (int)(M / BM);
      const long long total = (long long)tiles_n * tiles_m * batch;
      const long long grid = std::min<long long>(total, num_sms());
      return launch_pdl(k_cgemm_tc_stream<PREC>, dim3((unsigned)grid), dim3(kStreamThreads), smem, s, maps, k_tiles,
                        tiles_n, tiles_m, total, M, 2 * N, reinterpret_cast<float *>(C),
                        static_cast<int *>(status_word_ptr()), om);
    }
  }
  if constexpr (SPLIT_A && PREC == PREC_BF16) {
    return cudaErrorNotSupported;  // the on-chip BF16 split exists in the streaming form only
  } else {
    e = ensure_smem(reinterpret_cast<const void *>(k_cgemm_tc<PREC, SPLIT_A>), smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((2 * N) / BN), (unsigned)(M / BM), (unsigned)batch);
    return launch_pdl(k_cgemm_tc<PREC, SPLIT_A>, grid, dim3(kThreads), smem, s, maps, k_tiles, M, 2 * N,
                      reinterpret_cast<float *>(C), static_cast<int *>(status_word_ptr()), om);
  }
}

}  // namespace

size_t cgemm_workspace(int precision, long long batch, long long M, long long N, long long K) {
  if (precision == TN_PREC_FP32) return cgemm_fp32_workspace(batch, M, N, K);
  if (!tc_shape_ok(precision, M, N, K)) return 0;
  const int parts = precision == TN_PREC_3XTF32 ? 2 : 3;
  // A split on chip: only B's parts are stored
  if (split_a_on_chip(precision, N, K)) return parts * align256(part_bytes(precision, 2 * N, 2 * K, batch));
  return parts * (align256(part_bytes(precision, M, 2 * K, batch)) + align256(part_bytes(precision, 2 * N, 2 * K, batch)));
}

cudaError_t launch_cgemm(int precision, long long batch, long long M, long long N, long long K, const float2 *A,
                         const float2 *B, float2 *C, void *ws, size_t ws_bytes, cudaStream_t s, const OutMap *om) {
  if (precision == TN_PREC_FP32) return launch_cgemm_fp32(batch, M, N, K, A, B, C, ws, ws_bytes, s, om);
  const OutMap ident;
  const OutMap &m = om ? *om : ident;
  if (!tc_shape_ok(precision, M, N, K)) return cudaErrorNotSupported;
  if (batch > 65535 || M / BM > 65535) return cudaErrorNotSupported;
  if (ws_bytes < cgemm_workspace(precision, batch, M, N, K)) return cudaErrorInvalidValue;
  if (precision == TN_PREC_3XTF32)
    return split_a_on_chip(precision, N, K) ? run_tc<PREC_TF32, true>(batch, M, N, K, A, B, C, ws, s, m)
                                            : run_tc<PREC_TF32, false>(batch, M, N, K, A, B, C, ws, s, m);
  return split_a_on_chip(precision, N, K) ? run_tc<PREC_BF16, true>(batch, M, N, K, A, B, C, ws, s, m)
                                          : run_tc<PREC_BF16, false>(batch, M, N, K, A, B, C, ws, s, m);
}

}  // namespace tnq
