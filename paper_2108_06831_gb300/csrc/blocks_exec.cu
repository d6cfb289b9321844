// Launcher of the uniform-block state contraction (see blocks.h): per call, the block
// matrices are precontracted from the parameters (FP64), block 0 is applied to the basis
// state directly, and every further block is one batched complex GEMM (kernel c) of the
// state viewed as [2^(N-k)] x [2^k] against the block's 2^k x 2^k matrix, stored through the
// output map in the layout the next block reads.
#include <cstring>

#include "blocks.h"

namespace tnq {

namespace {

constexpr int kBuildThreads = 128;
constexpr int kBuildCols = 8;     // columns of a block matrix built per CTA
constexpr int kBuildChunk = 32;   // gate matrices evaluated together (in parallel) per round

__device__ __forceinline__ int insert_zero(int p, int t) { return ((p >> t) << (t + 1)) | (p & ((1 << t) - 1)); }

// CTA (block i, column chunk, batch element b): columns [c0, c0 + 8) of block i's matrix, by
// applying the block's gates in order to the unit vectors e_c (FP64, shared memory), stored as
// complex64 at mats[((i batch + b) 2^k + row) 2^k + col] (row-major: the GEMM's B operand).
// The gates' own matrices are evaluated kBuildChunk at a time, one per thread, then applied
// one after another by all threads.
__global__ void __launch_bounds__(kBuildThreads) k_block_build(const BlockGate *__restrict__ gates,
                                                               const int *__restrict__ meta, int k,
                                                               const double *__restrict__ params, int n_params,
                                                               int batch, float2 *__restrict__ mats) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double2 *col = reinterpret_cast<double2 *>(smraw);                   // [2^k rows][8 columns]
  __shared__ double gm[kBuildChunk][32];                              // gate matrices (re, im)
  const int i = blockIdx.x, c0 = blockIdx.y * kBuildCols, b = blockIdx.z;
  const int D = 1 << k;
  for (int e = threadIdx.x; e < D * kBuildCols; e += blockDim.x) {
    const int r = e / kBuildCols, cc = e % kBuildCols;
    col[e] = make_double2(r == c0 + cc ? 1.0 : 0.0, 0.0);
  }
  const int gb = meta[2 * i], gc = meta[2 * i + 1];
  const double *prow = params ? params + (long long)b * n_params : nullptr;
  for (int g0 = 0; g0 < gc; g0 += kBuildChunk) {
    const int gn = gc - g0 < kBuildChunk ? gc - g0 : kBuildChunk;
    __syncthreads();  // the previous round's matrices are no longer read
    if (threadIdx.x < gn) {
      const BlockGate &bg = gates[gb + g0 + threadIdx.x];
      double ang[3] = {bg.angle[0], bg.angle[1], bg.angle[2]};
      for (int a = 0; a < 3; ++a)
        for (int q = 0; q < 2; ++q)
          if (bg.pidx[a][q] >= 0 && prow) ang[a] += prow[bg.pidx[a][q]];
      gate_matrix(bg.kind, FORM_U, ang, bg.mat, gm[threadIdx.x]);
    }
    for (int g = 0; g < gn; ++g) {
      __syncthreads();  // matrices written / the previous gate's updates done
      const BlockGate &bg = gates[gb + g0 + g];
      const double *u = gm[g];
      if (bg.lb < 0) {
        const int t = bg.la;
        for (int e = threadIdx.x; e < (D / 2) * kBuildCols; e += blockDim.x) {
          const int p = e / kBuildCols, cc = e % kBuildCols;
          const int r0 = insert_zero(p, t), r1 = r0 | (1 << t);
          const double2 x = col[r0 * kBuildCols + cc], y = col[r1 * kBuildCols + cc];
          col[r0 * kBuildCols + cc] = make_double2(u[0] * x.x - u[1] * x.y + u[2] * y.x - u[3] * y.y,
                                                   u[0] * x.y + u[1] * x.x + u[2] * y.y + u[3] * y.x);
          col[r1 * kBuildCols + cc] = make_double2(u[4] * x.x - u[5] * x.y + u[6] * y.x - u[7] * y.y,
                                                   u[4] * x.y + u[5] * x.x + u[6] * y.y + u[7] * y.x);
        }
      } else {
        // 4x4 indexed 2 bit(first) + bit(second); first qubit at local bit la
        const int ta = bg.la, tb = bg.lb;
        const int lo = ta < tb ? ta : tb, hi = ta < tb ? tb : ta;
        for (int e = threadIdx.x; e < (D / 4) * kBuildCols; e += blockDim.x) {
          const int p = e / kBuildCols, cc = e % kBuildCols;
          const int r = insert_zero(insert_zero(p, lo), hi);
          int idx[4];
          double2 v[4];
          for (int m = 0; m < 4; ++m) {
            idx[m] = r | (((m >> 1) & 1) << ta) | ((m & 1) << tb);
            v[m] = col[idx[m] * kBuildCols + cc];
          }
          for (int m = 0; m < 4; ++m) {
            double re = 0.0, im = 0.0;
            for (int j = 0; j < 4; ++j) {
              const double ur = u[2 * (4 * m + j)], ui = u[2 * (4 * m + j) + 1];
              re += ur * v[j].x - ui * v[j].y;
              im += ur * v[j].y + ui * v[j].x;
            }
            col[idx[m] * kBuildCols + cc] = make_double2(re, im);
          }
        }
      }
    }
  }
  __syncthreads();
  float2 *dst = mats + ((long long)i * batch + b) * D * D;
  for (int e = threadIdx.x; e < D * kBuildCols; e += blockDim.x) {
    const int r = e / kBuildCols, cc = e % kBuildCols;
    const double2 v = col[e];
    dst[(long long)r * D + c0 + cc] = make_float2((float)v.x, (float)v.y);
  }
}

// Block 0 applied to the basis state: out[b][init_pos[r]] = U_0[b][r][init_local] (the rest of
// out was cleared).
__global__ void k_block_init(const float2 *__restrict__ mats, const long long *__restrict__ init_pos, int k,
                             int init_local, int n, int batch, float2 *__restrict__ out) {
  const int D = 1 << k;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= D * batch) return;
  const int b = e / D, r = e % D;
  out[((long long)b << n) + init_pos[r]] = mats[((long long)b * D + r) * D + init_local];
}

}  // namespace

tn_status upload_blocks(BlockPlan &bp, bool host_only, bool param_dependent, std::string &err) {
  const int nb = (int)bp.qubits.size();
  const size_t D = (size_t)1 << bp.k;
  const size_t state = ((size_t)sizeof(float2) << bp.n) * (size_t)bp.batch;
  auto align = [](size_t v) { return (v + 255) / 256 * 256; };
  bp.gemm_ws_bytes = cgemm_workspace(bp.precision, bp.batch, 1ll << (bp.n - bp.k), (long long)D, (long long)D);
  bp.ws_mats = 0;
  bp.ws_state = align((size_t)nb * bp.batch * D * D * sizeof(float2));
  bp.ws_gemm = align(bp.ws_state + state);
  bp.ws_bytes = align(bp.ws_gemm + bp.gemm_ws_bytes);
  if (host_only) return TN_OK;
  std::vector<int> meta((size_t)2 * nb);
  for (int i = 0; i < nb; ++i) {
    meta[(size_t)2 * i] = bp.gate_begin[(size_t)i];
    meta[(size_t)2 * i + 1] = bp.gate_count[(size_t)i];
  }
  cudaError_t e = cudaSuccess;
  auto up = [&](const void *src, size_t bytes, void **dst) {
    if (e != cudaSuccess || bytes == 0) return;
    e = cudaMalloc(dst, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
  };
  up(bp.gates.data(), bp.gates.size() * sizeof(BlockGate), (void **)&bp.d_gates);
  up(meta.data(), meta.size() * sizeof(int), (void **)&bp.d_meta);
  up(bp.init_pos.data(), bp.init_pos.size() * sizeof(long long), (void **)&bp.d_init_pos);
  if (e == cudaSuccess && !param_dependent) {
    // fixed angles: the block matrices are precontracted once, here
    const size_t mbytes = (size_t)nb * bp.batch * D * D * sizeof(float2);
    e = cudaMalloc((void **)&bp.d_fixed_mats, mbytes);
    if (e == cudaSuccess) e = build_block_mats(bp, nullptr, 0, bp.d_fixed_mats, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    err = std::string("block tables: ") + cudaGetErrorString(e);
    free_blocks(bp);
    return TN_ERR_CUDA;
  }
  return TN_OK;
}

cudaError_t build_block_mats(const BlockPlan &bp, const double *params, int n_params, float2 *mats, cudaStream_t s) {
  const int nb = (int)bp.qubits.size();
  const int D = 1 << bp.k;
  const size_t smem = (size_t)D * kBuildCols * sizeof(double2);
  k_block_build<<<dim3((unsigned)nb, (unsigned)(D / kBuildCols), (unsigned)bp.batch), kBuildThreads, smem, s>>>(
      bp.d_gates, bp.d_meta, bp.k, params, n_params, bp.batch, mats);
  return cudaGetLastError();
}

cudaError_t run_blocks(const BlockPlan &bp, const double *params, int n_params, float2 *state, void *ws,
                       cudaStream_t s) {
  const int nb = (int)bp.qubits.size();
  const int D = 1 << bp.k;
  char *w = static_cast<char *>(ws);
  float2 *mats = bp.d_fixed_mats ? bp.d_fixed_mats : reinterpret_cast<float2 *>(w + bp.ws_mats);
  float2 *other = reinterpret_cast<float2 *>(w + bp.ws_state);
  void *gws = bp.gemm_ws_bytes ? static_cast<void *>(w + bp.ws_gemm) : nullptr;
  cudaError_t e = cudaSuccess;
  if (!bp.d_fixed_mats) {
    e = build_block_mats(bp, params, n_params, mats, s);
    if (e != cudaSuccess) return e;
  }
  // the last GEMM must write `state`: start in the buffer that makes the ping-pong end there
  float2 *cur = ((nb - 1) % 2 == 0) ? state : other;
  float2 *nxt = cur == state ? other : state;
  e = cudaMemsetAsync(cur, 0, ((size_t)sizeof(float2) << bp.n) * (size_t)bp.batch, s);
  if (e != cudaSuccess) return e;
  const int ni = D * bp.batch;
  k_block_init<<<(ni + 255) / 256, 256, 0, s>>>(mats, bp.d_init_pos, bp.k, bp.init_local, bp.n, bp.batch, cur);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long M = 1ll << (bp.n - bp.k);
  for (int i = 1; i < nb; ++i) {
    const OutMap *om = bp.maps[(size_t)i].identity ? nullptr : &bp.maps[(size_t)i];
    e = launch_cgemm(bp.precision, bp.batch, M, D, D, cur, mats + (size_t)i * bp.batch * D * D, nxt, gws,
                     bp.gemm_ws_bytes, s, om);
    if (e != cudaSuccess) return e;
    float2 *t = cur;
    cur = nxt;
    nxt = t;
  }
  return cudaSuccess;
}

void free_blocks(BlockPlan &bp) {
  cudaFree(bp.d_fixed_mats);
  bp.d_fixed_mats = nullptr;
  cudaFree(bp.d_gates);
  cudaFree(bp.d_meta);
  cudaFree(bp.d_init_pos);
  bp.d_gates = nullptr;
  bp.d_meta = nullptr;
  bp.d_init_pos = nullptr;
}

}  // namespace tnq
