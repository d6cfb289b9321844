// FP64 reductions over the contracted state: Pauli-sum expectation values and H psi.
//
// Closing the state's open legs against an operator (Sec. 2.2.3 closes them with a basis
// state; an observable closes them with <psi| P) is a reduction over all 2^N entries:
//   <psi|P|psi> = sum_x i^ny (-1)^popc(x & zm) conj(psi[x ^ xm]) psi[x]
// for P with X/Y factors on the bits xm and Z/Y factors on zm.  Terms are grouped into
// tile passes whose tiles contain every flip bit of their terms, so each pass reads the
// state once (coalesced, staged in shared memory) and evaluates all of its terms from
// the tile.  Precision, step by step: a term's contribution and the sum over terms at one
// amplitude are FP32 (coefficients rounded to FP32); a thread's sum over its amplitudes of one
// tile (tile / 256 of them, 16 for 12-qubit tiles) is FP32; the sums across tiles, warps and
// CTAs are FP64, and the per-CTA partials are summed in a fixed order (deterministic result).
// The FP32 steps add at most about (terms + tile/256) 2^-24 sum_k |c_k| <ps|ps> to the result
// (about 1e-5 absolute for the 39 unit terms of a 20-qubit Ising chain); FP64 takes over where
// the long sums and their cancellation are, over the 2^N / 16 per-thread partials.  Doing the
// per-amplitude work in FP64 would make the pass FP64-bound on GB300 (a few FP64 operations
// per SM and clock) instead of HBM-bound.
#include "apply_common.cuh"
#include "kernels.h"

namespace tnq {

constexpr int kRedThreads = 256;
constexpr int kRedGroup = 8;  // amplitudes a thread holds in registers at once (a tile gives it up to 16)
constexpr int kRedMaxCTAs = 512;  // per pass and batch element

namespace {

__device__ __forceinline__ float2 times_i_pow(float2 z, int ny) {
  switch (ny & 3) {
    case 0: return z;
    case 1: return make_float2(-z.y, z.x);
    case 2: return make_float2(-z.x, -z.y);
    default: return make_float2(z.y, -z.x);
  }
}

struct TileCtx {
  int T, L, tile, lowmask;
  long long *run_off;
};

__device__ void setup_tile(const RedPass &rp, long long *run_off, TileCtx &c) {
  c.T = rp.T;
  c.L = c.T < kLowBits ? c.T : kLowBits;
  c.tile = 1 << c.T;
  c.lowmask = (1 << c.L) - 1;
  c.run_off = run_off;
  for (int r = threadIdx.x; r < (1 << (c.T - c.L)); r += blockDim.x) {
    long long off = 0;
    for (int j = 0; j < c.T - c.L; ++j)
      if ((r >> j) & 1) off |= 1ll << rp.tile_pos[c.L + j];
    run_off[r] = off;
  }
}

__device__ __forceinline__ unsigned long long tile_base(const RedPass &rp, long long t) {
  unsigned long long base = 0;
  for (int j = 0; j < rp.n_outer; ++j) base |= (unsigned long long)((t >> j) & 1) << rp.outer_pos[j];
  return base;
}

__device__ __forceinline__ void load_tile(float2 *sm, const float2 *st, unsigned long long base, const TileCtx &c) {
  for (int k = threadIdx.x; k < (c.tile >> 1); k += blockDim.x) {
    const int i = k << 1;
    const long long g = (long long)base + c.run_off[i >> c.L] + (i & c.lowmask);
    const float4 v = *reinterpret_cast<const float4 *>(st + g);
    sm[swz(i)] = make_float2(v.x, v.y);
    sm[swz(i + 1)] = make_float2(v.z, v.w);
  }
}

__device__ __forceinline__ double block_sum(double v, double *scratch) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += scratch[w];
  __syncthreads();
  return s;
}

}  // namespace

// Terms of a pass as the tile loop reads them: shared-memory copies with the tile-local
// Z mask (zl) and, per tile, the parity of the Z mask on the tile's outer bits (sb).
struct TermSm {
  float coef;
  int xl;   // tile-local flip mask
  int zl;   // tile-local Z/Y mask
  int ny;
  // sign parity of the tile bits above the thread bits: bit J is the parity of ((J << 8) ^ f) & zl
  // above bit 7, J = the 256-amplitude row of a tile index (f = xl for H psi, 0 for <P>), so the
  // parity of (i ^ f) & zl for i = tid + 256 J is that bit xor a per-thread one
  int hi;
};
// hi of a term: the parities for J = 0 .. 15 (tiles of at most 2^12 amplitudes)
__device__ __forceinline__ int row_parities(int f, int zl) {
  int h = 0;
  for (int J = 0; J < 16; ++J) h |= (__popc(((J << 8) ^ f) & zl & ~0xFF) & 1) << J;
  return h;
}

__device__ __forceinline__ int compress_bits(unsigned long long v, const RedPass &rp) {
  int r = 0;
  for (int j = 0; j < rp.T; ++j) r |= (int)((v >> rp.tile_pos[j]) & 1ull) << j;
  return r;
}

__global__ void __launch_bounds__(kRedThreads) k_expect_pass(const RedPass *__restrict__ passes, int pass_idx,
                                                             int n_passes, const DevTerm *__restrict__ terms,
                                                             const float2 *__restrict__ state, int N,
                                                             double *__restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RedPass rp;
  __shared__ double scratch[kRedThreads / 32];
  for (int i = threadIdx.x; i < (int)(sizeof(RedPass) / 4); i += blockDim.x)
    reinterpret_cast<int *>(&rp)[i] = reinterpret_cast<const int *>(passes + pass_idx)[i];
  __syncthreads();
  TileCtx c;
  float2 *sm = reinterpret_cast<float2 *>(smem_raw);
  long long *run_off = reinterpret_cast<long long *>(smem_raw + ((size_t)sizeof(float2) << rp.T));
  const int n_runs = (1 << (rp.T - (rp.T < kLowBits ? rp.T : kLowBits)));
  const int nt = rp.term_end - rp.term_begin;
  TermSm *st_terms = reinterpret_cast<TermSm *>(run_off + (n_runs < 2 ? 2 : n_runs));
  unsigned char *sb = reinterpret_cast<unsigned char *>(st_terms + nt);  // per-tile base parity
  setup_tile(rp, run_off, c);
  for (int k = threadIdx.x; k < nt; k += blockDim.x) {
    const DevTerm &tm = terms[rp.term_begin + k];
    const int zl = compress_bits(tm.zm, rp);
    st_terms[k] = TermSm{(float)tm.coef, tm.xl, zl, tm.ny, row_parities(0, zl)};
  }
  __syncthreads();
  const int b = blockIdx.y;
  const float2 *st = state + ((long long)b << N);
  const long long n_tiles = 1ll << rp.n_outer;
  double acc = 0.0;
  for (long long t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const unsigned long long base = tile_base(rp, t);
    for (int k = threadIdx.x; k < nt; k += blockDim.x)
      sb[k] = (unsigned char)(__popcll(base & terms[rp.term_begin + k].zm) & 1);
    load_tile(sm, st, base, c);
    __syncthreads();
    // the thread's amplitudes i = tid + j blockDim in registers and the terms in the outer loop, so
    // each term's record is read once per tile; swz is linear, so a partner sits at swz(i) ^ swz(xl).
    // Every amplitude still sums its terms in term order, and the thread its amplitudes in index
    // order (the same bits as one amplitude at a time).
    const int nj = c.tile < (int)blockDim.x ? 1 : c.tile / (int)blockDim.x;
    const bool live0 = (int)threadIdx.x < c.tile;
    float tacc = 0.f;
    for (int j0 = 0; j0 < nj && live0; j0 += kRedGroup) {
      float2 v[kRedGroup];
      float nrm[kRedGroup], sacc[kRedGroup];
      int si[kRedGroup];
#pragma unroll
      for (int j = 0; j < kRedGroup; ++j) {
        const int i = threadIdx.x + (j0 + j) * blockDim.x;
        si[j] = swz(i);
        v[j] = (j0 + j < nj) ? sm[si[j]] : make_float2(0.f, 0.f);
        nrm[j] = fmaf(v[j].x, v[j].x, v[j].y * v[j].y);
        sacc[j] = 0.f;
      }
      for (int k = 0; k < nt; ++k) {
        const TermSm tm = st_terms[k];
        const float c0 = sb[k] ? -tm.coef : tm.coef;
        // parity of i & zl = bit J of tm.hi, flipped in every bit by this thread's part (bits 0..7)
        const int par = (tm.hi >> j0) ^ -(__popc((int)threadIdx.x & tm.zl & 0xFF) & 1);
        if (tm.xl == 0) {  // diagonal term (ny is even and i^ny = +-1)
#pragma unroll
          for (int j = 0; j < kRedGroup; ++j) sacc[j] = fmaf(((par >> j) & 1) ? -c0 : c0, nrm[j], sacc[j]);
          continue;
        }
        const int sx = swz(tm.xl);
#pragma unroll
        for (int j = 0; j < kRedGroup; ++j) {
          if (j0 + j >= nj) break;
          const float sgn = ((par >> j) & 1) ? -c0 : c0;
          const float2 w = sm[si[j] ^ sx];
          const float2 z = make_float2(fmaf(w.x, v[j].x, w.y * v[j].y), fmaf(w.x, v[j].y, -w.y * v[j].x));  // conj(w) v
          sacc[j] = fmaf(sgn, times_i_pow(z, tm.ny).x, sacc[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < kRedGroup; ++j)
        if (j0 + j < nj) tacc += sacc[j];
    }
    acc += (double)tacc;
    __syncthreads();
  }
  const double tot = block_sum(acc, scratch);
  if (threadIdx.x == 0) part[((long long)b * n_passes + pass_idx) * kRedMaxCTAs + blockIdx.x] = tot;
}

// out[b] = sum over passes and CTAs of the partials (fixed order).
__global__ void k_expect_final(const double *__restrict__ part, int n_passes, int gx, double *__restrict__ out) {
  __shared__ double scratch[kRedThreads / 32];
  const int b = blockIdx.x;
  double v = 0.0;
  for (int k = threadIdx.x; k < n_passes * gx; k += blockDim.x) {
    const int p = k / gx, x = k % gx;
    v += part[((long long)b * n_passes + p) * kRedMaxCTAs + x];
  }
  const double tot = block_sum(v, scratch);
  if (threadIdx.x == 0) out[b] = tot;
}

// lam (+)= (sum of the pass's terms) psi, lam[x] = sum_t c_t i^ny (-1)^popc((x^xm)&zm) psi[x^xm].
// With dot != NULL (the last pass) the CTA also sums Re conj(psi[x]) lam[x] over its amplitudes:
// <psi|H|psi> from the finished lam, in the precision steps of k_expect_pass (the product and a
// thread's sum over its amplitudes of one tile FP32, the rest FP64), into dot[b][blockIdx.x].
__global__ void __launch_bounds__(kRedThreads) k_hamiltonian_pass(const RedPass *__restrict__ passes, int pass_idx,
                                                                  const DevTerm *__restrict__ terms,
                                                                  const float2 *__restrict__ psi,
                                                                  float2 *__restrict__ lam, int N, int accumulate,
                                                                  double *__restrict__ dot) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RedPass rp;
  __shared__ double scratch[kRedThreads / 32];
  for (int i = threadIdx.x; i < (int)(sizeof(RedPass) / 4); i += blockDim.x)
    reinterpret_cast<int *>(&rp)[i] = reinterpret_cast<const int *>(passes + pass_idx)[i];
  __syncthreads();
  TileCtx c;
  float2 *sm = reinterpret_cast<float2 *>(smem_raw);
  long long *run_off = reinterpret_cast<long long *>(smem_raw + ((size_t)sizeof(float2) << rp.T));
  const int n_runs = (1 << (rp.T - (rp.T < kLowBits ? rp.T : kLowBits)));
  const int nt = rp.term_end - rp.term_begin;
  TermSm *st_terms = reinterpret_cast<TermSm *>(run_off + (n_runs < 2 ? 2 : n_runs));
  unsigned char *sb = reinterpret_cast<unsigned char *>(st_terms + nt);
  setup_tile(rp, run_off, c);
  for (int k = threadIdx.x; k < nt; k += blockDim.x) {
    const DevTerm &tm = terms[rp.term_begin + k];
    const int zl = compress_bits(tm.zm, rp);
    st_terms[k] = TermSm{(float)tm.coef, tm.xl, zl, tm.ny, row_parities(tm.xl, zl)};
  }
  __syncthreads();
  const int b = blockIdx.y;
  const float2 *st = psi + ((long long)b << N);
  float2 *lt = lam + ((long long)b << N);
  const long long n_tiles = 1ll << rp.n_outer;
  double acc = 0.0;
  for (long long t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const unsigned long long base = tile_base(rp, t);
    // parity of the Z mask on the outer bits; x ^ xm has the same outer bits as x
    for (int k = threadIdx.x; k < nt; k += blockDim.x)
      sb[k] = (unsigned char)(__popcll(base & terms[rp.term_begin + k].zm) & 1);
    load_tile(sm, st, base, c);
    __syncthreads();
    // as in k_expect_pass: the thread's amplitudes in registers, terms in the outer loop, every
    // amplitude summing its terms in term order (the same bits as one amplitude at a time)
    const int nj = c.tile < (int)blockDim.x ? 1 : c.tile / (int)blockDim.x;
    const bool live0 = (int)threadIdx.x < c.tile;
    float tacc = 0.f;
    for (int j0 = 0; j0 < nj && live0; j0 += kRedGroup) {
      float2 sacc[kRedGroup];
      int si[kRedGroup];
#pragma unroll
      for (int j = 0; j < kRedGroup; ++j) {
        const int i = threadIdx.x + (j0 + j) * blockDim.x;
        si[j] = swz(i);
        sacc[j] = make_float2(0.f, 0.f);
        if (j0 + j < nj && accumulate)
          sacc[j] = lt[base + (unsigned long long)c.run_off[i >> c.L] + (unsigned long long)(i & c.lowmask)];
      }
      for (int k = 0; k < nt; ++k) {
        const TermSm tm = st_terms[k];
        const float c0 = sb[k] ? -tm.coef : tm.coef;
        const int sx = swz(tm.xl);
        // parity of (i ^ xl) & zl = bit J of tm.hi, flipped in every bit by this thread's part (bits 0..7)
        const int par = (tm.hi >> j0) ^ -(__popc(((int)threadIdx.x ^ tm.xl) & tm.zl & 0xFF) & 1);
#pragma unroll
        for (int j = 0; j < kRedGroup; ++j) {
          if (j0 + j >= nj) break;
          const float sgn = ((par >> j) & 1) ? -c0 : c0;
          const float2 w = times_i_pow(sm[si[j] ^ sx], tm.ny);
          sacc[j].x = fmaf(sgn, w.x, sacc[j].x);
          sacc[j].y = fmaf(sgn, w.y, sacc[j].y);
        }
      }
#pragma unroll
      for (int j = 0; j < kRedGroup; ++j) {
        if (j0 + j >= nj) break;
        const int i = threadIdx.x + (j0 + j) * blockDim.x;
        lt[base + (unsigned long long)c.run_off[i >> c.L] + (unsigned long long)(i & c.lowmask)] = sacc[j];
        if (dot) {
          const float2 v = sm[si[j]];
          tacc = fmaf(v.x, sacc[j].x, fmaf(v.y, sacc[j].y, tacc));
        }
      }
    }
    acc += (double)tacc;
    __syncthreads();
  }
  if (dot) {
    const double tot = block_sum(acc, scratch);
    if (threadIdx.x == 0) dot[(long long)b * kRedMaxCTAs + blockIdx.x] = tot;
  }
}

namespace {
size_t red_smem(const RedPass &rp) {
  const int T = rp.T;
  const int L = T < kLowBits ? T : kLowBits;
  const size_t runs = ((size_t)1 << (T - L)) < 2 ? 2 : ((size_t)1 << (T - L));
  const size_t nt = (size_t)(rp.term_end - rp.term_begin);
  return ((size_t)1 << T) * sizeof(float2) + runs * sizeof(long long) + nt * sizeof(TermSm) + ((nt + 15) & ~(size_t)15);
}
int red_grid_x(const tn_observable *o, int pass, int batch, const void *fn) {
  const RedPass &rp = o->passes[pass];
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kRedThreads, red_smem(rp)) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  long long gx = ((long long)num_sms() * per_sm + batch - 1) / batch;
  const long long n_tiles = 1ll << rp.n_outer;
  if (gx > n_tiles) gx = n_tiles;
  if (gx > kRedMaxCTAs) gx = kRedMaxCTAs;
  if (gx < 1) gx = 1;
  return (int)gx;
}
}  // namespace

size_t observable_partials(const tn_observable *o, int batch) {
  return (size_t)batch * o->passes.size() * kRedMaxCTAs;
}

cudaError_t launch_expectation(const tn_observable *o, int batch, const float2 *state, double *part, double *out,
                               cudaStream_t s) {
  const int np = (int)o->passes.size();
  if (np == 0) return cudaMemsetAsync(out, 0, sizeof(double) * batch, s);
  int gx_max = 1;
  for (int p = 0; p < np; ++p) {
    const size_t smem = red_smem(o->passes[p]);
    cudaError_t e = ensure_smem((const void *)k_expect_pass, smem);
    if (e != cudaSuccess) return e;
    const int gx = red_grid_x(o, p, batch, (const void *)k_expect_pass);
    gx_max = gx > gx_max ? gx : gx_max;
  }
  // passes with a smaller grid leave zero partials below gx_max (the final sum reads gx_max per pass)
  cudaError_t e = cudaMemsetAsync(part, 0, observable_partials(o, batch) * sizeof(double), s);
  if (e != cudaSuccess) return e;
  for (int p = 0; p < np; ++p) {
    const int gx = red_grid_x(o, p, batch, (const void *)k_expect_pass);
    dim3 grid((unsigned)gx, (unsigned)batch);
    k_expect_pass<<<grid, kRedThreads, red_smem(o->passes[p]), s>>>(o->d_passes, p, np, o->d_terms, state, o->n,
                                                                     part);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_expect_final<<<batch, kRedThreads, 0, s>>>(part, np, gx_max, out);
  return cudaGetLastError();
}

cudaError_t launch_apply_hamiltonian(const tn_observable *o, int batch, const float2 *psi, float2 *lam,
                                     cudaStream_t s, double *part, double *out) {
  const int np = (int)o->passes.size();
  if (np == 0) {
    cudaError_t e = cudaMemsetAsync(lam, 0, (sizeof(float2) << o->n) * batch, s);
    if (e == cudaSuccess && out) e = cudaMemsetAsync(out, 0, sizeof(double) * batch, s);
    return e;
  }
  int gx_last = 1;
  for (int p = 0; p < np; ++p) {
    const size_t smem = red_smem(o->passes[p]);
    cudaError_t e = ensure_smem((const void *)k_hamiltonian_pass, smem);
    if (e != cudaSuccess) return e;
    const int gx = red_grid_x(o, p, batch, (const void *)k_hamiltonian_pass);
    double *dot = (out && p == np - 1) ? part : nullptr;
    dim3 grid((unsigned)gx, (unsigned)batch);
    k_hamiltonian_pass<<<grid, kRedThreads, smem, s>>>(o->d_passes, p, o->d_terms, psi, lam, o->n, p > 0 ? 1 : 0,
                                                       dot);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    gx_last = gx;
  }
  if (out) {  // every CTA of the last pass wrote its partial: no clearing needed
    k_expect_final<<<batch, kRedThreads, 0, s>>>(part, 1, gx_last, out);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

}  // namespace tnq
