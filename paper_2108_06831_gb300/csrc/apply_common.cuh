// Device helpers of the fused gate-apply kernels (forward and adjoint).
//
// A tile of 2^T complex64 amplitudes lives in shared memory.  Tile index i is stored at
// position swz(i) = i ^ fold(i >> 4), where fold XORs the 4-bit groups of its argument:
// the map is GF(2)-linear, so swz(a | b) = swz(a) ^ swz(b) for disjoint a, b, and a
// warp whose 32 lanes vary five index bits whose positions cover every residue mod 4
// touches each pair of 4-byte banks exactly twice (two wavefronts, no conflict).
#pragma once

#include "tnq_internal.h"

namespace tnq {

__device__ __forceinline__ int swz(int i) {
  int h = i >> 4;
  h ^= h >> 4;
  h ^= h >> 8;
  return i ^ (h & 15);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a*x + b*y
__device__ __forceinline__ float2 cmul2(float2 a, float2 x, float2 b, float2 y) {
  float re = a.x * x.x;
  re = fmaf(-a.y, x.y, re);
  re = fmaf(b.x, y.x, re);
  re = fmaf(-b.y, y.y, re);
  float im = a.x * x.y;
  im = fmaf(a.y, x.x, im);
  im = fmaf(b.x, y.y, im);
  im = fmaf(b.y, y.x, im);
  return make_float2(re, im);
}
__device__ __forceinline__ float2 cneg_if(float2 a, uint32_t flip) {
  const uint32_t s = flip << 31;
  return make_float2(__uint_as_float(__float_as_uint(a.x) ^ s), __uint_as_float(__float_as_uint(a.y) ^ s));
}
__device__ __forceinline__ float2 csel(bool p, float2 a, float2 b) { return p ? a : b; }

// Op records and matrix entries may live in global or (staged) shared memory: generic loads.
__device__ __forceinline__ float2 ldg_c(const float2 *p) { return *p; }
__device__ __forceinline__ float4 ld4(const float2 *p) { return *reinterpret_cast<const float4 *>(p); }

// Bit r of every register index j < 2^K, as a mask over j.
__device__ __forceinline__ uint32_t reg_bit_mask(int r) {
  switch (r) {
    case 0: return 0xAAAAAAAAu;
    case 1: return 0xCCCCCCCCu;
    case 2: return 0xF0F0F0F0u;
    case 3: return 0xFF00FF00u;
    default: return 0xFFFF0000u;
  }
}

// Per-thread context of one phase: where a bit operand's value comes from.
struct BitCtx {
  int tb;                  // thread's tile-local base index (thread-index bits deposited)
  unsigned long long base; // tile's global base offset (outer bits)
  uint32_t full;           // mask of all 2^K register indices
};

// Mask over the thread's register indices where the bit operand (kind, pos) is 1.
__device__ __forceinline__ uint32_t src_mask(const BitCtx &c, int kind, int pos) {
  if (kind == SRC_REG) return reg_bit_mask(pos) & c.full;
  int v = (kind == SRC_TILE) ? ((c.tb >> pos) & 1) : (int)((c.base >> pos) & 1ull);
  return v ? c.full : 0u;
}

// 2x2 u on register bit R for the pairs whose lower member j has (pred >> j) & 1.
template <int K, int R, bool PRED>
__device__ __forceinline__ void reg_g1(float2 (&a)[1 << K], float2 u00, float2 u01, float2 u10, float2 u11,
                                       uint32_t pred) {
#pragma unroll
  for (int j = 0; j < (1 << K); ++j) {
    if (j & (1 << R)) continue;
    const int j1 = j | (1 << R);
    const float2 x = a[j], y = a[j1];
    const float2 nx = cmul2(u00, x, u01, y);
    const float2 ny = cmul2(u10, x, u11, y);
    if (PRED) {
      const bool p = (pred >> j) & 1u;
      a[j] = csel(p, nx, x);
      a[j1] = csel(p, ny, y);
    } else {
      a[j] = nx;
      a[j1] = ny;
    }
  }
}

template <int K, bool PRED>
__device__ __forceinline__ void reg_g1_dispatch(float2 (&a)[1 << K], int r, const float2 *m, uint32_t pred) {
  const float4 m01 = ld4(m);
  const float4 m23 = ld4(m + 2);
  const float2 u00 = make_float2(m01.x, m01.y), u01 = make_float2(m01.z, m01.w);
  const float2 u10 = make_float2(m23.x, m23.y), u11 = make_float2(m23.z, m23.w);
  switch (r) {
    case 0: reg_g1<K, 0, PRED>(a, u00, u01, u10, u11, pred); break;
    case 1: if constexpr (K > 1) reg_g1<K, 1, PRED>(a, u00, u01, u10, u11, pred); break;
    case 2: if constexpr (K > 2) reg_g1<K, 2, PRED>(a, u00, u01, u10, u11, pred); break;
    case 3: if constexpr (K > 3) reg_g1<K, 3, PRED>(a, u00, u01, u10, u11, pred); break;
    case 4: if constexpr (K > 4) reg_g1<K, 4, PRED>(a, u00, u01, u10, u11, pred); break;
  }
}

// 4x4 u on register bits (RA = high bit of the 4x4 index, RB = low bit).
template <int K, int RA, int RB>
__device__ __forceinline__ void reg_g2(float2 (&a)[1 << K], const float2 (&u)[16]) {
#pragma unroll
  for (int j = 0; j < (1 << K); ++j) {
    if (j & ((1 << RA) | (1 << RB))) continue;
    const int i0 = j, i1 = j | (1 << RB), i2 = j | (1 << RA), i3 = j | (1 << RA) | (1 << RB);
    const float2 v0 = a[i0], v1 = a[i1], v2 = a[i2], v3 = a[i3];
    float2 o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float2 s = cmul2(u[4 * k + 0], v0, u[4 * k + 1], v1);
      const float2 t = cmul2(u[4 * k + 2], v2, u[4 * k + 3], v3);
      o[k] = make_float2(s.x + t.x, s.y + t.y);
    }
    a[i0] = o[0];
    a[i1] = o[1];
    a[i2] = o[2];
    a[i3] = o[3];
  }
}

template <int K, int RA>
__device__ __forceinline__ void reg_g2_b(float2 (&a)[1 << K], int rb, const float2 (&u)[16]) {
  switch (rb) {
    case 0: if constexpr (RA != 0) reg_g2<K, RA, 0>(a, u); break;
    case 1: if constexpr (K > 1 && RA != 1) reg_g2<K, RA, 1>(a, u); break;
    case 2: if constexpr (K > 2 && RA != 2) reg_g2<K, RA, 2>(a, u); break;
    case 3: if constexpr (K > 3 && RA != 3) reg_g2<K, RA, 3>(a, u); break;
    case 4: if constexpr (K > 4 && RA != 4) reg_g2<K, RA, 4>(a, u); break;
  }
}

template <int K>
__device__ __forceinline__ void reg_g2_dispatch(float2 (&a)[1 << K], int ra, int rb, const float2 *m, bool packed) {
  if constexpr (K >= 2) {
    float2 u[16];
    if (packed) {  // SHAPE_M4X: entry k is (re, re, -im, im)
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float4 v = ld4(m + 2 * k);
        u[k] = make_float2(v.x, v.w);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float4 v = ld4(m + 2 * k);
        u[2 * k] = make_float2(v.x, v.y);
        u[2 * k + 1] = make_float2(v.z, v.w);
      }
    }
    switch (ra) {
      case 0: reg_g2_b<K, 0>(a, rb, u); break;
      case 1: reg_g2_b<K, 1>(a, rb, u); break;
      case 2: if constexpr (K > 2) reg_g2_b<K, 2>(a, rb, u); break;
      case 3: if constexpr (K > 3) reg_g2_b<K, 3>(a, rb, u); break;
      case 4: if constexpr (K > 4) reg_g2_b<K, 4>(a, rb, u); break;
    }
  }
}

// SWAP of register bits RA and RB: exchange the amplitudes whose two bits differ.
template <int K, int RA, int RB>
__device__ __forceinline__ void reg_swap(float2 (&a)[1 << K]) {
#pragma unroll
  for (int j = 0; j < (1 << K); ++j)
    if ((j & (1 << RA)) && !(j & (1 << RB))) {
      const int j2 = (j & ~(1 << RA)) | (1 << RB);
      const float2 t = a[j];
      a[j] = a[j2];
      a[j2] = t;
    }
}
template <int K, int RA>
__device__ __forceinline__ void reg_swap_b(float2 (&a)[1 << K], int rb) {
  switch (rb) {
    case 0: if constexpr (RA != 0) reg_swap<K, RA, 0>(a); break;
    case 1: if constexpr (K > 1 && RA != 1) reg_swap<K, RA, 1>(a); break;
    case 2: if constexpr (K > 2 && RA != 2) reg_swap<K, RA, 2>(a); break;
    case 3: if constexpr (K > 3 && RA != 3) reg_swap<K, RA, 3>(a); break;
    case 4: if constexpr (K > 4 && RA != 4) reg_swap<K, RA, 4>(a); break;
  }
}
template <int K>
__device__ __forceinline__ void reg_swap_dispatch(float2 (&a)[1 << K], int ra, int rb) {
  if constexpr (K >= 2) {
    switch (ra) {
      case 0: reg_swap_b<K, 0>(a, rb); break;
      case 1: reg_swap_b<K, 1>(a, rb); break;
      case 2: if constexpr (K > 2) reg_swap_b<K, 2>(a, rb); break;
      case 3: if constexpr (K > 3) reg_swap_b<K, 3>(a, rb); break;
      case 4: if constexpr (K > 4) reg_swap_b<K, 4>(a, rb); break;
    }
  }
}

// diag(d0, d1) selected by mask m (1 -> d1).
template <int K>
__device__ __forceinline__ void reg_diag(float2 (&a)[1 << K], uint32_t m, float2 d0, float2 d1) {
#pragma unroll
  for (int j = 0; j < (1 << K); ++j) a[j] = cmul(a[j], csel((m >> j) & 1u, d1, d0));
}
// phase e on the indices in mask m.
template <int K>
__device__ __forceinline__ void reg_phase(float2 (&a)[1 << K], uint32_t m, float2 e) {
#pragma unroll
  for (int j = 0; j < (1 << K); ++j) a[j] = csel((m >> j) & 1u, cmul(a[j], e), a[j]);
}
template <int K>
__device__ __forceinline__ void reg_flush_sign(float2 (&a)[1 << K], uint32_t neg) {
#pragma unroll
  for (int j = 0; j < (1 << K); ++j) a[j] = cneg_if(a[j], (neg >> j) & 1u);
}

// Apply one op to the registers.  Sign flips of CZ ops accumulate in neg and are applied
// lazily: they commute with every diagonal op and with every op whose register bits they do
// not depend on; the planner sets OPF_FLUSH on the ops where that is not the case.  A SWAP is a
// register exchange; SWAP_REGS = false applies it as the dense 4x4 permutation instead (one code
// path for every two-qubit op, for kernels whose register budget the exchange code would exceed).
template <int K, bool SWAP_REGS = true>
__device__ __forceinline__ void apply_op(float2 (&a)[1 << K], const OpDesc &op, const BitCtx &c,
                                         const float2 *mats, uint32_t &neg) {
  switch (op.type) {
    case OP_G1:
      if (op.flags & OPF_FLUSH) {
        if (neg) reg_flush_sign<K>(a, neg);
        neg = 0;
      }
      reg_g1_dispatch<K, false>(a, op.a_pos, mats + op.mat, 0u);
      break;
    case OP_C1: {
      if (op.flags & OPF_FLUSH) {
        if (neg) reg_flush_sign<K>(a, neg);
        neg = 0;
      }
      const uint32_t pm = src_mask(c, op.a_kind, op.a_pos);
      if (pm == c.full) reg_g1_dispatch<K, false>(a, op.b_pos, mats + op.mat, 0u);
      else if (pm != 0u) reg_g1_dispatch<K, true>(a, op.b_pos, mats + op.mat, pm);
      break;
    }
    case OP_G2:
      if (op.flags & OPF_FLUSH) {
        if (neg) reg_flush_sign<K>(a, neg);
        neg = 0;
      }
      if (SWAP_REGS && (op.flags & OPF_SWAP)) reg_swap_dispatch<K>(a, op.a_pos, op.b_pos);
      else reg_g2_dispatch<K>(a, op.a_pos, op.b_pos, mats + op.mat, (op.flags & OPF_PACKED) != 0);
      break;
    case OP_D1: {
      const float4 d = ld4(mats + op.mat);
      reg_diag<K>(a, src_mask(c, op.a_kind, op.a_pos), make_float2(d.x, d.y), make_float2(d.z, d.w));
      break;
    }
    case OP_CZ:
      neg ^= src_mask(c, op.a_kind, op.a_pos) & src_mask(c, op.b_kind, op.b_pos);
      break;
    case OP_DP: {
      const uint32_t m = src_mask(c, op.a_kind, op.a_pos) & src_mask(c, op.b_kind, op.b_pos);
      if (m) reg_phase<K>(a, m, ldg_c(mats + op.mat));
      break;
    }
  }
}

// Copy n 16-byte records (n4 int4 words) from global to shared memory, all threads.
__device__ __forceinline__ void stage_int4(int4 *dst, const int4 *src, int n4) {
  for (int i = threadIdx.x; i < n4; i += blockDim.x) dst[i] = __ldg(src + i);
}

// Deposit the low bits of v into the tile positions pos[0..n).
__device__ __forceinline__ int deposit(int v, const uint8_t *pos, int n) {
  int r = 0;
  for (int j = 0; j < n; ++j) r |= ((v >> j) & 1) << pos[j];
  return r;
}

}  // namespace tnq
