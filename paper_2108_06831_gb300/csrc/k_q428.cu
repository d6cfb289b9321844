// Fixed-point emulation of the paper's datapath (Sec. 3: complex arithmetic in 32-bit fixed
// point with 28 bits behind the binary point, Q4.28).
//
// The state is int32 pairs (re, im) with value q / 2^28.  Every gate is quantised once,
// Uq = round(U 2^28), and applied once: each output component is the exact sum of the
// integer products (64-bit; for unitary gates on states of norm <= 1 every sum stays below
// 2^60) rounded back to Q4.28, round half up ((acc + 2^27) >> 28, an arithmetic shift), and
// saturated to the int32 range.  One launch per gate: every amplitude is read and written
// once (16 bytes), so a gate is an HBM-bound pass over the state; integer sums are exact in
// any order, so the result is bit-for-bit reproducible.
#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "kernels.h"
#include "tnq_internal.h"

namespace tnq {

namespace {

struct Q428U2 {
  int32_t u[8];  // 2x2, row-major, (re, im) interleaved
};
struct Q428U4 {
  int32_t u[32];  // 4x4
};

__device__ __forceinline__ int32_t q_round(long long acc) {
  const long long r = (acc + (1ll << 27)) >> 28;
  return (int32_t)(r > INT_MAX ? (long long)INT_MAX : (r < INT_MIN ? (long long)INT_MIN : r));
}

// (a + ib) (c + id) accumulated into (re, im), exactly
__device__ __forceinline__ void cmac(long long &re, long long &im, int32_t ur, int32_t ui, int2 v) {
  re += (long long)ur * v.x - (long long)ui * v.y;
  im += (long long)ur * v.y + (long long)ui * v.x;
}

// Insert a zero bit at position p of j.
__device__ __forceinline__ long long insert0(long long j, int p) {
  return ((j >> p) << (p + 1)) | (j & ((1ll << p) - 1));
}

__global__ void k_q428_g1(int2 *__restrict__ st, long long pairs, int p, const __grid_constant__ Q428U2 g) {
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < pairs; j += (long long)gridDim.x * blockDim.x) {
    const long long i0 = insert0(j, p), i1 = i0 | (1ll << p);
    const int2 a = st[i0], b = st[i1];
    long long r0 = 0, m0 = 0, r1 = 0, m1 = 0;
    cmac(r0, m0, g.u[0], g.u[1], a);
    cmac(r0, m0, g.u[2], g.u[3], b);
    cmac(r1, m1, g.u[4], g.u[5], a);
    cmac(r1, m1, g.u[6], g.u[7], b);
    st[i0] = make_int2(q_round(r0), q_round(m0));
    st[i1] = make_int2(q_round(r1), q_round(m1));
  }
}

// pa: bit of the first qubit (high bit of the 4x4 index), pb: the second's
__global__ void k_q428_g2(int2 *__restrict__ st, long long quads, int pa, int pb, const __grid_constant__ Q428U4 g) {
  const int lo = pa < pb ? pa : pb, hi = pa < pb ? pb : pa;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < quads; j += (long long)gridDim.x * blockDim.x) {
    const long long i00 = insert0(insert0(j, lo), hi);
    long long idx[4];
    idx[0] = i00;
    idx[1] = i00 | (1ll << pb);
    idx[2] = i00 | (1ll << pa);
    idx[3] = i00 | (1ll << pa) | (1ll << pb);
    int2 v[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) v[m] = st[idx[m]];
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      long long re = 0, im = 0;
#pragma unroll
      for (int m = 0; m < 4; ++m) cmac(re, im, g.u[2 * (4 * l + m)], g.u[2 * (4 * l + m) + 1], v[m]);
      st[idx[l]] = make_int2(q_round(re), q_round(im));
    }
  }
}

__global__ void k_q428_basis(int2 *__restrict__ st, long long n_amps, unsigned long long init) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_amps; i += (long long)gridDim.x * blockDim.x)
    st[i] = make_int2(i == (long long)init ? (1 << 28) : 0, 0);
}

unsigned grid_for(long long items) {
  return (unsigned)std::max<long long>(1, std::min<long long>((items + 255) / 256, 152ll * 16));
}

}  // namespace

int32_t q428_quantize(double x) {
  const double r = std::floor(x * 268435456.0 + 0.5);  // x 2^28, round half up (exact for |x| < 2^24)
  return (int32_t)std::max(std::min(r, (double)INT_MAX), (double)INT_MIN);
}

void q428_build(const tn_circuit &c, std::vector<Q428Gate> &out) {
  out.clear();
  for (const TnGate &g : c.gates) {
    double m[32];
    const int dim = gate_matrix(g.kind, FORM_U, g.angle, g.mat, m);
    Q428Gate q;
    q.nq = dim == 2 ? 1 : 2;
    q.pos[0] = c.n - 1 - g.q[0];
    q.pos[1] = q.nq == 2 ? c.n - 1 - g.q[1] : -1;
    for (int i = 0; i < 2 * dim * dim; ++i) q.u[i] = q428_quantize(m[i]);
    out.push_back(q);
  }
}

cudaError_t launch_q428(const std::vector<Q428Gate> &gates, int n, unsigned long long init, int32_t *state,
                        cudaStream_t s) {
  int2 *st = reinterpret_cast<int2 *>(state);
  const long long amps = 1ll << n;
  k_q428_basis<<<grid_for(amps), 256, 0, s>>>(st, amps, init);
  cudaError_t e = cudaGetLastError();
  for (size_t k = 0; e == cudaSuccess && k < gates.size(); ++k) {
    const Q428Gate &q = gates[k];
    if (q.nq == 1) {
      Q428U2 g;
      std::copy(q.u, q.u + 8, g.u);
      k_q428_g1<<<grid_for(amps / 2), 256, 0, s>>>(st, amps / 2, q.pos[0], g);
    } else {
      Q428U4 g;
      std::copy(q.u, q.u + 32, g.u);
      k_q428_g2<<<grid_for(amps / 4), 256, 0, s>>>(st, amps / 4, q.pos[0], q.pos[1], g);
    }
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace tnq
