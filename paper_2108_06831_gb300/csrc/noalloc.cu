// tn_state_expectation_noalloc: the Pauli-sum reduction of tn_state_expectation with its
// scratch in a fixed array compiled into this library instead of a caller-supplied
// workspace.
//
// Some callers cannot hand the library a workspace: their device memory is owned by
// another allocator with a fixed budget (a framework's caching pool that must see every
// allocation), or they run on a path where a cudaMalloc would implicitly synchronise the
// device and stall unrelated streams.  For them this entry point takes only the state and
// the output; the per-CTA partial sums live in g_noalloc_partials below.
//
// Consequences a caller must know:
//   - the array holds kNoAllocPartials doubles (1 MiB) on every GPU that loads the library,
//     for the life of the process; a request whose partials (batch x reduction passes x 512)
//     would not fit is rejected with TN_ERR_INVALID_ARG;
//   - every call on a device uses the same array, and it keeps the previous call's contents:
//     the reduction clears the slots it reads before writing them, but two calls that overlap
//     on the GPU (different streams, no ordering between them) race on the array;
//   - every call looks up the array's device address with cudaGetSymbolAddress on the
//     current device (a host-side lookup; nothing is cached, so an address stays right after
//     cudaDeviceReset rebuilds the context).  The first lookup on a device loads the module
//     there, so make the first call on each device before any stream capture begins.

#include "kernels.h"
#include "tnq_internal.h"

namespace tnq {

constexpr size_t kNoAllocPartials = 131072;  // doubles: 1 MiB of device memory per GPU

static __device__ __align__(256) double g_noalloc_partials[kNoAllocPartials];

namespace {
// Device address of g_noalloc_partials in the current device's context.  In host code the
// symbol's name stands for a host-side shadow, so the address must come from the runtime.
tn_status noalloc_scratch(double **out) {
  double *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_partials);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the built-in scratch array");
  *out = p;
  return TN_OK;
}
}  // namespace

}  // namespace tnq

using namespace tnq;

extern "C" tn_status tn_state_expectation_noalloc(const tn_observable *H, int32_t batch, const void *state_dev,
                                                  double *out_dev, tn_stream_t s) {
  if (H == nullptr || state_dev == nullptr || out_dev == nullptr) {
    set_error("NULL argument");
    return TN_ERR_INVALID_ARG;
  }
  if (batch < 1) {
    set_error("batch < 1");
    return TN_ERR_INVALID_ARG;
  }
  if (((uintptr_t)state_dev & 15) != 0) {
    set_error("state_dev must be 16-byte aligned");
    return TN_ERR_INVALID_ARG;
  }
  const size_t need = observable_partials(H, batch);
  if (need > kNoAllocPartials) {
    set_error("tn_state_expectation_noalloc: batch %d x %zu reduction passes needs %zu partial sums, more than the "
              "%zu the built-in scratch holds; use tn_state_expectation with a workspace",
              batch, H->passes.size(), need, kNoAllocPartials);
    return TN_ERR_INVALID_ARG;
  }
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (cur != H->device) {
    set_error("observable was built on device %d but device %d is current", H->device, cur);
    return TN_ERR_INVALID_ARG;
  }
  double *scratch = nullptr;
  tn_status st = noalloc_scratch(&scratch);
  if (st != TN_OK) return st;
  e = launch_expectation(H, batch, static_cast<const float2 *>(state_dev), scratch, out_dev,
                         reinterpret_cast<cudaStream_t>(s));
  if (e != cudaSuccess) return cuda_fail(e, "expectation kernel");
  return TN_OK;
}
