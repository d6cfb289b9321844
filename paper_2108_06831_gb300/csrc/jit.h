// Plan-specialised gate-apply kernels (generated CUDA C++, compiled with NVRTC).
#pragma once

#include <string>
#include <vector>

#include "tnq_internal.h"

namespace tnq {
// Whether every forward (adjoint) pass of the plan has the shape the generator handles.
bool jit_supported(const tn_plan &p);
bool jit_bwd_supported(const tn_plan &p);
// Generate, compile (or fetch from the cache) and load the plan's forward or adjoint pass
// kernels.  op_kind[o] is the gate kind of op o of that direction.  compile_only: stop
// after compiling (no GPU needed).
tn_status jit_build(tn_plan &p, const std::vector<int> &op_kind, bool backward, bool compile_only, std::string &err);
void jit_release(tn_plan &p);
// Whether the forward pass kernels read their matrix entries from per-pass __constant__ tables
// (fixed angles, or batch 1); the host copies each pass's entries there before it runs.
bool jit_const_mats(const tn_plan &p);
}  // namespace tnq
