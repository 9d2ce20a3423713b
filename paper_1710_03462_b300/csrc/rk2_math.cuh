// Selects the per-particle step implementation used by every kernel.
#pragma once
#include "rk2_native.cuh"

namespace soax {
__device__ __forceinline__ void rk2_step(const FlowK& f, double inv_tau, double x[3], float v[3],
                                         float a2out[3]) {
  rk2_step_native(f, inv_tau, x, v, a2out);
}
}  // namespace soax
