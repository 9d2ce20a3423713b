// Selects the per-particle step implementation used by every kernel: the float-float
// evaluation of rk2_fast.cuh (binary64 accuracy off the FP64 pipe).
#pragma once
#include "rk2_fast.cuh"

namespace soax {
// One particle, either path (see near_shift).
template <bool ACC, class Trig>
__device__ __forceinline__ void rk2_step(const StepC& k, const Trig& trig, double x[3], float v[3], float a2out[3]) {
  rk2_step_fast<ACC, false>(k, trig, x, v, a2out);
}
}  // namespace soax
