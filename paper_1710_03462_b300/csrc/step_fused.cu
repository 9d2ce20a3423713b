// soax_step_fused: nsteps midpoint-RK2 steps per particle in one pass over the planes.
#include <mutex>

#include "soax_internal.h"
#include "step_fused.cuh"

namespace soax {

float2 split_ff(double d);

// Launch shape, picked by timing shapes on 16.7M particles x 10 steps.
constexpr int kFusedPPT = 1;
constexpr int kFusedBlock = 512;
constexpr int kFusedMinBlocks = 2;

using FusedKernel = void (*)(EnsArgs, FlowK, TurnsK, int);

// The kernel for a tau field (TAU) and an acceleration field (ACC).
static FusedKernel fused_kernel(bool tau, bool acc) {
  if (tau)
    return acc ? k_step_soa_fused<kFusedPPT, kFusedBlock, kFusedMinBlocks, true, true>
               : k_step_soa_fused<kFusedPPT, kFusedBlock, kFusedMinBlocks, true, false>;
  return acc ? k_step_soa_fused<kFusedPPT, kFusedBlock, kFusedMinBlocks, false, true>
             : k_step_soa_fused<kFusedPPT, kFusedBlock, kFusedMinBlocks, false, false>;
}

// Dynamic shared memory above 48 KB and the largest carveout for the four kernels, set
// once per device.
static int prepare_fused_kernels() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return cuda_fail(cudaGetLastError(), "soax_step_fused: device");
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return SOAX_OK;
  for (int v = 0; v < 4; ++v) {
    const void* fn = (const void*)fused_kernel(v & 1, v & 2);
    cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kScaledTrigBytes);
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (err != cudaSuccess) return cuda_fail(err, "soax_step_fused: kernel attributes");
  }
  done[dev] = true;
  return SOAX_OK;
}

TurnsK make_turns_k(double dt) {
  const double turn32 = 4294967296.0 / SOAX_TWO_PI_HOST;  // 2^32 / 2pi
  TurnsK t;
  const float2 a = split_ff(dt * turn32), b = split_ff(0.5 * dt * turn32);
  t.dtT = ff{a.x, a.y};
  t.hdtT = ff{b.x, b.y};
  return t;
}

}  // namespace soax

using namespace soax;

extern "C" int soax_step_fused(soax_t h, const soax_flow* fl, int32_t nsteps, void* stream) {
  if (int r = check_handle(h)) return r;
  if (nsteps < 0) return fail(SOAX_EINVAL, "soax_step_fused: nsteps < 0");
  EnsArgs e;
  FlowK f;
  if (int r = make_ens_args(h, fl, h->current, &e, &f, "soax_step_fused")) return r;
  if (h->n == 0 || nsteps == 0) return SOAX_OK;
  if (int r = prepare_fused_kernels()) return r;
  const FusedKernel kern = fused_kernel(e.tau_src != nullptr, e.ax != nullptr);
  const int grid = persistent_grid((const void*)kern, kFusedBlock, kScaledTrigBytes,
                                   grid_for((h->n + kFusedPPT - 1) / kFusedPPT, kFusedBlock));
  kern<<<grid, kFusedBlock, kScaledTrigBytes, as_stream(stream)>>>(e, f, make_turns_k(fl->dt), nsteps);
  return check_launch("soax_step_fused");
}
