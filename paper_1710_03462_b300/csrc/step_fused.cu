// soax_step_fused: nsteps midpoint-RK2 steps per particle in one pass over the planes.
#include <mutex>

#include "soax_internal.h"
#include "step_fused.cuh"

namespace soax {

float2 split_ff(double d);
CellKeyK make_cell_key_k(int grid);

// Launch shape, picked by timing shapes on 16.7M particles x 10 steps.
constexpr int kFusedPPT = 1;
constexpr int kFusedBlock = 512;
constexpr int kFusedMinBlocks = 2;

using FusedKernel = void (*)(EnsArgs, FlowK, TurnsK, int, uint32_t*, CellKeyK);

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

static int step_fused(soax_t h, const soax_flow* fl, int32_t nsteps, int32_t grid, uint32_t* keys, void* stream,
                      const char* who) {
  if (int r = check_handle(h)) return r;
  if (nsteps < 0) return fail(SOAX_EINVAL, std::string(who) + ": nsteps < 0");
  EnsArgs e;
  FlowK f;
  if (int r = make_ens_args(h, fl, h->current, &e, &f, who)) return r;
  CellKeyK ck{};
  if (grid) {
    if (grid < 1 || grid > 1024) return fail(SOAX_EINVAL, std::string(who) + ": grid must be in 1..1024");
    if (h->n > 0 && !keys) return fail(SOAX_EINVAL, std::string(who) + ": keys is NULL");
    if (!aligned16(keys)) return fail(SOAX_EALIGN, std::string(who) + ": keys not 16-byte aligned");
    ck = make_cell_key_k(grid);
  }
  if (h->n == 0) return SOAX_OK;
  if (nsteps == 0) return grid ? soax_cell_keys(h, fl->pos_field, grid, keys, stream) : SOAX_OK;
  if (int r = prepare_fused_kernels()) return r;
  const FusedKernel kern = fused_kernel(e.tau_src != nullptr, e.ax != nullptr);
  const int gsz = persistent_grid((const void*)kern, kFusedBlock, kScaledTrigBytes,
                                  grid_for((h->n + kFusedPPT - 1) / kFusedPPT, kFusedBlock));
  kern<<<gsz, kFusedBlock, kScaledTrigBytes, as_stream(stream)>>>(e, f, make_turns_k(fl->dt), nsteps,
                                                                   grid ? keys : nullptr, ck);
  return check_launch(who);
}

}  // namespace soax

extern "C" int soax_step_fused(soax_t h, const soax_flow* fl, int32_t nsteps, void* stream) {
  return soax::step_fused(h, fl, nsteps, 0, nullptr, stream, "soax_step_fused");
}

extern "C" int soax_step_fused_keys(soax_t h, const soax_flow* fl, int32_t nsteps, int32_t grid, uint32_t* keys,
                                    void* stream) {
  if (grid == 0) return soax::fail(SOAX_EINVAL, "soax_step_fused_keys: grid must be in 1..1024");
  return soax::step_fused(h, fl, nsteps, grid, keys, stream, "soax_step_fused_keys");
}
