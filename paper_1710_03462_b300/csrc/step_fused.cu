// soax_step_fused: nsteps midpoint-RK2 steps per particle in one pass over the planes.
#include <cmath>
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

// umax: a bound of |u_c| for every particle of the launch (the largest sum of two
// amplitudes), used by fast_positions.
TurnsK make_turns_k(double dt, double umax) {
  const double turn32 = 4294967296.0 / SOAX_TWO_PI_HOST;  // 2^32 / 2pi
  TurnsK t;
  const float2 a = split_ff(dt * turn32), b = split_ff(0.5 * dt * turn32);
  t.dtT = ff{a.x, a.y};
  t.hdtT = ff{b.x, b.y};
  t.umax = (float)(umax * (1.0 + 1e-6));
  t.vsafe = -1.0f;
  return t;
}

double amplitude_bound(const soax_flow* fl) {
  const double a = std::fabs(fl->A), b = std::fabs(fl->B), c = std::fabs(fl->C);
  return std::fmax(a + c, std::fmax(b + a, c + b));
}

// The turns constants of a call of nsteps steps, with vsafe (TurnsK) when tau is uniform.
// One step gives
//   v' = v (1 - h + h^2/2) + h u(xm) - (h^2/2) u(x),   h = dt/tau,
// so with |v_c| <= M and |u_c| <= umax <= M every component obeys |v'_c| <= M (1 + h^2)
// (1 - h + h^2/2 >= 0 for every h), times 1 + 2^-23 for the f32 rounding of v'.  After
// nsteps steps the speeds stay below M F, F = ((1 + h^2)(1 + 2^-23))^nsteps; with
// M <= vsafe = vnear / (1.001 F) (the margin covers the float-pair errors of u) every step
// is within the shift series.  -1 when umax itself exceeds that.
TurnsK make_turns_k(const soax_flow* fl, const FlowK& f, int nsteps) {
  TurnsK t = make_turns_k(fl->dt, amplitude_bound(fl));
  if (fl->tau_field >= 0 || nsteps < 0) return t;  // per-particle tau: no launch-wide h
  const float vnear = 0x1p-9f / f.hdtf.x;        // StepC::vnear, the same float division
  const double h = f.dt / fl->tau;
  const double F = std::pow((1.0 + h * h) * (1.0 + 0x1p-23), (double)nsteps);
  const double vs = (double)vnear / (1.001 * F);
  if (std::isfinite(vs) && vs >= (double)t.umax) t.vsafe = (float)vs;
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
  kern<<<gsz, kFusedBlock, kScaledTrigBytes, as_stream(stream)>>>(e, f, make_turns_k(fl, f, nsteps), nsteps,
                                                                   grid ? keys : nullptr, ck);
  return check_launch(who);
}

using GatherKernel = void (*)(EnsArgs, EnsArgs, GatherArgs, FlowK, TurnsK, int, uint32_t*, CellKeyK);

static GatherKernel gather_kernel(bool tau, bool acc) {
  if (tau)
    return acc ? k_step_soa_fused_gather<kFusedBlock, kFusedMinBlocks, true, true>
               : k_step_soa_fused_gather<kFusedBlock, kFusedMinBlocks, true, false>;
  return acc ? k_step_soa_fused_gather<kFusedBlock, kFusedMinBlocks, false, true>
             : k_step_soa_fused_gather<kFusedBlock, kFusedMinBlocks, false, false>;
}

static int prepare_gather_kernels() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return cuda_fail(cudaGetLastError(), "soax_permute_step_fused: device");
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return SOAX_OK;
  for (int v = 0; v < 4; ++v) {
    const void* fn = (const void*)gather_kernel(v & 1, v & 2);
    cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kScaledTrigBytes);
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (err != cudaSuccess) return cuda_fail(err, "soax_permute_step_fused: kernel attributes");
  }
  done[dev] = true;
  return SOAX_OK;
}

static int permute_step_fused(soax_t h, const uint32_t* perm, const soax_flow* fl, int32_t nsteps, int32_t grid,
                              uint32_t* keys, void* stream) {
  const char* who = "soax_permute_step_fused";
  if (int r = check_handle(h)) return r;
  if (nsteps < 0) return fail(SOAX_EINVAL, std::string(who) + ": nsteps < 0");
  const int src = h->current, dst = src ^ 1;
  EnsArgs ein, eout;
  FlowK f;
  if (int r = make_ens_args(h, fl, src, &ein, &f, who)) return r;
  if (int r = make_ens_args(h, fl, dst, &eout, &f, who)) return r;
  CellKeyK ck{};
  if (grid) {
    if (grid < 1 || grid > 1024) return fail(SOAX_EINVAL, std::string(who) + ": grid must be in 1..1024");
    if (h->n > 0 && !keys) return fail(SOAX_EINVAL, std::string(who) + ": keys is NULL");
    if (!aligned16(keys)) return fail(SOAX_EALIGN, std::string(who) + ": keys not 16-byte aligned");
    ck = make_cell_key_k(grid);
  }
  if (h->n == 0) {
    h->current = dst;
    return SOAX_OK;
  }
  if (!perm) return fail(SOAX_EINVAL, std::string(who) + ": perm is NULL");
  if (!aligned16(perm)) return fail(SOAX_EALIGN, std::string(who) + ": perm not 16-byte aligned");
  if (int r = live_planes_bound(h, src)) return r;
  if (int r = live_planes_bound(h, dst)) return r;
  if (nsteps == 0) {  // the permute alone, then the keys of the permuted positions
    if (int r = soax_permute(h, perm, stream)) return r;
    return grid ? soax_cell_keys(h, fl->pos_field, grid, keys, stream) : SOAX_OK;
  }
  GatherArgs g;
  g.perm = perm;
  g.status = status_word();
  if (!g.status) return fail(SOAX_ECUDA, std::string(who) + ": status word");
  g.nother = 0;
  for (int fi = 0; fi < (int)h->fields.size(); ++fi) {
    if (fi == fl->pos_field || fi == fl->vel_field || fi == fl->acc_field) continue;
    for (int c = 0; c < h->fields[fi].ncomp; ++c) {
      const int pl = h->fields[fi].first_plane + c;
      g.in[g.nother] = h->planes[src][pl];
      g.out[g.nother] = h->planes[dst][pl];
      g.es[g.nother] = h->plane_esize[pl];
      ++g.nother;
    }
  }
  if (int r = prepare_gather_kernels()) return r;
  const GatherKernel kern = gather_kernel(ein.tau_src != nullptr, ein.ax != nullptr);
  const int gsz = persistent_grid((const void*)kern, kFusedBlock, kScaledTrigBytes, grid_for(h->n, kFusedBlock));
  kern<<<gsz, kFusedBlock, kScaledTrigBytes, as_stream(stream)>>>(ein, eout, g, f, make_turns_k(fl, f, nsteps), nsteps,
                                                                  grid ? keys : nullptr, ck);
  if (int r = check_launch(who)) return r;
  h->current = dst;
  return SOAX_OK;
}

}  // namespace soax

extern "C" int soax_permute_step_fused(soax_t h, const uint32_t* perm, const soax_flow* fl, int32_t nsteps,
                                       int32_t grid, uint32_t* keys, void* stream) {
  return soax::permute_step_fused(h, perm, fl, nsteps, grid, keys, stream);
}

extern "C" int soax_step_fused(soax_t h, const soax_flow* fl, int32_t nsteps, void* stream) {
  return soax::step_fused(h, fl, nsteps, 0, nullptr, stream, "soax_step_fused");
}

extern "C" int soax_step_fused_keys(soax_t h, const soax_flow* fl, int32_t nsteps, int32_t grid, uint32_t* keys,
                                    void* stream) {
  if (grid == 0) return soax::fail(SOAX_EINVAL, "soax_step_fused_keys: grid must be in 1..1024");
  return soax::step_fused(h, fl, nsteps, grid, keys, stream, "soax_step_fused_keys");
}
