// soax_step_batched: many independent ensembles (each its own handle, flow amplitudes
// and tau) advanced by one persistent launch per step, and soax_autotune, which times
// the candidate launch shapes and returns the fastest.
//
// The ensembles are cut into tiles of block*PPT particles; tile t belongs to the
// ensemble e with prefix[e] <= t < prefix[e+1].  A grid sized to fill the GPU once walks
// the tiles (the per-step form: each block an equal contiguous range of them; the fused
// form: a fixed stride), so no block waits on another.  Two forms: one launch per step, with soax_step's per-particle function, and
// the fused form (tune.fuse_steps), all steps of the call in registers with
// soax_step_fused's per-particle function.  Every launch shape of a form gives the same
// bits as the matching single-ensemble call.
#include <cmath>
#include <map>
#include <mutex>
#include <vector>

#include "soax_internal.h"
#include "step_core.cuh"
#include "step_fused.cuh"

namespace soax {

TurnsK make_turns_k(double dt, double umax);
double amplitude_bound(const soax_flow* fl);

constexpr int kMaxEnsembles = 4096;

static size_t b256(size_t x) { return (x + 255) & ~size_t(255); }

// The plan in a workspace: this header, then the ensemble table (nens EnsArgs), then the
// tile prefix (nens + 1 int64), each region 256-byte aligned.  The kernels compare the
// header with their launch arguments before touching anything else, so a plan the
// memory no longer holds (the caller reused the workspace behind the library's back) is
// reported through the status word instead of being followed.
struct PlanHeader {
  uint64_t magic;
  int64_t nens, ntiles, tile_parts;
};
constexpr uint64_t kPlanMagic = 0x534F4158504C414Eull;  // "SOAXPLAN"
constexpr size_t kHeaderBytes = 256;

static size_t batched_ws_bytes(int nens) {
  return kHeaderBytes + b256((size_t)nens * sizeof(EnsArgs)) + b256((size_t)(nens + 1) * sizeof(int64_t));
}

// True (for every thread of the block alike) when the plan header matches the launch.
__device__ __forceinline__ bool plan_ok(const PlanHeader* hdr, int nens, int64_t ntiles, int64_t tile_parts,
                                        int* status) {
  const bool ok = hdr->magic == kPlanMagic && hdr->nens == nens && hdr->ntiles == ntiles &&
                  hdr->tile_parts == tile_parts;
  if (!ok && threadIdx.x == 0 && blockIdx.x == 0) atomicExch(status, (int)SOAX_EINVAL);
  return ok;
}

// One launch per step.  Each block takes a contiguous range of tiles (an equal share of
// all of them), so it stays within one ensemble for long stretches: it finds the
// ensemble of its first tile once, steps to the next ensemble when its tiles run out, and
// only then reloads the ensemble's arguments and rebuilds the three amplitude-scaled
// sin/cos tables (96 KB of dynamic shared memory) -- the tables and per-particle
// function of soax_step, hence its bits.  PLAIN: no ensemble has a tau or acceleration
// field (one per-particle form, fewer registers); otherwise the form is chosen per
// ensemble.
template <int PPT, int VB, bool PLAIN>
__global__ void __launch_bounds__(512, 2) k_step_batched(const PlanHeader* __restrict__ hdr,
                                                      const EnsArgs* __restrict__ ens,
                                                      const int64_t* __restrict__ prefix, int nens, int64_t ntiles,
                                                      FlowK f, int nsteps_inner, int* status) {
  extern __shared__ float4 s_tab3[];
  __shared__ EnsArgs s_e;
  const int64_t tile_parts = (int64_t)blockDim.x * PPT;
  if (!plan_ok(hdr, nens, ntiles, tile_parts, status)) return;
  const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * per;
  const int64_t t1 = t0 + per < ntiles ? t0 + per : ntiles;
  if (t0 >= t1) return;  // uniform over the block
  int lo = 0, hi = nens;  // the ensemble of t0: prefix[lo] <= t0 < prefix[lo + 1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= t0) lo = mid; else hi = mid;
  }
  int cur = -1;
  int64_t next = 0;  // prefix[lo + 1] while lo == cur
  for (int64_t t = t0; t < t1; ++t) {
    if (cur < 0 || t >= next) {  // uniform over the block, as t is
      while (prefix[lo + 1] <= t) ++lo;
      __syncthreads();  // every thread is done with the previous ensemble's tables
      if (threadIdx.x == 0) s_e = ens[lo];
      load_scaled_trig_tables(s_tab3, ff_from2(ens[lo].Af), ff_from2(ens[lo].Bf), ff_from2(ens[lo].Cf));
      cur = lo;
      next = prefix[lo + 1];
    }
    const EnsArgs& e = s_e;
    const int64_t i0 = (t - prefix[cur]) * tile_parts + (int64_t)threadIdx.x * PPT;
    if (i0 < e.n) {
      const StepC kc = make_stepc(e, f);
      const TrigScaled tg{s_tab3};
      const int64_t cnt = e.n - i0;
      if constexpr (PLAIN) {
        step_span_t<PPT, VB, false, false>(e, kc, tg, i0, cnt, nsteps_inner);
      } else if (e.tau_src) {
        if (e.ax) step_span_t<PPT, VB, true, true>(e, kc, tg, i0, cnt, nsteps_inner);
        else step_span_t<PPT, VB, true, false>(e, kc, tg, i0, cnt, nsteps_inner);
      } else {
        if (e.ax) step_span_t<PPT, VB, false, true>(e, kc, tg, i0, cnt, nsteps_inner);
        else step_span_t<PPT, VB, false, false>(e, kc, tg, i0, cnt, nsteps_inner);
      }
    }
  }
}

// Fused form: every particle loaded once, advanced nsteps steps in registers (positions
// as fixed-point turns) and stored once.  A tile covers one ensemble, so the block
// rebuilds the three amplitude-scaled sin/cos tables (96 KB of dynamic shared memory)
// only when its next tile belongs to another ensemble: a tile carries
// block*PPT*nsteps particle-steps against 6144 table entries.  FORM: 0 = no tau or
// acceleration field in any ensemble, 1 = tau fields, 2 = acceleration fields, 3 = both,
// 4 = a mix (decided per ensemble, with more registers).
template <int FORM, bool TAU, bool ACC, int PPT>
__device__ __forceinline__ void batched_fused_span(const EnsArgs& e, const StepC& kc, const TurnsK& tk,
                                                   const TrigScaled& tg, int64_t i0, int64_t cnt, int nsteps) {
  if constexpr (FORM == 4) {
    if (e.tau_src) {
      if (e.ax) fused_span<PPT, true, true>(e, kc, tk, tg, i0, cnt, nsteps);
      else fused_span<PPT, true, false>(e, kc, tk, tg, i0, cnt, nsteps);
    } else {
      if (e.ax) fused_span<PPT, false, true>(e, kc, tk, tg, i0, cnt, nsteps);
      else fused_span<PPT, false, false>(e, kc, tk, tg, i0, cnt, nsteps);
    }
  } else {
    fused_span<PPT, TAU, ACC>(e, kc, tk, tg, i0, cnt, nsteps);
  }
}

// TurnsK::vsafe for nsteps steps of ensemble e (its own h = dt/tau and amplitude bound),
// as make_turns_k(fl, f, nsteps) forms it for one ensemble; -1 with tau per particle.
__device__ __forceinline__ float ensemble_vsafe(const EnsArgs& e, const FlowK& f, int nsteps) {
  if (e.tau_src) return -1.0f;
  const float vnear = __fdiv_rn(0x1p-9f, f.hdtf.x);  // StepC::vnear
  const double h = f.dt * e.inv_tau;
  const double F = pow((1.0 + h * h) * (1.0 + 0x1p-23), (double)nsteps);
  const double a = fabs(e.A), b = fabs(e.B), c = fabs(e.C);
  const double um = fmax(a + c, fmax(b + a, c + b)) * (1.0 + 1e-6);
  const double vs = (double)vnear / (1.001 * F);
  return isfinite(vs) && vs >= um ? (float)vs : -1.0f;
}

template <int PPT, int MINB, int FORM>
__global__ void __launch_bounds__(512, MINB) k_step_batched_fused(const PlanHeader* __restrict__ hdr,
                                                                  const EnsArgs* __restrict__ ens,
                                                                  const int64_t* __restrict__ prefix, int nens,
                                                                  int64_t ntiles, FlowK f, TurnsK tk, int nsteps,
                                                                  int* status) {
  extern __shared__ float4 s_tab3[];
  __shared__ EnsArgs s_e;  // the current ensemble's arguments (read, not held in registers)
  __shared__ float s_vsafe;  // and its TurnsK::vsafe for this call
  const int64_t tile_parts = (int64_t)blockDim.x * PPT;
  if (!plan_ok(hdr, nens, ntiles, tile_parts, status)) return;
  int cur = -1;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int lo = 0, hi = nens;
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (prefix[mid] <= t) lo = mid; else hi = mid;
    }
    if (lo != cur) {  // uniform over the block, as t is
      __syncthreads();  // every thread is done with the previous ensemble's tables
      if (threadIdx.x == 0) {
        s_e = ens[lo];
        s_vsafe = ensemble_vsafe(ens[lo], f, nsteps);
      }
      load_scaled_trig_tables(s_tab3, ff_from2(ens[lo].Af), ff_from2(ens[lo].Bf), ff_from2(ens[lo].Cf));
      cur = lo;
    }
    const EnsArgs& e = s_e;
    const int64_t i0 = (t - prefix[lo]) * tile_parts + (int64_t)threadIdx.x * PPT;
    if (i0 < e.n) {
      const StepC kc = make_stepc(e, f);
      const TrigScaled tg{s_tab3};
      TurnsK tke = tk;
      tke.vsafe = s_vsafe;
      batched_fused_span<FORM, FORM == 1 || FORM == 3, FORM == 2 || FORM == 3, PPT>(e, kc, tke, tg, i0, e.n - i0,
                                                                                     nsteps);
    }
  }
}

using BatchedKernel = void (*)(const PlanHeader*, const EnsArgs*, const int64_t*, int, int64_t, FlowK, int, int*);
using BatchedFusedKernel = void (*)(const PlanHeader*, const EnsArgs*, const int64_t*, int, int64_t, FlowK, TurnsK,
                                    int, int*);

template <bool PLAIN>
static BatchedKernel pick_kernel_form(int ppt, int vb) {
  if (ppt == 1) return k_step_batched<1, 64, PLAIN>;
  if (ppt == 2) return vb == 128 ? k_step_batched<2, 128, PLAIN> : k_step_batched<2, 64, PLAIN>;
  if (ppt == 4) return vb == 128 ? k_step_batched<4, 128, PLAIN> : k_step_batched<4, 64, PLAIN>;
  return nullptr;
}

static BatchedKernel pick_kernel(int ppt, int vb, int form) {
  return form == 0 ? pick_kernel_form<true>(ppt, vb) : pick_kernel_form<false>(ppt, vb);
}

template <int FORM>
static BatchedFusedKernel pick_fused_form(int ppt) {
  if (ppt == 1) return k_step_batched_fused<1, 2, FORM>;
  if (ppt == 2) return k_step_batched_fused<2, 1, FORM>;
  if (ppt == 4) return k_step_batched_fused<4, 1, FORM>;
  return nullptr;
}

static BatchedFusedKernel pick_fused_kernel(int ppt, int form) {
  switch (form) {
    case 0: return pick_fused_form<0>(ppt);
    case 1: return pick_fused_form<1>(ppt);
    case 2: return pick_fused_form<2>(ppt);
    case 3: return pick_fused_form<3>(ppt);
    default: return pick_fused_form<4>(ppt);
  }
}

static int check_tune(const soax_tune& t) {
  if (t.parts_per_thread != 1 && t.parts_per_thread != 2 && t.parts_per_thread != 4)
    return fail(SOAX_EINVAL, "soax_tune: parts_per_thread must be 1, 2 or 4");
  if (t.block < 64 || t.block > 512 || t.block % 32)
    return fail(SOAX_EINVAL, "soax_tune: block must be a multiple of 32 in 64..512");
  if (t.vec_bits != 64 && t.vec_bits != 128) return fail(SOAX_EINVAL, "soax_tune: vec_bits must be 64 or 128");
  return SOAX_OK;
}

// Plans already copied into a workspace, keyed by the workspace address.
static std::mutex g_plan_mu;
static std::map<void*, std::vector<char>> g_plans;

struct Prepared {
  int64_t ntiles = 0;
  FlowK f{};
  double umax = 0.0;  // the largest amplitude bound over the ensembles
  BatchedKernel kern = nullptr;
  BatchedFusedKernel fkern = nullptr;
  int* status = nullptr;
  int grid = 0, block = 0;
  size_t smem = 0;
};

static int prepare(const soax_t* hs, const soax_flow* fls, int nens, const soax_tune& t, void* ws, size_t ws_bytes,
                   cudaStream_t s, Prepared* out) {
  if (!hs || !fls) return fail(SOAX_EINVAL, "soax_step_batched: NULL ensemble arrays");
  if (nens < 1 || nens > kMaxEnsembles) return fail(SOAX_EINVAL, "soax_step_batched: nens must be in 1..4096");
  if (int r = check_tune(t)) return r;
  const size_t need = batched_ws_bytes(nens);
  if (!ws || ws_bytes < need) return fail(SOAX_ENOMEM, "soax_step_batched: workspace too small");
  if (!aligned16(ws)) return fail(SOAX_EALIGN, "soax_step_batched: workspace not 16-byte aligned");
  std::vector<char> host(need, 0);
  PlanHeader* hdr = reinterpret_cast<PlanHeader*>(host.data());
  EnsArgs* table = reinterpret_cast<EnsArgs*>(host.data() + kHeaderBytes);
  int64_t* prefix = reinterpret_cast<int64_t*>(host.data() + kHeaderBytes + b256((size_t)nens * sizeof(EnsArgs)));
  const int64_t tile_parts = (int64_t)t.block * t.parts_per_thread;
  prefix[0] = 0;
  for (int k = 0; k < nens; ++k) {
    if (int r = check_handle(hs[k])) return r;
    FlowK fk;
    if (int r = make_ens_args(hs[k], &fls[k], hs[k]->current, &table[k], &fk, "soax_step_batched")) return r;
    if (k == 0)
      out->f = fk;
    else if (fk.dt != out->f.dt)
      return fail(SOAX_EINVAL, "soax_step_batched: every ensemble must use the same dt");
    prefix[k + 1] = prefix[k] + (hs[k]->n + tile_parts - 1) / tile_parts;
    out->umax = std::fmax(out->umax, amplitude_bound(&fls[k]));
  }
  out->ntiles = prefix[nens];
  hdr->magic = kPlanMagic;
  hdr->nens = nens;
  hdr->ntiles = out->ntiles;
  hdr->tile_parts = tile_parts;
  out->status = status_word();
  if (!out->status) return fail(SOAX_ECUDA, "soax_step_batched: status word");
  // The fields every ensemble carries: one kernel form for all, or the mixed one.
  int form = -1;
  for (int k = 0; k < nens; ++k) {
    const int fk = (table[k].tau_src ? 1 : 0) | (table[k].ax ? 2 : 0);
    form = (form < 0 || form == fk) ? fk : 4;
  }
  {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto it = g_plans.find(ws);
    if (it == g_plans.end() || it->second != host) {
      cudaError_t e = cudaMemcpyAsync(ws, host.data(), need, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        g_plans.erase(ws);
        return cuda_fail(e, "soax_step_batched: plan upload");
      }
      g_plans[ws] = std::move(host);
    }
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const void* fn = nullptr;
  out->block = t.block;
  if (t.fuse_steps) {
    out->fkern = pick_fused_kernel(t.parts_per_thread, form);
    out->smem = kScaledTrigBytes;
    fn = (const void*)out->fkern;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)out->smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return cuda_fail(e, "soax_step_batched: fused kernel attributes");
  } else {
    out->kern = pick_kernel(t.parts_per_thread, t.vec_bits, form);
    out->smem = kScaledTrigBytes;
    fn = (const void*)out->kern;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)out->smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return cuda_fail(e, "soax_step_batched: kernel attributes");
  }
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, t.block, out->smem);
  if (e != cudaSuccess || per_sm < 1) per_sm = 1;
  int64_t g = (int64_t)sms * per_sm;
  if (g > out->ntiles) g = out->ntiles;
  out->grid = (int)(g < 1 ? 1 : g);
  return SOAX_OK;
}

static const soax_tune kDefaultTune = {4, 256, 128, 0};

}  // namespace soax

using namespace soax;

extern "C" int soax_batched_workspace_bytes(const soax_t* hs, int32_t nens, const soax_tune* tune, size_t* bytes) {
  (void)hs;
  (void)tune;
  if (!bytes || nens < 1 || nens > kMaxEnsembles) return fail(SOAX_EINVAL, "soax_batched_workspace_bytes: bad argument");
  *bytes = batched_ws_bytes(nens);
  return SOAX_OK;
}

extern "C" int soax_batched_forget(const void* ws) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  g_plans.erase(const_cast<void*>(ws));
  return SOAX_OK;
}

extern "C" int soax_step_batched(const soax_t* hs, const soax_flow* fls, int32_t nens, int32_t nsteps,
                                 const soax_tune* tune, void* ws, size_t ws_bytes, void* stream) {
  if (nsteps < 0) return fail(SOAX_EINVAL, "soax_step_batched: nsteps < 0");
  const soax_tune t = tune ? *tune : kDefaultTune;
  cudaStream_t s = as_stream(stream);
  Prepared p;
  if (int r = prepare(hs, fls, nens, t, ws, ws_bytes, s, &p)) return r;
  if (p.ntiles == 0 || nsteps == 0) return SOAX_OK;
  const PlanHeader* hdr = static_cast<const PlanHeader*>(ws);
  const EnsArgs* table = reinterpret_cast<const EnsArgs*>(static_cast<char*>(ws) + kHeaderBytes);
  const int64_t* prefix = reinterpret_cast<const int64_t*>(static_cast<char*>(ws) + kHeaderBytes +
                                                           b256((size_t)nens * sizeof(EnsArgs)));
  if (t.fuse_steps) {
    p.fkern<<<p.grid, p.block, p.smem, s>>>(hdr, table, prefix, nens, p.ntiles, p.f, make_turns_k(p.f.dt, p.umax), nsteps,
                                            p.status);
    return check_launch("soax_step_batched");
  }
  for (int k = 0; k < nsteps; ++k) {
    p.kern<<<p.grid, p.block, p.smem, s>>>(hdr, table, prefix, nens, p.ntiles, p.f, 1, p.status);
    if (int r = check_launch("soax_step_batched")) return r;
  }
  return SOAX_OK;
}

extern "C" int soax_autotune(const soax_t* hs, const soax_flow* fls, int32_t nens, int32_t nsteps_probe, void* ws,
                             size_t ws_bytes, soax_tune* out, void* stream) {
  if (!out || nsteps_probe < 1) return fail(SOAX_EINVAL, "soax_autotune: bad argument");
  cudaStream_t s = as_stream(stream);
  const int fuse = out->fuse_steps ? 1 : 0;  // the form to tune, given on entry
  std::vector<soax_tune> cands;
  for (int ppt : {1, 2, 4})
    for (int vb : {64, 128}) {
      if (ppt == 1 && vb == 128) continue;  // a single particle never fills a 16-byte load
      if (fuse && vb == 64) continue;       // the fused form loads each plane once: width is moot
      for (int block : {128, 256, 512}) cands.push_back(soax_tune{ppt, block, vb, fuse});
    }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return fail(SOAX_ECUDA, "soax_autotune: event create");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(SOAX_ECUDA, "soax_autotune: event create");
  }
  float best = 1e30f;
  soax_tune bt = kDefaultTune;
  bt.fuse_steps = fuse;
  int rc = SOAX_OK;
  for (const soax_tune& c : cands) {
    if ((rc = soax_step_batched(hs, fls, nens, nsteps_probe, &c, ws, ws_bytes, stream))) break;  // warm-up, upload
    cudaEventRecord(e0, s);
    if ((rc = soax_step_batched(hs, fls, nens, nsteps_probe, &c, ws, ws_bytes, stream))) break;
    cudaEventRecord(e1, s);
    cudaError_t ce = cudaEventSynchronize(e1);
    if (ce != cudaSuccess) {
      rc = cuda_fail(ce, "soax_autotune");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      bt = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  *out = bt;
  return SOAX_OK;
}
