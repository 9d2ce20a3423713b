// soax_step_batched: many independent ensembles (each its own handle, flow amplitudes
// and tau) advanced by one persistent launch per step, and soax_autotune, which times
// the candidate launch shapes and returns the fastest.
//
// The ensembles are cut into tiles of block*PPT particles; tile t belongs to the
// ensemble e with prefix[e] <= t < prefix[e+1] (binary search over the prefix held in
// shared memory).  A grid sized to fill the GPU once walks the tiles with a fixed
// stride, so no block waits on another.  The per-particle arithmetic is the same device
// function as soax_step's, so every launch shape gives bit-identical results.
#include <map>
#include <mutex>
#include <vector>

#include "soax_internal.h"
#include "step_core.cuh"

namespace soax {

constexpr int kMaxEnsembles = 4096;

static size_t b256(size_t x) { return (x + 255) & ~size_t(255); }

static size_t batched_ws_bytes(int nens) {
  return b256((size_t)nens * sizeof(EnsArgs)) + b256((size_t)(nens + 1) * sizeof(int64_t));
}

template <int PPT, int VB>
__global__ void __launch_bounds__(512) k_step_batched(const EnsArgs* __restrict__ ens,
                                                      const int64_t* __restrict__ prefix, int nens, int64_t ntiles,
                                                      FlowK f, int nsteps_inner) {
  extern __shared__ int64_t s_prefix[];
  __shared__ float4 s_tab[SOAX_TRIG_TABLE_SIZE];
  for (int k = threadIdx.x; k <= nens; k += blockDim.x) s_prefix[k] = prefix[k];
  load_trig_table(s_tab);
  const int64_t tile_parts = (int64_t)blockDim.x * PPT;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int lo = 0, hi = nens;
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (s_prefix[mid] <= t) lo = mid; else hi = mid;
    }
    const EnsArgs e = ens[lo];
    const int64_t i0 = (t - s_prefix[lo]) * tile_parts + (int64_t)threadIdx.x * PPT;
    if (i0 < e.n) {
      const StepC kc = make_stepc(e, f);
      const TrigUnscaled tg = trig_unscaled(s_tab, e);
      const int64_t cnt = e.n - i0;
      if (e.tau_src) {
        if (e.ax) step_span_t<PPT, VB, true, true>(e, kc, tg, i0, cnt, nsteps_inner);
        else step_span_t<PPT, VB, true, false>(e, kc, tg, i0, cnt, nsteps_inner);
      } else {
        if (e.ax) step_span_t<PPT, VB, false, true>(e, kc, tg, i0, cnt, nsteps_inner);
        else step_span_t<PPT, VB, false, false>(e, kc, tg, i0, cnt, nsteps_inner);
      }
    }
  }
}

using BatchedKernel = void (*)(const EnsArgs*, const int64_t*, int, int64_t, FlowK, int);

static BatchedKernel pick_kernel(int ppt, int vb) {
  if (ppt == 1) return k_step_batched<1, 64>;
  if (ppt == 2) return vb == 128 ? k_step_batched<2, 128> : k_step_batched<2, 64>;
  if (ppt == 4) return vb == 128 ? k_step_batched<4, 128> : k_step_batched<4, 64>;
  return nullptr;
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
  BatchedKernel kern = nullptr;
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
  EnsArgs* table = reinterpret_cast<EnsArgs*>(host.data());
  int64_t* prefix = reinterpret_cast<int64_t*>(host.data() + b256((size_t)nens * sizeof(EnsArgs)));
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
  }
  out->ntiles = prefix[nens];
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
  out->kern = pick_kernel(t.parts_per_thread, t.vec_bits);
  out->block = t.block;
  out->smem = (size_t)(nens + 1) * sizeof(int64_t);
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (out->smem > 16 * 1024) {  // plus 32 KB of static shared memory (the sin/cos table)
    cudaError_t e =
        cudaFuncSetAttribute((const void*)out->kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)out->smem);
    if (e != cudaSuccess) return cuda_fail(e, "soax_step_batched: smem attribute");
  }
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)out->kern, t.block, out->smem);
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

extern "C" int soax_step_batched(const soax_t* hs, const soax_flow* fls, int32_t nens, int32_t nsteps,
                                 const soax_tune* tune, void* ws, size_t ws_bytes, void* stream) {
  if (nsteps < 0) return fail(SOAX_EINVAL, "soax_step_batched: nsteps < 0");
  const soax_tune t = tune ? *tune : kDefaultTune;
  cudaStream_t s = as_stream(stream);
  Prepared p;
  if (int r = prepare(hs, fls, nens, t, ws, ws_bytes, s, &p)) return r;
  if (p.ntiles == 0 || nsteps == 0) return SOAX_OK;
  const EnsArgs* table = static_cast<const EnsArgs*>(ws);
  const int64_t* prefix = reinterpret_cast<const int64_t*>(static_cast<char*>(ws) + b256((size_t)nens * sizeof(EnsArgs)));
  if (t.fuse_steps) {
    p.kern<<<p.grid, p.block, p.smem, s>>>(table, prefix, nens, p.ntiles, p.f, nsteps);
    return check_launch("soax_step_batched");
  }
  for (int k = 0; k < nsteps; ++k) {
    p.kern<<<p.grid, p.block, p.smem, s>>>(table, prefix, nens, p.ntiles, p.f, 1);
    if (int r = check_launch("soax_step_batched")) return r;
  }
  return SOAX_OK;
}

extern "C" int soax_autotune(const soax_t* hs, const soax_flow* fls, int32_t nens, int32_t nsteps_probe, void* ws,
                             size_t ws_bytes, soax_tune* out, void* stream) {
  if (!out || nsteps_probe < 1) return fail(SOAX_EINVAL, "soax_autotune: bad argument");
  cudaStream_t s = as_stream(stream);
  std::vector<soax_tune> cands;
  for (int ppt : {1, 2, 4})
    for (int vb : {64, 128}) {
      if (ppt == 1 && vb == 128) continue;  // a single particle never fills a 16-byte load
      for (int block : {128, 256, 512}) cands.push_back(soax_tune{ppt, block, vb, 0});
    }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return fail(SOAX_ECUDA, "soax_autotune: event create");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(SOAX_ECUDA, "soax_autotune: event create");
  }
  float best = 1e30f;
  soax_tune bt = kDefaultTune;
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
