// soax_step (SoA) and soax_step_aos: one pass over memory per midpoint-RK2 step.
#include <cmath>
#include <mutex>

#include "soax_internal.h"
#include "step_core.cuh"

namespace soax {

// d as a float pair: hi = nearest float, lo = nearest float to d - hi.
float2 split_ff(double d) {
  const float h = (float)d;
  return make_float2(h, (float)(d - (double)h));
}

// Resident blocks per SM of a kernel at the given block size (cached per kernel).
int persistent_grid(const void* kern, int block, size_t smem, int64_t work_blocks) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  int64_t g = (int64_t)sms * per_sm;
  if (g > work_blocks) g = work_blocks;
  return (int)(g < 1 ? 1 : g);
}

int make_ens_args(soax_t h, const soax_flow* fl, int buf, EnsArgs* e, FlowK* f, const char* who) {
  std::string w(who);
  if (!fl) return fail(SOAX_EINVAL, w + ": flow is NULL");
  if (!(fl->dt > 0.0) || !std::isfinite(fl->dt)) return fail(SOAX_EINVAL, w + ": dt must be finite and > 0");
  if (!std::isfinite(fl->A) || !std::isfinite(fl->B) || !std::isfinite(fl->C))
    return fail(SOAX_EINVAL, w + ": flow amplitudes must be finite");
  if (int r = check_field(h, fl->pos_field, SOAX_F64, 3, "position")) return r;
  if (int r = check_field(h, fl->vel_field, SOAX_F32, 3, "velocity")) return r;
  if (fl->acc_field >= 0) {
    if (int r = check_field(h, fl->acc_field, SOAX_F32, 3, "acceleration")) return r;
  } else if (fl->acc_field != -1) {
    return fail(SOAX_ESCHEMA, w + ": acc_field must be -1 or a field index");
  }
  if (fl->tau_field >= 0) {
    if (int r = check_field(h, fl->tau_field, SOAX_F32, 1, "tau source")) return r;
    if (!(fl->tau_scale > 0.0) || !std::isfinite(fl->tau_scale))
      return fail(SOAX_EINVAL, w + ": tau_scale must be finite and > 0");
  } else {
    if (fl->tau_field != -1) return fail(SOAX_ESCHEMA, w + ": tau_field must be -1 or a field index");
    if (!(fl->tau > 0.0) || !std::isfinite(fl->tau)) return fail(SOAX_EINVAL, w + ": tau must be finite and > 0");
  }
  auto plane = [&](int field, int comp) -> void* { return h->planes[buf][h->fields[field].first_plane + comp]; };
  e->px = (double*)plane(fl->pos_field, 0);
  e->py = (double*)plane(fl->pos_field, 1);
  e->pz = (double*)plane(fl->pos_field, 2);
  e->vx = (float*)plane(fl->vel_field, 0);
  e->vy = (float*)plane(fl->vel_field, 1);
  e->vz = (float*)plane(fl->vel_field, 2);
  e->ax = e->ay = e->az = nullptr;
  if (fl->acc_field >= 0) {
    e->ax = (float*)plane(fl->acc_field, 0);
    e->ay = (float*)plane(fl->acc_field, 1);
    e->az = (float*)plane(fl->acc_field, 2);
  }
  e->tau_src = fl->tau_field >= 0 ? (const float*)plane(fl->tau_field, 0) : nullptr;
  e->n = h->n;
  e->A = fl->A;
  e->B = fl->B;
  e->C = fl->C;
  e->inv_tau = fl->tau_field >= 0 ? 0.0 : 1.0 / fl->tau;
  e->tau_scale = fl->tau_scale;
  e->Af = split_ff(fl->A);
  e->Bf = split_ff(fl->B);
  e->Cf = split_ff(fl->C);
  e->itf = split_ff(e->inv_tau);
  e->tsf = split_ff(fl->tau_scale);
  if (h->n > 0) {
    if (!e->px || !e->py || !e->pz || !e->vx || !e->vy || !e->vz ||
        (fl->acc_field >= 0 && (!e->ax || !e->ay || !e->az)) || (fl->tau_field >= 0 && !e->tau_src))
      return fail(SOAX_EUNBOUND, w + ": a plane the step needs is not bound");
  }
  f->A = fl->A;
  f->B = fl->B;
  f->C = fl->C;
  f->dt = fl->dt;
  f->hdt = 0.5 * fl->dt;
  f->dtf = split_ff(f->dt);
  f->hdtf = split_ff(f->hdt);
  return SOAX_OK;
}

// Launch shape of the plain step, picked by timing launch shapes on 16.7M particles:
// 2 particles per thread, 512 threads, 2 resident blocks per SM (64 registers).
constexpr int kStepPPT = 2;
constexpr int kStepBlock = 512;
constexpr int kStepMinBlocks = 2;

template <int PPT, int VB, bool TAU, bool ACC>
__device__ __forceinline__ void step_soa_loop(const EnsArgs& e, const StepC& kc, const TrigScaled& tg) {
  const int64_t ngroups = (e.n + PPT - 1) / PPT;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += (int64_t)gridDim.x * blockDim.x)
    step_span_t<PPT, VB, TAU, ACC>(e, kc, tg, g * PPT, e.n - g * PPT, 1);
}

// Persistent: a grid that fills the GPU once walks groups of PPT particles with a
// fixed stride, so each block builds its amplitude-scaled tables (96 KB of dynamic
// shared memory) only once.
template <int PPT, int VB>
__global__ void __launch_bounds__(kStepBlock, kStepMinBlocks) k_step_soa(EnsArgs e, FlowK f) {
  extern __shared__ float4 s_tab3[];
  load_scaled_trig_tables(s_tab3, ff_from2(e.Af), ff_from2(e.Bf), ff_from2(e.Cf));
  const StepC kc = make_stepc(e, f);
  const TrigScaled tg{s_tab3};
  if (e.tau_src) {
    if (e.ax) step_soa_loop<PPT, VB, true, true>(e, kc, tg);
    else step_soa_loop<PPT, VB, true, false>(e, kc, tg);
  } else {
    if (e.ax) step_soa_loop<PPT, VB, false, true>(e, kc, tg);
    else step_soa_loop<PPT, VB, false, false>(e, kc, tg);
  }
}

// Dynamic shared memory above 48 KB and the largest carveout, set once per device.
static int prepare_step_kernel() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cuda_fail(cudaGetLastError(), "soax_step: device");
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return SOAX_OK;
  const void* fn = (const void*)k_step_soa<kStepPPT, 128>;
  cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kScaledTrigBytes);
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (err != cudaSuccess) return cuda_fail(err, "soax_step: kernel attributes");
  done[dev] = true;
  return SOAX_OK;
}

struct AosArgs {
  char* rec;
  int64_t R, pos_off, vel_off, acc_off, tau_off;  // offsets in bytes; -1 = absent
  int64_t n;
  EnsArgs e;  // flow amplitudes and tau (the plane pointers are unused)
};

template <bool ACC>
__device__ __forceinline__ void step_aos_loop(const AosArgs& a, const StepC& kc, const TrigScaled& tg) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    char* r = a.rec + i * a.R;
    const double* pp = reinterpret_cast<const double*>(r + a.pos_off);
    const float* vp = reinterpret_cast<const float*>(r + a.vel_off);
    double p[3] = {pp[0], pp[1], pp[2]};
    float v[3] = {vp[0], vp[1], vp[2]}, acc[3];
    StepC k = kc;
    if (a.tau_off >= 0) set_inv_tau(k, ff_inv_tau(a.e.tsf, *reinterpret_cast<const float*>(r + a.tau_off)));
    // The SoA step's dispatch (step_group with one particle): straight-line code within
    // the shift series, the per-coordinate checks otherwise; the same bits either way.
    if (near_shift(k, v))
      rk2_step_fast<ACC, true>(k, tg, p, v, acc);
    else
      rk2_step_fast<ACC, false>(k, tg, p, v, acc);
    double* pw = reinterpret_cast<double*>(r + a.pos_off);
    float* vw = reinterpret_cast<float*>(r + a.vel_off);
    pw[0] = p[0]; pw[1] = p[1]; pw[2] = p[2];
    vw[0] = v[0]; vw[1] = v[1]; vw[2] = v[2];
    if constexpr (ACC) {
      float* aw = reinterpret_cast<float*>(r + a.acc_off);
      aw[0] = acc[0]; aw[1] = acc[1]; aw[2] = acc[2];
    }
  }
}

// The same arithmetic and tables as k_step_soa (the amplitude-scaled tables in 96 KB of
// dynamic shared memory, two 512-thread blocks per SM), so that the SoA-AoS comparison
// differs in the memory layout alone.
constexpr int kAosBlock = 512;

__global__ void __launch_bounds__(kAosBlock, 2) k_step_aos(AosArgs a, FlowK f) {
  extern __shared__ float4 s_tab3[];
  load_scaled_trig_tables(s_tab3, ff_from2(a.e.Af), ff_from2(a.e.Bf), ff_from2(a.e.Cf));
  const StepC kc = make_stepc(a.e, f);
  const TrigScaled tg{s_tab3};
  if (a.acc_off >= 0)
    step_aos_loop<true>(a, kc, tg);
  else
    step_aos_loop<false>(a, kc, tg);
}

static int prepare_aos_kernel() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return cuda_fail(cudaGetLastError(), "soax_step_aos: device");
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return SOAX_OK;
  cudaError_t err = cudaFuncSetAttribute((const void*)k_step_aos, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kScaledTrigBytes);
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute((const void*)k_step_aos, cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared);
  if (err != cudaSuccess) return cuda_fail(err, "soax_step_aos: kernel attributes");
  done[dev] = true;
  return SOAX_OK;
}

}  // namespace soax

using namespace soax;

extern "C" int soax_step(soax_t h, const soax_flow* fl, int32_t nsteps, void* stream) {
  if (int r = check_handle(h)) return r;
  if (nsteps < 0) return fail(SOAX_EINVAL, "soax_step: nsteps < 0");
  EnsArgs e;
  FlowK f;
  if (int r = make_ens_args(h, fl, h->current, &e, &f, "soax_step")) return r;
  if (h->n == 0 || nsteps == 0) return SOAX_OK;
  if (int r = prepare_step_kernel()) return r;
  const int grid = persistent_grid((const void*)k_step_soa<kStepPPT, 128>, kStepBlock, kScaledTrigBytes,
                                   grid_for((h->n + kStepPPT - 1) / kStepPPT, kStepBlock));
  cudaStream_t s = as_stream(stream);
  for (int k = 0; k < nsteps; ++k) {
    k_step_soa<kStepPPT, 128><<<grid, kStepBlock, kScaledTrigBytes, s>>>(e, f);
    if (int r = check_launch("soax_step")) return r;
  }
  return SOAX_OK;
}

extern "C" int soax_step_aos(soax_t h, void* aos_dev, const soax_flow* fl, int32_t nsteps, void* stream) {
  if (int r = check_handle(h)) return r;
  if (nsteps < 0) return fail(SOAX_EINVAL, "soax_step_aos: nsteps < 0");
  if (!aos_dev && h->n > 0) return fail(SOAX_EINVAL, "soax_step_aos: NULL records");
  if (!aligned16(aos_dev)) return fail(SOAX_EALIGN, "soax_step_aos: records not 16-byte aligned");
  // Validate the flow against the schema; the planes are not used, so pretend they are bound.
  EnsArgs e;
  FlowK f;
  soax_s probe = *h;
  for (int p = 0; p < probe.nplanes; ++p) probe.planes[0][p] = (void*)16;
  if (int r = make_ens_args(&probe, fl, 0, &e, &f, "soax_step_aos")) return r;
  if (h->n == 0 || nsteps == 0) return SOAX_OK;
  AosArgs a;
  a.rec = (char*)aos_dev;
  a.R = h->record_bytes;
  a.pos_off = h->offsets[fl->pos_field];
  a.vel_off = h->offsets[fl->vel_field];
  a.acc_off = fl->acc_field >= 0 ? h->offsets[fl->acc_field] : -1;
  a.tau_off = fl->tau_field >= 0 ? h->offsets[fl->tau_field] : -1;
  a.n = h->n;
  a.e = e;
  if (int r = prepare_aos_kernel()) return r;
  const int grid = persistent_grid((const void*)k_step_aos, kAosBlock, kScaledTrigBytes, grid_for(h->n, kAosBlock));
  // One pass over the records per step, like soax_step.
  for (int k = 0; k < nsteps; ++k) {
    k_step_aos<<<grid, kAosBlock, kScaledTrigBytes, as_stream(stream)>>>(a, f);
    if (int r = check_launch("soax_step_aos")) return r;
  }
  return SOAX_OK;
}
