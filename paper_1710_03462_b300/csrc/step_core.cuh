// Per-thread particle processing shared by the plain, batched and checkpointed steps:
// vectorised loads of a thread's PPT consecutive particles from the SoA planes, the
// per-particle step, and vectorised stores.  Every form calls the same per-particle
// function, so their results are bit-identical particle by particle.
#pragma once
#include <cstdint>

#include "rk2_math.cuh"

namespace soax {

// One ensemble's planes and flow parameters.
struct EnsArgs {
  double* px;
  double* py;
  double* pz;
  float* vx;
  float* vy;
  float* vz;
  float* ax;  // may be null (no acceleration field)
  float* ay;
  float* az;
  const float* tau_src;  // may be null (uniform tau)
  int64_t n;
  double A, B, C;
  double inv_tau;    // 1/tau when tau_src is null
  double tau_scale;  // tau_i = tau_scale * tau_src[i] otherwise
  float2 Af, Bf, Cf, itf, tsf;  // A, B, C, inv_tau, tau_scale as float pairs (hi, lo)
};

// 1/tau of particle i of ensemble e (TAU: tau from a field, else uniform).
template <bool TAU>
__device__ __forceinline__ ff particle_inv_tau(const EnsArgs& e, int64_t i) {
  if constexpr (TAU)
    return ff_inv_tau(e.tsf, e.tau_src[i]);
  else
    return ff_from2(e.itf);
}

// The step constants shared by the particles of ensemble e (dt from f); with a uniform
// tau also the ones that depend on it.
__device__ __forceinline__ StepC make_stepc(const EnsArgs& e, const FlowK& f) {
  StepC c;
  c.dt = ff_from2(f.dtf);
  c.hdt = ff_from2(f.hdtf);
  c.dt_d = f.dt;
  c.vnear = __fdiv_rn(SOAX_SHIFT_MAX, f.hdtf.x);
  set_inv_tau(c, ff_from2(e.itf));
  return c;
}

// make_stepc for particle i (its own tau when the ensemble has a tau field).
__device__ __forceinline__ StepC make_stepc(const EnsArgs& e, const FlowK& f, int64_t i) {
  StepC c = make_stepc(e, f);
  if (e.tau_src) set_inv_tau(c, particle_inv_tau<true>(e, i));
  return c;
}

// The plain table scaled per lookup with the amplitudes of ensemble e.
__device__ __forceinline__ TrigUnscaled trig_unscaled(const float4* tab, const EnsArgs& e) {
  TrigUnscaled t;
  t.t = tab;
  t.amp[0] = ff_from2(e.Bf);
  t.amp[1] = ff_from2(e.Cf);
  t.amp[2] = ff_from2(e.Af);
  return t;
}

template <int PPT, int VB>
__device__ __forceinline__ void load_f64(const double* __restrict__ p, int64_t i0, double (&o)[PPT]) {
  if constexpr (VB == 128 && PPT % 2 == 0) {
#pragma unroll
    for (int j = 0; j < PPT / 2; ++j) {
      double2 t = *reinterpret_cast<const double2*>(p + i0 + 2 * j);
      o[2 * j] = t.x;
      o[2 * j + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < PPT; ++j) o[j] = p[i0 + j];
  }
}

template <int PPT, int VB>
__device__ __forceinline__ void store_f64(double* __restrict__ p, int64_t i0, const double (&o)[PPT]) {
  if constexpr (VB == 128 && PPT % 2 == 0) {
#pragma unroll
    for (int j = 0; j < PPT / 2; ++j)
      *reinterpret_cast<double2*>(p + i0 + 2 * j) = make_double2(o[2 * j], o[2 * j + 1]);
  } else {
#pragma unroll
    for (int j = 0; j < PPT; ++j) p[i0 + j] = o[j];
  }
}

template <int PPT, int VB>
__device__ __forceinline__ void load_f32(const float* __restrict__ p, int64_t i0, float (&o)[PPT]) {
  if constexpr (VB == 128 && PPT == 4) {
    float4 t = *reinterpret_cast<const float4*>(p + i0);
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
  } else if constexpr (VB >= 64 && PPT % 2 == 0) {
#pragma unroll
    for (int j = 0; j < PPT / 2; ++j) {
      float2 t = *reinterpret_cast<const float2*>(p + i0 + 2 * j);
      o[2 * j] = t.x;
      o[2 * j + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < PPT; ++j) o[j] = p[i0 + j];
  }
}

template <int PPT, int VB>
__device__ __forceinline__ void store_f32(float* __restrict__ p, int64_t i0, const float (&o)[PPT]) {
  if constexpr (VB == 128 && PPT == 4) {
    *reinterpret_cast<float4*>(p + i0) = make_float4(o[0], o[1], o[2], o[3]);
  } else if constexpr (VB >= 64 && PPT % 2 == 0) {
#pragma unroll
    for (int j = 0; j < PPT / 2; ++j)
      *reinterpret_cast<float2*>(p + i0 + 2 * j) = make_float2(o[2 * j], o[2 * j + 1]);
  } else {
#pragma unroll
    for (int j = 0; j < PPT; ++j) p[i0 + j] = o[j];
  }
}

// Advance the PPT particles i0..i0+PPT-1 (all < n) by nsteps steps, one load and one
// store of each plane.  kc: make_stepc(e, f); TAU: tau per particle from e.tau_src;
// ACC: store the last stage acceleration; trig: the amplitude-scaled table entries.
template <int PPT, int VB, bool TAU, bool ACC, class Trig>
__device__ __forceinline__ void step_group(const EnsArgs& e, const StepC& kc, const Trig& trig, int64_t i0,
                                           int nsteps) {
  double x[PPT], y[PPT], z[PPT];
  float vx[PPT], vy[PPT], vz[PPT];
  load_f64<PPT, VB>(e.px, i0, x);
  load_f64<PPT, VB>(e.py, i0, y);
  load_f64<PPT, VB>(e.pz, i0, z);
  load_f32<PPT, VB>(e.vx, i0, vx);
  load_f32<PPT, VB>(e.vy, i0, vy);
  load_f32<PPT, VB>(e.vz, i0, vz);
  float ax[PPT], ay[PPT], az[PPT];
  ff sj[PPT];
  if constexpr (TAU) {
#pragma unroll
    for (int j = 0; j < PPT; ++j) sj[j] = particle_inv_tau<true>(e, i0 + j);
  }
  StepC k = kc;
  // Steps outside, particles inside: the PPT particles' steps are independent, so the
  // compiler can interleave them whatever the number of steps.  A group whose speeds
  // are all within the shift series (near_shift) runs straight-line code.
  for (int s = 0; s < nsteps; ++s) {
    bool near = true;
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const float v[3] = {vx[j], vy[j], vz[j]};
      near = near && near_shift(k, v);
    }
    if (near) {
#pragma unroll
      for (int j = 0; j < PPT; ++j) {
        if constexpr (TAU) set_inv_tau(k, sj[j]);
        double p[3] = {x[j], y[j], z[j]};
        float v[3] = {vx[j], vy[j], vz[j]}, a[3];
        rk2_step_fast<ACC, true>(k, trig, p, v, a);
        x[j] = p[0]; y[j] = p[1]; z[j] = p[2];
        vx[j] = v[0]; vy[j] = v[1]; vz[j] = v[2];
        if constexpr (ACC) { ax[j] = a[0]; ay[j] = a[1]; az[j] = a[2]; }
      }
    } else {
#pragma unroll
      for (int j = 0; j < PPT; ++j) {
        if constexpr (TAU) set_inv_tau(k, sj[j]);
        double p[3] = {x[j], y[j], z[j]};
        float v[3] = {vx[j], vy[j], vz[j]}, a[3];
        rk2_step_fast<ACC, false>(k, trig, p, v, a);
        x[j] = p[0]; y[j] = p[1]; z[j] = p[2];
        vx[j] = v[0]; vy[j] = v[1]; vz[j] = v[2];
        if constexpr (ACC) { ax[j] = a[0]; ay[j] = a[1]; az[j] = a[2]; }
      }
    }
  }
  store_f64<PPT, VB>(e.px, i0, x);
  store_f64<PPT, VB>(e.py, i0, y);
  store_f64<PPT, VB>(e.pz, i0, z);
  store_f32<PPT, VB>(e.vx, i0, vx);
  store_f32<PPT, VB>(e.vy, i0, vy);
  store_f32<PPT, VB>(e.vz, i0, vz);
  if constexpr (ACC) {
    if (nsteps > 0) {
      store_f32<PPT, VB>(e.ax, i0, ax);
      store_f32<PPT, VB>(e.ay, i0, ay);
      store_f32<PPT, VB>(e.az, i0, az);
    }
  }
}

// Scalar path for the ragged tail: particles i0..i0+cnt-1.
template <bool TAU, bool ACC, class Trig>
__device__ __forceinline__ void step_tail(const EnsArgs& e, const StepC& kc, const Trig& trig, int64_t i0, int cnt,
                                          int nsteps) {
  for (int j = 0; j < cnt; ++j) {
    int64_t i = i0 + j;
    double p[3] = {e.px[i], e.py[i], e.pz[i]};
    float v[3] = {e.vx[i], e.vy[i], e.vz[i]}, a[3] = {0.f, 0.f, 0.f};
    StepC k = kc;
    if constexpr (TAU) set_inv_tau(k, particle_inv_tau<true>(e, i));
    for (int s = 0; s < nsteps; ++s) rk2_step<ACC>(k, trig, p, v, a);
    e.px[i] = p[0]; e.py[i] = p[1]; e.pz[i] = p[2];
    e.vx[i] = v[0]; e.vy[i] = v[1]; e.vz[i] = v[2];
    if constexpr (ACC) {
      if (nsteps > 0) { e.ax[i] = a[0]; e.ay[i] = a[1]; e.az[i] = a[2]; }
    }
  }
}

// The particles [i0, i0 + cnt) of e, cnt <= PPT: the vector path for a full group, the
// scalar path for a ragged one.  Dispatches on the ensemble's tau and acceleration fields.
template <int PPT, int VB, bool TAU, bool ACC, class Trig>
__device__ __forceinline__ void step_span_t(const EnsArgs& e, const StepC& kc, const Trig& trig, int64_t i0,
                                            int64_t cnt, int nsteps) {
  if (cnt >= PPT)
    step_group<PPT, VB, TAU, ACC>(e, kc, trig, i0, nsteps);
  else
    step_tail<TAU, ACC>(e, kc, trig, i0, (int)cnt, nsteps);
}

}  // namespace soax
