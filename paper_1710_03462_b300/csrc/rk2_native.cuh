// Per-particle midpoint-RK2 step of an inertial particle in the ABC flow, in native
// binary64 arithmetic (CUDA's f64 sincos), and its reverse-mode derivative.  Every
// multiply and add of the forward step is an explicitly rounded intrinsic, so the
// compiler cannot contract or reorder them.
//
//   u(x)   = (A sin z + C cos y, B sin x + A cos z, C sin y + B cos x)
//   a1     = (u(x) - v) / tau
//   xm     = x + (dt/2) v            (fused multiply-add)
//   vm     = v + (dt/2) a1
//   a2     = (u(xm) - vm) / tau
//   x'     = x + dt vm               (fused multiply-add), wrapped once into [0, 2pi)
//   v'     = v + dt a2, rounded to f32
//
// Generalises the Euler advection x += dt*v of Eq. 1 (Sec. 2) to inertial particles.
#pragma once
#include <cstdint>

namespace soax {

#define SOAX_TWO_PI 6.283185307179586  // binary64 nearest to 2pi (0x401921FB54442D18)

struct FlowK {
  double A, B, C;
  double dt, hdt;     // hdt = dt/2 (exact)
  float2 dtf, hdtf;   // dt and dt/2 as float pairs (hi, lo)
};

__device__ __forceinline__ void abc_flow_native(const FlowK& f, const double x[3], double u[3]) {
  double sx, cx, sy, cy, sz, cz;
  sincos(x[0], &sx, &cx);
  sincos(x[1], &sy, &cy);
  sincos(x[2], &sz, &cz);
  u[0] = __dadd_rn(__dmul_rn(f.A, sz), __dmul_rn(f.C, cy));
  u[1] = __dadd_rn(__dmul_rn(f.B, sx), __dmul_rn(f.A, cz));
  u[2] = __dadd_rn(__dmul_rn(f.C, sy), __dmul_rn(f.B, cx));
}

__device__ __forceinline__ double wrap_2pi(double x) {
  if (x >= SOAX_TWO_PI) return __dsub_rn(x, SOAX_TWO_PI);
  if (x < 0.0) return __dadd_rn(x, SOAX_TWO_PI);
  return x;
}

// One step.  x: f64 position (in/out); v: stored f32 velocity (in/out);
// a2out: the last stage acceleration rounded to f32 (out).
__device__ __forceinline__ void rk2_step_native(const FlowK& f, double inv_tau, double x[3], float v[3],
                                                float a2out[3]) {
  double vd[3] = {(double)v[0], (double)v[1], (double)v[2]};
  double u0[3], u1[3], a1[3], xm[3], vm[3];
  abc_flow_native(f, x, u0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    a1[c] = __dmul_rn(__dsub_rn(u0[c], vd[c]), inv_tau);
    xm[c] = __fma_rn(f.hdt, vd[c], x[c]);
    vm[c] = __dadd_rn(vd[c], __dmul_rn(f.hdt, a1[c]));
  }
  abc_flow_native(f, xm, u1);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double a2 = __dmul_rn(__dsub_rn(u1[c], vm[c]), inv_tau);
    x[c] = wrap_2pi(__fma_rn(f.dt, vm[c], x[c]));
    v[c] = __double2float_rn(__dadd_rn(vd[c], __dmul_rn(f.dt, a2)));
    a2out[c] = __double2float_rn(a2);
  }
}

// Vector-Jacobian product of the flow at x: xb += J(x)^T ub and th[0..2] +=
// (du/d(A,B,C))(x)^T ub, with J = [[0, -C sin y, A cos z], [B cos x, 0, -A sin z],
// [-B sin x, C cos y, 0]], du/dA = (sin z, cos z, 0), du/dB = (0, sin x, cos x),
// du/dC = (cos y, 0, sin y).
__device__ __forceinline__ void abc_vjp_native(const FlowK& f, const double x[3], const double ub[3], double xb[3],
                                               double th[4]) {
  double sx, cx, sy, cy, sz, cz;
  sincos(x[0], &sx, &cx);
  sincos(x[1], &sy, &cy);
  sincos(x[2], &sz, &cz);
  xb[0] += f.B * cx * ub[1] - f.B * sx * ub[2];
  xb[1] += -f.C * sy * ub[0] + f.C * cy * ub[2];
  xb[2] += f.A * cz * ub[0] - f.A * sz * ub[1];
  th[0] += sz * ub[0] + cz * ub[1];
  th[1] += sx * ub[1] + cx * ub[2];
  th[2] += cy * ub[0] + sy * ub[2];
}

// Reverse of one step: given the adjoints (xb, vb) of (x', v'), overwrite them with the
// adjoints of (x, v) and accumulate d/d(A, B, C, tau) into th.  (x, vf) is the state
// before the step.  The f32 rounding of v' and the periodic wrap are differentiated as
// the identity.  Reverse-mode differentiation of the statements above, last first:
//   x' = x + dt vm:       xb += xb',  vmb = dt xb'
//   v' = v + dt a2:       vb += vb',  a2b = dt vb'
//   a2 = (u(xm) - vm) s:  u1b = s a2b,  vmb -= s a2b,  sb += a2b . (u1 - vm)
//   u1 = u(xm):           xmb = J(xm)^T u1b,  thb += (du/dtheta)(xm)^T u1b
//   vm = v + dt/2 a1:     vb += vmb,  a1b = dt/2 vmb
//   xm = x + dt/2 v:      xb += xmb,  vb += dt/2 xmb
//   a1 = (u(x) - v) s:    u0b = s a1b,  vb -= s a1b,  sb += a1b . (u0 - v)
//   u0 = u(x):            xb += J(x)^T u0b,  thb += (du/dtheta)(x)^T u0b
//   s = 1/tau:            taub = -s^2 sb
__device__ __forceinline__ void rk2_reverse_native(const FlowK& f, double s, const double x[3], const float vf[3],
                                                   double xb[3], double vb[3], double th[4]) {
  const double v[3] = {(double)vf[0], (double)vf[1], (double)vf[2]};
  double u0[3], u1[3], xm[3], vm[3];
  abc_flow_native(f, x, u0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double a1 = __dmul_rn(__dsub_rn(u0[c], v[c]), s);
    xm[c] = __fma_rn(f.hdt, v[c], x[c]);
    vm[c] = __dadd_rn(v[c], __dmul_rn(f.hdt, a1));
  }
  abc_flow_native(f, xm, u1);
  double sb = 0.0, u1b[3], vmb[3], xmb[3] = {0.0, 0.0, 0.0}, u0b[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double a2b = f.dt * vb[c];
    u1b[c] = s * a2b;
    vmb[c] = f.dt * xb[c] - s * a2b;
    sb += a2b * (u1[c] - vm[c]);
  }
  abc_vjp_native(f, xm, u1b, xmb, th);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double a1b = f.hdt * vmb[c];
    vb[c] += vmb[c] + f.hdt * xmb[c];
    xb[c] += xmb[c];
    u0b[c] = s * a1b;
    vb[c] -= s * a1b;
    sb += a1b * (u0[c] - v[c]);
  }
  abc_vjp_native(f, x, u0b, xb, th);
  th[3] -= s * s * sb;
}

}  // namespace soax
