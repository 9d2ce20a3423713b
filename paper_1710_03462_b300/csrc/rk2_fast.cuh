// Per-particle midpoint-RK2 step of an inertial particle in the ABC flow, and its
// reverse-mode derivative:
//
//   u(x)   = (A sin z + C cos y, B sin x + A cos z, C sin y + B cos x)
//   a1     = (u(x) - v) / tau,      xm = x + (dt/2) v,      vm = v + (dt/2) a1
//   a2     = (u(xm) - vm) / tau
//   x'     = x + dt vm, wrapped once into [0, 2pi);   v' = v + dt a2, rounded to f32
//
// (the Euler advection x += dt*v of Eq. 1, Sec. 2, generalised to inertial particles),
// evaluated to binary64 accuracy without the FP64 pipe for the trigonometry and the
// velocity arithmetic.
//
// B300 executes FP64 at a small fraction of its FP32 and integer rates (measured: one to
// 1.6 FP64 FMA lanes per SM per clock against ~124 FP32 FMA lanes), and a native binary64 sincos
// costs ~25 FP64 instructions; the native step is therefore bound by the FP64 pipe at a
// few percent of HBM bandwidth.  Here:
//
//  * real numbers are float-float pairs (hi + lo, ~48 significant bits), built from the
//    error-free transformations two_sum (Knuth) and two_prod (via FMA), all with
//    explicitly rounded intrinsics so the compiler cannot contract or reassociate them;
//  * sin/cos of a position x in [0, 2pi) use an exact fixed-point reduction: x (binary64)
//    becomes a 64-bit integer X = x 2^61, T = X (4/pi) 2^-63 is frac(x / 2pi) in 2^-64
//    turns, its top 11 bits select theta_k = 2 pi k / 2048 from a float-float table and
//    the rest is the residual r = x - theta_k (|r| <= pi/2048) as a float pair; then
//    sin(theta_k + r) = S + (C sin r + S (cos r - 1)) with short Taylor series for the
//    residual (a table-driven method in the manner of Tang);
//  * each coordinate enters u with one amplitude (x with B, y with C, z with A), so the
//    table entries are read pre-scaled (P = a sin, Q = a cos), and u(xm) - u(x) is the
//    same combination of the changes of P and Q over the shift delta = (dt/2) v from the
//    angle addition formula (|delta| <= 2^-9; longer shifts take the table at xm);
//  * the new velocity v + dt a2 is rounded to f32 from the float pair correctly (rounding
//    to odd, round_sum_f32); the new position is x + dt vm with vm = vm_hi + vm_lo
//    applied as two binary64 FMAs (the only FP64 instructions of the step).
//
// Accuracy (checked against the CPU oracle by the parity tests and against a long-double
// evaluation of the step on the host): sin/cos to ~5e-15 absolute (the 2^-48 precision
// of a float pair); the flow enters v' scaled by dt/tau, so at dt/tau = 0.01 the velocity
// before its f32 rounding is within ~1.2e-15 absolute (rms 1e-16) of the exact step, and
// positions are within about one binary64 ulp per step.
#pragma once
#include <cstdint>

#include "trig_table.inc"

namespace soax {

#define SOAX_TWO_PI 6.283185307179586  // binary64 nearest to 2pi (0x401921FB54442D18)

// Step parameters shared by every particle of a launch.
struct FlowK {
  double A, B, C;
  double dt, hdt;     // hdt = dt/2 (exact)
  float2 dtf, hdtf;   // dt and dt/2 as float pairs (hi, lo)
};

struct ff {
  float h, l;  // the value h + l
};

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// Requires |a| >= |b| or a == 0.
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  ff p = two_prod(a.h, b.h);
  p.l = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l));
  return p;
}

__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  ff p = two_prod(a.h, b);
  p.l = __fmaf_rn(a.l, b, p.l);
  return p;
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = two_sum(a.h, b.h);
  s.l = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
  return s;
}

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff{-b.h, -b.l}); }

// a + b when |a.h| >= |b.h| or a.h == 0 (Dekker's fast two-sum on the high parts).
__device__ __forceinline__ ff ff_add_ordered(ff a, ff b) {
  ff s = fast_two_sum(a.h, b.h);
  s.l = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
  return s;
}

__device__ __forceinline__ ff ff_add_f(ff a, float b) {
  ff s = two_sum(a.h, b);
  s.l = __fadd_rn(s.l, a.l);
  return s;
}

// Exact conversion of a binary32 to binary64 with integer instructions (zero and
// subnormal inputs give a signed zero).
__device__ __forceinline__ double f2d_exact(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFFu;
  uint32_t hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u >> 3) & 0xFFFFFu);
  uint32_t lo = u << 29;
  if (e == 0) {
    hi = u & 0x80000000u;
    lo = 0;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// Per-particle constants of the step, as float pairs.
struct StepC {
  ff dt, hdt;    // dt and dt/2
  ff s;          // 1/tau
  ff hs, ds, gh; // (dt/2)/tau, dt/tau and 1 - (dt/2)/tau (set_inv_tau)
  double dt_d;   // dt as binary64, for the position update
  float vnear;   // SOAX_SHIFT_MAX / (dt/2): the speeds the shift series covers
};

__device__ __forceinline__ ff ff_from2(const float2 p) { return ff{p.x, p.y}; }

// 1/(ts * m) as a float pair (one Newton step on a correctly rounded float reciprocal).
__device__ __forceinline__ ff ff_inv_tau(const float2 ts, float m) {
  const ff t = ff_mul_f(ff_from2(ts), m);
  const float y0 = __frcp_rn(t.h);
  const float e = __fsub_rn(__fmaf_rn(-t.h, y0, 1.0f), __fmul_rn(t.l, y0));
  return fast_two_sum(y0, __fmul_rn(y0, e));
}

// s = 1/tau and the products of the update that depend on it alone.
__device__ __forceinline__ void set_inv_tau(StepC& k, ff s) {
  k.s = s;
  k.hs = ff_mul(k.hdt, s);
  k.ds = ff_mul(k.dt, s);
  k.gh = ff_add_f(ff{-k.hs.h, -k.hs.l}, 1.0f);
}

// frac(x / 2pi) 2^64 for a binary64 x with 0 <= x < 8: the position as a 64-bit
// fixed-point fraction of a turn (within 3 units of 2^-64 turn).
__device__ __forceinline__ uint64_t to_turns(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const int e = (int)((hi >> 20) & 0x7FFu);
  const uint64_t m = ((uint64_t)((hi & 0xFFFFFu) | 0x100000u) << 32) | lo;
  const int sh = e - 1014;  // X = x 2^61 = m 2^(e - 1075 + 61)
  uint64_t X;
  if (sh >= 0)
    X = m << sh;  // exact: x >= 2^-8 and x < 8 give 0 <= sh <= 11
  else
    X = sh > -64 ? (m >> -sh) : 0ull;  // bits below 2^-61 dropped (< 5e-19)
  // T = X (4/pi) 2^-63 = frac(x / 2pi) 2^64 (within 3 units of the last place).
  return __umul64hi(X, SOAX_FOUR_OVER_PI_2P63) << 1;
}

// Angle T (2^-64 turns) -> table index k and residual r = 2 pi T 2^-64 - 2 pi k / 2048
// in radians (|r| <= pi/2048) as a float pair.
__device__ __forceinline__ void turns_angle(uint64_t T, int& k, ff& r) {
  const uint64_t U = T + (1ull << 52);
  k = (int)(U >> 53) & (SOAX_TRIG_TABLE_SIZE - 1);
  // rho = U mod 2^53 = residual + 2^52 in 2^-64 turns, 0 <= rho < 2^53.  Its bits 30..52
  // and 7..29 are converted exactly by planting each in a float mantissa; the 7 bits
  // below are dropped (less than 2^-57 turn = 5e-17 rad).
  const uint32_t rl = (uint32_t)U, rh = (uint32_t)(U >> 32);
  const uint32_t chi = __funnelshift_r(rl, rh, 30) & 0x7FFFFFu;
  const uint32_t clo = (rl >> 7) & 0x7FFFFFu;
  const float fhi = __fsub_rn(__uint_as_float(0x5A000000u | chi), 0x1.8p53f);  // chi 2^30 - 2^52
  const float flo = __fsub_rn(__uint_as_float(0x4E800000u | clo), 0x1p30f);    // clo 2^7
  const ff rt = {fhi, flo};
  r = ff_mul(rt, ff{SOAX_TWO_PI_2M64_HI, SOAX_TWO_PI_2M64_LO});
}

// x (binary64, 0 <= x < 8) -> table index k and residual r = x - 2 pi k / 2048.
__device__ __forceinline__ void reduce_angle(double x, int& k, ff& r) { turns_angle(to_turns(x), k, r); }

// amp times the table entry t = (sin, cos) as float pairs, packed like the entry.
__device__ __forceinline__ float4 scale_entry(ff amp, float4 t) {
  const ff a = ff_mul(amp, ff{t.x, t.y}), b = ff_mul(amp, ff{t.z, t.w});
  return make_float4(a.h, a.l, b.h, b.l);
}

// Each coordinate enters u with one amplitude, for its sine and its cosine alike:
// x with B, y with C, z with A.  The forward step therefore reads amplitude-scaled
// entries P = a sin, Q = a cos, from one of two sources that give identical bits:
// three tables scaled once per block, or the plain table scaled per lookup.
struct TrigScaled {
  const float4* __restrict__ t;  // 3 x SOAX_TRIG_TABLE_SIZE entries: x, y, z
  __device__ __forceinline__ float4 operator()(int c, int k) const { return t[c * SOAX_TRIG_TABLE_SIZE + k]; }
};
struct TrigPlain {
  const float4* __restrict__ t;  // the plain table: unscaled sin and cos for every coordinate
  __device__ __forceinline__ float4 operator()(int, int k) const { return t[k]; }
};
struct TrigUnscaled {
  const float4* __restrict__ t;  // the plain table
  ff amp[3];                     // B, C, A
  __device__ __forceinline__ float4 operator()(int c, int k) const { return scale_entry(amp[c], t[k]); }
};

// a sin and a cos of theta_k + r from the entry (S, C) = (a sin theta_k, a cos theta_k)
// of a table scaled by the amplitude a (a = 1: the plain table), |r| <= pi/2048.
// m = -r^2/2 as a float pair, and from it cos r - 1 = m + m^2/6 and sin r = r + m r/3
// (r^6/720 < 2e-20 and r^5/120 < 8e-17 dropped; m^2/6 < 3e-13 and m r/3 < 6e-10 are
// exact enough in float: errors < 4e-17).  -r.h/2 is exact, so two_prod(r.h, -r.h/2)
// is r.h^2 (-1/2) exactly, and -r.h r.l adds the cross term.
__device__ __forceinline__ void series_terms(ff r, ff& cm, ff& sr) {
  ff m = two_prod(r.h, __fmul_rn(-0.5f, r.h));
  m.l = __fmaf_rn(-r.h, r.l, m.l);
  cm = ff{m.h, __fmaf_rn(__fmul_rn(m.h, 1.0f / 6.0f), m.h, m.l)};
  sr = ff{r.h, __fmaf_rn(__fmul_rn(m.h, r.h), 1.0f / 3.0f, r.l)};
}

__device__ __forceinline__ void sincos_tab(const float4 t, ff r, ff& s, ff& c) {
  ff cm, sr;  // cos r - 1, sin r
  series_terms(r, cm, sr);
  // Every entry of the plain table is 0 or at least sin(2pi/2048) = 3.07e-3 in magnitude
  // while |r| <= pi/2048 = 1.54e-3, so in each sum below the first term is zero or the
  // larger one: |S|, |C| > |C sr|, |S sr| >= 3.07e-3 |r| > r^2/2 >= |S cm|, |C cm|.  A
  // common amplitude scales every term alike and keeps the order.
  const ff S = {t.x, t.y}, C = {t.z, t.w};
  const ff Ssr = ff_mul(S, sr), Csr = ff_mul(C, sr);
  s = ff_add_ordered(S, ff_add_ordered(Csr, ff_mul(S, cm)));
  c = ff_add_ordered(C, ff_add_ordered(ff{-Ssr.h, -Ssr.l}, ff_mul(C, cm)));
}

// The changes of sin and cos from a to a + d, given those at a, |d| <= ~2e-3:
//   sin(a + d) - sin a = cos a sin d + sin a (cos d - 1)  -> qs
//   cos(a + d) - cos a = cos a (cos d - 1) - sin a sin d  -> qc
__device__ __forceinline__ void sincos_delta(ff sa, ff ca, ff d, ff& qs, ff& qc) {
  // cos d - 1 and sin d by the series of series_terms (d^5/120 < 2e-16 relative, dropped)
  ff cmd, sd;
  series_terms(d, cmd, sd);
  qs = ff_add(ff_mul(ca, sd), ff_mul(sa, cmd));
  qc = ff_sub(ff_mul(ca, cmd), ff_mul(sa, sd));
}

// sin and cos of a + d from those of a, |d| <= ~2e-3 (or both times one amplitude: the
// formulas are linear in sa, ca).
__device__ __forceinline__ void sincos_shift(ff sa, ff ca, ff d, ff& s, ff& c) {
  // cos d - 1 and sin d by the series of series_terms (d^5/120 < 2e-16 relative, dropped)
  ff cmd, sd;
  series_terms(d, cmd, sd);
  s = ff_add(sa, ff_add(ff_mul(ca, sd), ff_mul(sa, cmd)));
  c = ff_add(ca, ff_sub(ff_mul(ca, cmd), ff_mul(sa, sd)));
}

__device__ __forceinline__ double wrap_2pi_fast(double x) {
  const long long b = __double_as_longlong(x);
  if (b >= 0x401921FB54442D18ll) return __dsub_rn(x, 6.283185307179586);   // x >= 2pi
  if (b < 0 && b != (long long)0x8000000000000000ull) return __dadd_rn(x, 6.283185307179586);  // x < 0
  return x;
}

// The series of sincos_delta / sincos_shift hold for |delta| <= SOAX_SHIFT_MAX (their first
// dropped terms, delta^5/120 and delta^6/720, stay below 2.5e-16); a longer shift takes
// the table at the midpoint itself.
#define SOAX_SHIFT_MAX 0x1p-9f

// xm = x + (dt/2) v as binary64 (one rounding, as the binary64 arithmetic forms it),
// reduced into [0, 2pi] for reduce_angle with a two-part 2pi (Cody and Waite).
__device__ __forceinline__ double far_midpoint(double dt, double x, float v) {
  double xm = __fma_rn(0.5 * dt, f2d_exact(v), x);
  const double q = floor(xm * 0x1.45f306dc9c883p-3);  // xm / 2pi
  xm = __fma_rn(-q, 0x1.921fb54442d18p+2, xm);
  xm = __fma_rn(-q, 0x1.1a62633145c07p-52, xm);
  return xm < 0.0 ? xm + SOAX_TWO_PI : xm;
}

// u = (A sin z + C cos y, B sin x + A cos z, C sin y + B cos x).  SCALED: from the
// amplitude-scaled sines and cosines P_c = a_c sin x_c, Q_c = a_c cos x_c (a = (B, C, A));
// otherwise P, Q are sin and cos and amp = (B, C, A) multiplies them in.
template <bool SCALED>
__device__ __forceinline__ void abc_u(const ff amp[3], const ff P[3], const ff Q[3], ff u[3]) {
  if constexpr (SCALED) {
    u[0] = ff_add(P[2], Q[1]);
    u[1] = ff_add(P[0], Q[2]);
    u[2] = ff_add(P[1], Q[0]);
  } else {
    u[0] = ff_add(ff_mul(amp[2], P[2]), ff_mul(amp[1], Q[1]));
    u[1] = ff_add(ff_mul(amp[0], P[0]), ff_mul(amp[2], Q[2]));
    u[2] = ff_add(ff_mul(amp[1], P[1]), ff_mul(amp[0], Q[0]));
  }
}

// One step: x (binary64 position, in/out), v (f32 velocity, in/out), a2out (the last
// stage acceleration rounded to f32, computed when ACC).  trig gives the amplitude-scaled
// table entries.  With P_c = a_c sin x_c, Q_c = a_c cos x_c (a = (B, C, A)),
//   u(x) = (P_z + Q_y, P_x + Q_z, P_y + Q_x),
// and u(xm) - u(x) is the same combination of the changes dP, dQ over the shift
// (dt/2) v (sincos_delta), so sin and cos of xm are never formed.  Then, with
// w0 = u(x) - v, hs = (dt/2)/tau, ds = dt/tau:
//   vm = v + hs w0,   u(xm) - vm = (1 - hs) w0 + du,   v' = v + ds (u(xm) - vm).
// RN32(v + t.h + t.l), correctly rounded: v + t.h = s + e exactly (two_sum), e + t.l
// is rounded to odd (toward zero, last bit set when inexact), and rounding s plus that
// to nearest gives the rounding of the exact sum (Boldo and Melquiond, rounding to odd:
// a rounding boundary of s is a short binary fraction, even at the precision of e + t.l,
// so it can neither equal the odd value nor fall between it and e + t.l).
__device__ __forceinline__ float round_sum_f32(float v, ff t) {
  const ff se = two_sum(v, t.h);
  const float up = __fadd_ru(se.l, t.l), dn = __fadd_rd(se.l, t.l);
  const float z = fabsf(up) < fabsf(dn) ? up : dn;
  const float odd = __uint_as_float(__float_as_uint(z) | (up != dn ? 1u : 0u));
  return __fadd_rn(se.h, odd);
}

// The update from u(x) - v = w0 and du = u(xm) - u(x) (shared by the two paths below).
template <bool ACC>
__device__ __forceinline__ void rk2_update(const StepC& k, const ff u0[3], const ff du[3], double x[3], float v[3],
                                           float a2out[3]) {
  float vn[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const ff w0 = ff_add_f(u0[c], -v[c]);
    const ff vm = ff_add_f(ff_mul(k.hs, w0), v[c]);
    const ff w1 = ff_add(ff_mul(k.gh, w0), du[c]);  // u(xm) - vm
    vn[c] = round_sum_f32(v[c], ff_mul(k.ds, w1));
    if constexpr (ACC) {
      const ff a2 = ff_mul(k.s, w1);
      a2out[c] = __fadd_rn(a2.h, a2.l);
    }
    double xn = __fma_rn(k.dt_d, f2d_exact(vm.h), x[c]);
    xn = __fma_rn(k.dt_d, f2d_exact(vm.l), xn);
    x[c] = wrap_2pi_fast(xn);
  }
  v[0] = vn[0];
  v[1] = vn[1];
  v[2] = vn[2];
}

// True when every component of v is short enough for the shift series: |v_c| <= vnear
// = SOAX_SHIFT_MAX / (dt/2).  The same test picks each coordinate's path below, so a
// particle gets the same bits whether its group took the NEAR path or not.
__device__ __forceinline__ bool near_shift(const StepC& k, const float v[3]) {
  return fmaxf(fabsf(v[0]), fmaxf(fabsf(v[1]), fabsf(v[2]))) <= k.vnear;
}

// NEAR: the caller has checked near_shift (straight-line code); otherwise each
// coordinate takes the series or, for a long shift, the table at the midpoint itself.
template <bool ACC, bool NEAR, class Trig>
__device__ __forceinline__ void rk2_step_fast(const StepC& k, const Trig& trig, double x[3], float v[3],
                                              float a2out[3]) {
  ff P[3], Q[3], dP[3], dQ[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    int idx;
    ff r;
    reduce_angle(x[c], idx, r);
    sincos_tab(trig(c, idx), r, P[c], Q[c]);
    if (NEAR || fabsf(v[c]) <= k.vnear) {
      sincos_delta(P[c], Q[c], ff_mul_f(k.hdt, v[c]), dP[c], dQ[c]);
    } else {
      ff P1, Q1;
      reduce_angle(far_midpoint(k.dt_d, x[c], v[c]), idx, r);
      sincos_tab(trig(c, idx), r, P1, Q1);
      dP[c] = ff_sub(P1, P[c]);
      dQ[c] = ff_sub(Q1, Q[c]);
    }
  }
  const ff u0[3] = {ff_add(P[2], Q[1]), ff_add(P[0], Q[2]), ff_add(P[1], Q[0])};
  const ff du[3] = {ff_add(dP[2], dQ[1]), ff_add(dP[0], dQ[2]), ff_add(dP[1], dQ[0])};
  rk2_update<ACC>(k, u0, du, x, v, a2out);
}

// xb += J(x)^T ub and G[0..2] += (w du/dA, w du/dB, w du/dC)^T ub at the point whose
// sines and cosines are P, Q.  SCALED: P_c = a_c sin x_c, Q_c = a_c cos x_c (a = (B, C, A))
// and the weights w are the amplitudes (A, B, C); otherwise P, Q are sin and cos, w = 1
// and amp = (B, C, A) multiplies each column of J.  In the scaled form
// J = [[0, -P_y, Q_z], [Q_x, 0, -P_z], [-P_x, Q_y, 0]], A du/dA = (P_z, Q_z, 0),
// B du/dB = (0, P_x, Q_x), C du/dC = (Q_y, 0, P_y): each coordinate's four products serve
// its column of J and its amplitude's gradient.
template <bool SCALED>
__device__ __forceinline__ void abc_vjp(const ff amp[3], const ff P[3], const ff Q[3], const ff ub[3], ff xb[3],
                                        ff G[4]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    // coordinate c enters u_{c+1} as a sine (P) and u_{c+2} as a cosine (Q), indices mod 3
    const int p = c == 2 ? 0 : c + 1, q = c == 0 ? 2 : c - 1;
    ff col = ff_sub(ff_mul(Q[c], ub[p]), ff_mul(P[c], ub[q]));
    if constexpr (!SCALED) col = ff_mul(amp[c], col);
    xb[c] = ff_add(xb[c], col);
    // the amplitude of coordinate c: x -> B (G[1]), y -> C (G[2]), z -> A (G[0])
    const int g = c == 2 ? 0 : c + 1;
    G[g] = ff_add(G[g], ff_add(ff_mul(P[c], ub[p]), ff_mul(Q[c], ub[q])));
  }
}

// Reverse of one step: given the adjoints (xb, vb) of (x', v'), overwrite them with the
// adjoints of (x, v), and accumulate into G the parameter gradients G[0..2] (w dL/dA,
// w dL/dB, w dL/dC with the weights of abc_vjp) and the sum G[3] = S with dL/ds = dt S
// (s = 1/tau); the caller finishes them once per particle.  (x, v) is the state before the
// step, given by v and the sines and cosines at x (P0, Q0) and at xm = x + (dt/2) v
// (P1, Q1), amplitude-scaled when SCALED.  The f32 rounding of v' and the periodic wrap are
// differentiated as the identity.  With hs = (dt/2) s, ds = dt s, d0 = u(x) - v,
// d1 = u(xm) - vm, the step's statements in reverse order:
//   x' = x + dt vm:       xb += xb',  vmb = dt xb'
//   v' = v + ds d1:       vb += vb',  u1b = ds vb',  vmb -= ds vb',  S += vb' . d1
//   u1 = u(xm):           xmb = J(xm)^T u1b,  G += (w du/dtheta)(xm)^T u1b
//   vm = v + hs d0:       vb += vmb,  u0b = hs vmb,  vb -= hs vmb,  S += vmb . d0 / 2
//   xm = x + (dt/2) v:    xb += xmb,  vb += (dt/2) xmb
//   u0 = u(x):            xb += J(x)^T u0b,  G += (w du/dtheta)(x)^T u0b
template <bool SCALED>
__device__ __forceinline__ void rk2_reverse_core(const StepC& k, const ff amp[3], const ff P0[3], const ff Q0[3],
                                                 const ff P1[3], const ff Q1[3], const float v[3], ff xb[3], ff vb[3],
                                                 ff G[4]) {
  ff u0[3], u1[3];
  abc_u<SCALED>(amp, P0, Q0, u0);
  abc_u<SCALED>(amp, P1, Q1, u1);
  ff d0[3], u1b[3], vmb[3], xmb[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    d0[c] = ff_add_f(u0[c], -v[c]);
    const ff vm = ff_add_f(ff_mul(k.hs, d0[c]), v[c]);
    const ff d1 = ff_sub(u1[c], vm);
    u1b[c] = ff_mul(k.ds, vb[c]);
    vmb[c] = ff_sub(ff_mul(k.dt, xb[c]), u1b[c]);
    G[3] = ff_add(G[3], ff_mul(vb[c], d1));
  }
  abc_vjp<SCALED>(amp, P1, Q1, u1b, xmb, G);
  ff u0b[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    u0b[c] = ff_mul(k.hs, vmb[c]);
    vb[c] = ff_sub(ff_add(vb[c], ff_add(vmb[c], ff_mul(k.hdt, xmb[c]))), u0b[c]);
    xb[c] = ff_add(xb[c], xmb[c]);
    G[3] = ff_add(G[3], ff_mul(ff{__fmul_rn(0.5f, vmb[c].h), __fmul_rn(0.5f, vmb[c].l)}, d0[c]));
  }
  abc_vjp<SCALED>(amp, P0, Q0, u0b, xb, G);
}

static __device__ const float4 kTrigTable[SOAX_TRIG_TABLE_SIZE] = {SOAX_TRIG_TABLE_ENTRIES};

// Copy the table (32 KB) into shared memory (every thread of the block must call this).
__device__ __forceinline__ void load_trig_table(float4* s_tab) {
  for (int i = threadIdx.x; i < SOAX_TRIG_TABLE_SIZE; i += blockDim.x) s_tab[i] = kTrigTable[i];
  __syncthreads();
}

constexpr int kScaledTrigBytes = 3 * SOAX_TRIG_TABLE_SIZE * 16;  // 96 KB

// Fill the three amplitude-scaled tables (x with B, y with C, z with A) in shared memory
// (every thread of the block must call this).
__device__ __forceinline__ void load_scaled_trig_tables(float4* s_tab, ff A, ff B, ff C) {
  for (int i = threadIdx.x; i < 3 * SOAX_TRIG_TABLE_SIZE; i += blockDim.x) {
    const int c = i / SOAX_TRIG_TABLE_SIZE;
    const ff amp = c == 0 ? B : (c == 1 ? C : A);
    s_tab[i] = scale_entry(amp, kTrigTable[i - c * SOAX_TRIG_TABLE_SIZE]);
  }
  __syncthreads();
}

}  // namespace soax
