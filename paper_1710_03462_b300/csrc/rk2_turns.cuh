// The midpoint-RK2 step of rk2_fast.cuh with the position held between steps as a 64-bit
// fixed-point fraction of a turn, T = frac(x / 2pi) 2^64, for kernels that advance a
// particle several steps in registers.
//
// In this form the periodic box is the integers modulo 2^64: the wrap of x' into
// [0, 2pi) is free, the table index and residual of sin/cos are bit fields of T (no
// reduction per step), and the position update x' = x + dt vm is one 64-bit integer add
// of dt vm converted to 2^-64 turns.  No FP64 instruction runs between the load and the
// store.  2^-64 turn (3.4e-19 rad) is finer than binary64 anywhere in [2^-8, 2pi), so T
// follows x + dt vm more closely than a binary64 position rounded every step; the
// velocity arithmetic (float pairs, f32 rounding of v every step) is the one of
// rk2_fast.cuh, operation for operation.
#pragma once
#include <cstdint>

#include "rk2_fast.cuh"

namespace soax {

// Per-launch constants of the fixed-point update: dt and dt/2 times 2^32 / 2pi as float
// pairs, so dt vm becomes a displacement in units of 2^-32 turn with one float-pair
// product; umax bounds |u_c| over the launch (|A| + |C|, |B| + |A|, |C| + |B|, largest).
struct TurnsK {
  ff dtT, hdtT;
  float umax;
  // A particle whose speeds are all <= vsafe at the start of a call stays within the
  // shift series (|v_c| <= vnear) for every step of it (set per launch from dt, tau and
  // the number of steps by the host; -1: no such guarantee).
  float vsafe;
};

// f (a displacement in units of 2^-32 turn, any magnitude) as 2^-64 turns modulo 2^64,
// rounded to nearest (ties away from zero).  Exact integer arithmetic on the bits of f.
__device__ __forceinline__ uint64_t f_to_turns64(float f) {
  const uint32_t u = __float_as_uint(f);
  const int e = (int)((u >> 23) & 0xFFu);
  if (e == 0) return 0ull;  // zero or subnormal: below 2^-158 turn
  const uint64_t m = (uint64_t)((u & 0x7FFFFFu) | 0x800000u);
  const int sh = e - 118;   // f 2^32 = m 2^(e - 150 + 32)
  uint64_t r;
  if (sh >= 64)
    r = 0ull;               // a multiple of 2^64: whole turns
  else if (sh >= 0)
    r = m << sh;
  else if (sh > -26)
    r = (m + (1ull << (-sh - 1))) >> -sh;
  else
    r = 0ull;               // below half a unit
  return (u >> 31) ? 0ull - r : r;
}

// T + q (mod 2^64) for a displacement q = q.h + q.l in units of 2^-32 turn with
// |q.h| <= 4194000 (|dt vm| <= 6.1e-3 rad) and |q.l| < 1: the float magic-number split
// below is exact up to the rounding of s (2^-56 turn).
__device__ __forceinline__ uint64_t turns_add_fast(uint64_t T, ff q) {
  // t = q.h + 1.5 2^23 lies in [2^23, 2^24), where the float spacing is 1: t - 1.5 2^23
  // is rint(q.h), and its mantissa bits are that integer plus 2^22.
  const float t = __fadd_rn(q.h, 0x1.8p23f);
  const float fq = __fsub_rn(t, 0x1.8p23f);
  const int qi = (int)(__float_as_uint(t) - 0x4B400000u);
  // The rest, s = q.h - rint(q.h) + q.l with |s| < 1.5, as an integer number of 2^-62
  // turns (|s 2^30| < 2^31).
  const float s = __fadd_rn(__fsub_rn(q.h, fq), q.l);
  const int ri = __float2int_rn(__fmul_rn(s, 0x1p30f));
  return T + (uint64_t)(((int64_t)qi << 32) + ((int64_t)ri << 2));
}

// T + q (mod 2^64) for any displacement: turns_add_fast where its bounds hold, else the
// exact conversion of both floats (f_to_turns64).  The pair need not be normalised: q.l
// comes from sums of float-pair products, and where vm = v + (dt/2) a1 cancels it can be
// many ulps of q.h.
__device__ __forceinline__ uint64_t turns_add(uint64_t T, ff q) {
  if (fabsf(q.h) <= 4194000.0f && fabsf(q.l) < 1.0f) return turns_add_fast(T, q);
  return T + f_to_turns64(q.h) + f_to_turns64(q.l);
}

// True when every step of a particle whose speeds are within the shift series
// (|v_c| <= vnear) has a displacement within turns_add_fast's bounds, so such steps need
// no check.  With hs = (dt/2)/tau and |u_c| <= umax:
//   vm = (1 - hs) v + hs u(x),  |vm| <= |1 - hs| vnear + hs umax = b;
//   |q.h| <= dtT b (1 + 2^-23);  |q.l| <= 2^-24 dtT (3 b + 2 hs (umax + vnear))
// (q = dtT vm as a float pair; vm.l holds the two-sum error of vm and the low part of
// hs w0).  Both are taken with margins and compared with 4194000 and 1.
__device__ __forceinline__ bool fast_positions(const StepC& k, const TurnsK& tk) {
  const float hs = k.hs.h;
  const float b = __fmaf_rn(fabsf(1.0f - hs) + 1e-3f, k.vnear, hs * tk.umax) * 1.001f;
  const float qh = tk.dtT.h * b * 1.001f;
  const float ql = tk.dtT.h * 0x1p-24f * (3.0f * b + 2.0f * hs * (tk.umax + k.vnear)) * 1.1f;
  return qh <= 4194000.0f && ql < 1.0f;
}

// x = 2 pi T 2^-64 in binary64, wrapped once into [0, 2pi).  T = Th 2^32 + Tl; 2 pi 2^-32
// as a double pair (C1H + C1L), so the only rounding that matters is the last one.
__device__ __forceinline__ double turns_to_x(uint64_t T) {
  const double th = (double)(uint32_t)(T >> 32), tl = (double)(uint32_t)T;  // exact
  const double x = __fma_rn(th, 0x1.921fb54442d18p-30,
                            __fma_rn(th, 0x1.1a62633145c07p-84, __dmul_rn(tl, 0x1.921fb54442d18p-62)));
  // A T just below 2^64 can round to the binary64 2pi itself: wrap it as the step does.
  return x >= SOAX_TWO_PI ? __dsub_rn(x, SOAX_TWO_PI) : x;
}

// One step of the particle (T, v): the arithmetic of rk2_step_fast, with the midpoint of a
// long shift and the new position formed in turns.  NEAR: every |v_c| <= vnear and
// fast_positions hold (checked by the caller); otherwise each coordinate takes the series
// or the table at the midpoint, and each displacement is checked.
// FAST (with NEAR): fast_positions holds, so the position update takes turns_add_fast
// without a check (the same bits as turns_add there).
template <bool ACC, bool NEAR, class Trig, bool FAST = NEAR>
__device__ __forceinline__ void rk2_step_turns(const StepC& k, const TurnsK& tk, const Trig& trig, uint64_t T[3],
                                               float v[3], float a2out[3]) {
  ff P[3], Q[3], dP[3], dQ[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    int idx;
    ff r;
    turns_angle(T[c], idx, r);
    sincos_tab(trig(c, idx), r, P[c], Q[c]);
    if (NEAR || fabsf(v[c]) <= k.vnear) {
      sincos_delta(P[c], Q[c], ff_mul_f(k.hdt, v[c]), dP[c], dQ[c]);
    } else {
      ff P1, Q1;
      turns_angle(turns_add(T[c], ff_mul_f(tk.hdtT, v[c])), idx, r);
      sincos_tab(trig(c, idx), r, P1, Q1);
      dP[c] = ff_sub(P1, P[c]);
      dQ[c] = ff_sub(Q1, Q[c]);
    }
  }
  const ff u0[3] = {ff_add(P[2], Q[1]), ff_add(P[0], Q[2]), ff_add(P[1], Q[0])};
  const ff du[3] = {ff_add(dP[2], dQ[1]), ff_add(dP[0], dQ[2]), ff_add(dP[1], dQ[0])};
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
    if constexpr (FAST)
      T[c] = turns_add_fast(T[c], ff_mul(tk.dtT, vm));
    else
      T[c] = turns_add(T[c], ff_mul(tk.dtT, vm));
  }
  v[0] = vn[0];
  v[1] = vn[1];
  v[2] = vn[2];
}

// The amplitude-scaled sines and cosines of the three coordinates of the position T
// (P0, Q0) and of the midpoint T + (dt/2) v (P1, Q1): the shift series, or the table at
// the midpoint for a long shift, chosen per coordinate as in rk2_step_turns (NEAR: the
// caller has checked near_shift).
template <bool NEAR, class Trig>
__device__ __forceinline__ void step_trig_turns(const StepC& k, const TurnsK& tk, const Trig& trig, const uint64_t T[3],
                                                const float v[3], ff P0[3], ff Q0[3], ff P1[3], ff Q1[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    int idx;
    ff r;
    turns_angle(T[c], idx, r);
    sincos_tab(trig(c, idx), r, P0[c], Q0[c]);
    if (NEAR || fabsf(v[c]) <= k.vnear) {
      sincos_shift(P0[c], Q0[c], ff_mul_f(k.hdt, v[c]), P1[c], Q1[c]);
    } else {
      turns_angle(turns_add(T[c], ff_mul_f(tk.hdtT, v[c])), idx, r);
      sincos_tab(trig(c, idx), r, P1[c], Q1[c]);
    }
  }
}

}  // namespace soax
