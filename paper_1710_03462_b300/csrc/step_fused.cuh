// Kernel template of soax_step_fused: each thread loads groups of PPT particles once,
// advances them nsteps midpoint-RK2 steps in registers (positions as 64-bit fixed-point
// turns, rk2_turns.cuh) and stores them once; optionally with the cell keys of the final
// positions (cell_key.cuh, the definition soax_cell_keys uses) written beside them.
#pragma once
#include <cstdint>

#include "cell_key.cuh"
#include "rk2_turns.cuh"
#include "soax_internal.h"
#include "step_core.cuh"

namespace soax {

// The cell key of a particle whose position is held as turns T and stored as
// x = turns_to_x(T), without waiting for x: with y = G T 2^-64 (G <= 1024), the stored
// binary64 x (within 2^-53 relative of 2 pi T 2^-64, plus terms below 1e-24), c = RN(G/2pi)
// and the rounding of x c give RN(x c) = y (1 + eta), |eta| <= 4.01 2^-53, i.e. within
// 1024 * 4.01 * 2^-53 = 4.6e-13 of y.  So floor(RN(x c)) = floor(y) = floor(G T / 2^64)
// (the high word of G T) unless frac(y), the low word, lies within 2^-40 of an integer
// (T at the top of the turn, where x may wrap to 0, included); there cell_index of the
// stored x decides.  Same bits as cell_key(x, y, z).
// The exact path, out of line: it runs about once per 2^39 coordinates, and inlined at
// every key site it made the plain fused step 1.9 % slower.
static __device__ __noinline__ int cell_index_exact(double x, uint64_t cfx, uint64_t cm, int ce, int G) {
  return min(cell_index(x, cfx, cm, ce), G - 1);
}

__device__ __forceinline__ int cell_index_turns(uint64_t T, double x, const CellKeyK& k) {
  const uint64_t lo = T * (uint64_t)k.G;
  if (lo >= (1ull << 24) && lo <= 0ull - (1ull << 24)) return (int)__umul64hi(T, (uint64_t)k.G);
  return cell_index_exact(x, k.cfx, k.cm, k.ce, k.G);
}

__device__ __forceinline__ uint32_t cell_key_turns(const uint64_t T[3], double x, double y, double z,
                                                   const CellKeyK& k) {
  const int ix = cell_index_turns(T[0], x, k), iy = cell_index_turns(T[1], y, k), iz = cell_index_turns(T[2], z, k);
  return (uint32_t)((iz * k.G + iy) * k.G + ix);
}

// nsteps steps of one particle (the ragged tail of a launch).  Same per-particle
// function as fused_group, so a particle gets the same bits on either path.
template <bool TAU, bool ACC, class Trig>
__device__ __forceinline__ void fused_tail(const EnsArgs& e, const StepC& kc, const TurnsK& tk, const Trig& trig,
                                           int64_t i0, int cnt, int nsteps, uint32_t* keys, const CellKeyK& ck) {
  for (int j = 0; j < cnt; ++j) {
    const int64_t i = i0 + j;
    uint64_t T[3] = {to_turns(e.px[i]), to_turns(e.py[i]), to_turns(e.pz[i])};
    float v[3] = {e.vx[i], e.vy[i], e.vz[i]}, a[3] = {0.f, 0.f, 0.f};
    StepC k = kc;
    if constexpr (TAU) set_inv_tau(k, particle_inv_tau<true>(e, i));
    for (int s = 0; s < nsteps; ++s) rk2_step_turns<ACC, false>(k, tk, trig, T, v, a);
    const double x = turns_to_x(T[0]), y = turns_to_x(T[1]), z = turns_to_x(T[2]);
    e.px[i] = x;
    e.py[i] = y;
    e.pz[i] = z;
    if (keys) keys[i] = cell_key_turns(T, x, y, z, ck);
    e.vx[i] = v[0]; e.vy[i] = v[1]; e.vz[i] = v[2];
    if constexpr (ACC) { e.ax[i] = a[0]; e.ay[i] = a[1]; e.az[i] = a[2]; }
  }
}

// The PPT particles i0..i0+PPT-1 (all < n): one vectorised load and store of each plane,
// nsteps steps in between (nsteps >= 1).  A group whose speeds are all within the shift
// series (near_shift), with displacements that need no check (fast_positions), runs
// straight-line code for that step.
template <int PPT, bool TAU, bool ACC, class Trig>
__device__ __forceinline__ void fused_group(const EnsArgs& e, const StepC& kc, const TurnsK& tk, const Trig& trig,
                                            int64_t i0, int nsteps, uint32_t* keys, const CellKeyK& ck) {
  double x[PPT], y[PPT], z[PPT];
  float vx[PPT], vy[PPT], vz[PPT];
  load_f64<PPT, 128>(e.px, i0, x);
  load_f64<PPT, 128>(e.py, i0, y);
  load_f64<PPT, 128>(e.pz, i0, z);
  load_f32<PPT, 128>(e.vx, i0, vx);
  load_f32<PPT, 128>(e.vy, i0, vy);
  load_f32<PPT, 128>(e.vz, i0, vz);
  uint64_t T[PPT][3];
  float v[PPT][3], a[PPT][3];
  ff sj[PPT];
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    T[j][0] = to_turns(x[j]);
    T[j][1] = to_turns(y[j]);
    T[j][2] = to_turns(z[j]);
    v[j][0] = vx[j]; v[j][1] = vy[j]; v[j][2] = vz[j];
    if constexpr (TAU) sj[j] = particle_inv_tau<true>(e, i0 + j);
  }
  StepC k = kc;
  // Whether the displacements of steps within the shift series need no check (fixed for
  // the call: it depends on tau, dt and the amplitudes only).
  bool fast = true;
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    if constexpr (TAU) set_inv_tau(k, sj[j]);
    fast = fast && fast_positions(k, tk);
  }
  // Every step of the call stays within the shift series when every particle starts at
  // speeds <= vsafe (TurnsK::vsafe): then no check per step (the same bits).
  // (With tau per particle there is no launch-wide guarantee: vsafe is -1.)
  bool safe = !TAU && fast;
#pragma unroll
  for (int j = 0; j < PPT; ++j) safe = safe && fmaxf(fabsf(v[j][0]), fmaxf(fabsf(v[j][1]), fabsf(v[j][2]))) <= tk.vsafe;
  if constexpr (!TAU) {
    if (safe) {
      for (int s = 0; s < nsteps; ++s) {
#pragma unroll
        for (int j = 0; j < PPT; ++j) rk2_step_turns<ACC, true>(k, tk, trig, T[j], v[j], a[j]);
      }
    }
  }
  for (int s = 0; s < (safe ? 0 : nsteps); ++s) {
    bool near = fast;
#pragma unroll
    for (int j = 0; j < PPT; ++j) near = near && near_shift(k, v[j]);
    if (near) {
#pragma unroll
      for (int j = 0; j < PPT; ++j) {
        if constexpr (TAU) set_inv_tau(k, sj[j]);
        rk2_step_turns<ACC, true>(k, tk, trig, T[j], v[j], a[j]);
      }
    } else {
#pragma unroll
      for (int j = 0; j < PPT; ++j) {
        if constexpr (TAU) set_inv_tau(k, sj[j]);
        rk2_step_turns<ACC, false>(k, tk, trig, T[j], v[j], a[j]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    x[j] = turns_to_x(T[j][0]);
    y[j] = turns_to_x(T[j][1]);
    z[j] = turns_to_x(T[j][2]);
    vx[j] = v[j][0]; vy[j] = v[j][1]; vz[j] = v[j][2];
  }
  store_f64<PPT, 128>(e.px, i0, x);
  store_f64<PPT, 128>(e.py, i0, y);
  store_f64<PPT, 128>(e.pz, i0, z);
  if (keys) {
#pragma unroll
    for (int j = 0; j < PPT; ++j) keys[i0 + j] = cell_key_turns(T[j], x[j], y[j], z[j], ck);
  }
  store_f32<PPT, 128>(e.vx, i0, vx);
  store_f32<PPT, 128>(e.vy, i0, vy);
  store_f32<PPT, 128>(e.vz, i0, vz);
  if constexpr (ACC) {
    float o[PPT];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
      for (int j = 0; j < PPT; ++j) o[j] = a[j][c];
      store_f32<PPT, 128>(c == 0 ? e.ax : (c == 1 ? e.ay : e.az), i0, o);
    }
  }
}

// The particles [i0, i0 + cnt): the vector path for a full group, the scalar path for a
// ragged one.
template <int PPT, bool TAU, bool ACC, class Trig>
__device__ __forceinline__ void fused_span(const EnsArgs& e, const StepC& kc, const TurnsK& tk, const Trig& trig,
                                           int64_t i0, int64_t cnt, int nsteps, uint32_t* keys = nullptr,
                                           const CellKeyK& ck = CellKeyK{}) {
  if (cnt >= PPT)
    fused_group<PPT, TAU, ACC>(e, kc, tk, trig, i0, nsteps, keys, ck);
  else
    fused_tail<TAU, ACC>(e, kc, tk, trig, i0, (int)cnt, nsteps, keys, ck);
}

template <int PPT, bool TAU, bool ACC>
__device__ __forceinline__ void fused_loop(const EnsArgs& e, const StepC& kc, const TurnsK& tk, const TrigScaled& tg,
                                           int nsteps, uint32_t* keys, const CellKeyK& ck) {
  const int64_t ngroups = (e.n + PPT - 1) / PPT;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = g * PPT;
    fused_span<PPT, TAU, ACC>(e, kc, tk, tg, i0, e.n - i0, nsteps, keys, ck);
  }
}

// Persistent grid over groups of PPT particles; each block builds the three
// amplitude-scaled sin/cos tables (96 KB of dynamic shared memory) once.  TAU: tau per
// particle from e.tau_src; ACC: store the last stage acceleration (one kernel per
// combination, so the plain one is not sized for the others' registers).  keys: NULL, or
// n u32 receiving the cell keys of the final positions on the grid of ck.
template <int PPT, int BLOCK, int MINB, bool TAU, bool ACC>
__global__ void __launch_bounds__(BLOCK, MINB) k_step_soa_fused(EnsArgs e, FlowK f, TurnsK tk, int nsteps,
                                                                uint32_t* __restrict__ keys, CellKeyK ck) {
  extern __shared__ float4 s_tab3[];
  load_scaled_trig_tables(s_tab3, ff_from2(e.Af), ff_from2(e.Bf), ff_from2(e.Cf));
  const StepC kc = make_stepc(e, f);
  const TrigScaled tg{s_tab3};
  fused_loop<PPT, TAU, ACC>(e, kc, tk, tg, nsteps, keys, ck);
}

// soax_permute_step_fused: the permute-gather of every plane fused into the step's one
// pass.  Particle i of the output (the other buffer set) is particle perm[i] of the input
// (the live set): its position and velocity are gathered, stepped and stored at i, its
// other planes copied to i, so the planes are read and written once for the permute and
// all the steps together.
struct GatherArgs {
  const uint32_t* perm;
  int* status;                  // a perm entry >= n is recorded here (element 0 is used)
  int nother;                   // planes copied unchanged (everything but pos, vel, acc)
  const void* in[kMaxPlanes];
  void* out[kMaxPlanes];
  int es[kMaxPlanes];           // element size: 1, 4 or 8 bytes
};

template <int BLOCK, int MINB, bool TAU, bool ACC>
__global__ void __launch_bounds__(BLOCK, MINB) k_step_soa_fused_gather(EnsArgs ein, EnsArgs eout, GatherArgs g,
                                                                       FlowK f, TurnsK tk, int nsteps,
                                                                       uint32_t* __restrict__ keys, CellKeyK ck) {
  extern __shared__ float4 s_tab3[];
  load_scaled_trig_tables(s_tab3, ff_from2(ein.Af), ff_from2(ein.Bf), ff_from2(ein.Cf));
  const StepC kc = make_stepc(ein, f);
  const TrigScaled tg{s_tab3};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t src_next = i < ein.n ? g.perm[i] : 0u;
  for (; i < ein.n; i += stride) {
    int64_t src = src_next;
    if (src >= ein.n) {
      atomicExch(g.status, (int)SOAX_EINVAL);
      src = 0;
    }
    // The next particle's source: read its perm entry now and start moving its position
    // and velocity into L2, so that its gather does not wait on HBM after this particle's
    // steps.  An entry >= n is prefetched as 0 (and reported when it is used).
    if (i + stride < ein.n) {
      src_next = g.perm[i + stride];
      const int64_t pf = src_next < ein.n ? (int64_t)src_next : 0;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(ein.px + pf));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(ein.py + pf));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(ein.pz + pf));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(ein.vx + pf));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(ein.vy + pf));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(ein.vz + pf));
    }
    // The copied planes; a 4-byte first one (an i32 id) without the per-plane size
    // dispatch (21 fewer instructions per particle, 0.8 % of the launch).
    int p0 = 0;
    if (g.nother > 0 && g.es[0] == 4) {
      static_cast<uint32_t*>(g.out[0])[i] = static_cast<const uint32_t*>(g.in[0])[src];
      p0 = 1;
    }
    for (int p = p0; p < g.nother; ++p) {
      const int es = g.es[p];
      if (es == 8)
        static_cast<unsigned long long*>(g.out[p])[i] = static_cast<const unsigned long long*>(g.in[p])[src];
      else if (es == 4)
        static_cast<uint32_t*>(g.out[p])[i] = static_cast<const uint32_t*>(g.in[p])[src];
      else
        static_cast<uint8_t*>(g.out[p])[i] = static_cast<const uint8_t*>(g.in[p])[src];
    }
    uint64_t T[3] = {to_turns(ein.px[src]), to_turns(ein.py[src]), to_turns(ein.pz[src])};
    float v[3] = {ein.vx[src], ein.vy[src], ein.vz[src]}, a[3] = {0.f, 0.f, 0.f};
    StepC k = kc;
    if constexpr (TAU) set_inv_tau(k, particle_inv_tau<true>(ein, src));
    const bool fast = fast_positions(k, tk);
    if (!TAU && fast && fmaxf(fabsf(v[0]), fmaxf(fabsf(v[1]), fabsf(v[2]))) <= tk.vsafe) {
      // Every step of this call stays within the shift series (TurnsK::vsafe): no check
      // per step.  The same bits as the checked loop below.
      for (int s = 0; s < nsteps; ++s) rk2_step_turns<ACC, true>(k, tk, tg, T, v, a);
    } else {
      for (int s = 0; s < nsteps; ++s) {
        if (fast && near_shift(k, v))
          rk2_step_turns<ACC, true>(k, tk, tg, T, v, a);
        else
          rk2_step_turns<ACC, false>(k, tk, tg, T, v, a);
      }
    }
    const double x = turns_to_x(T[0]), y = turns_to_x(T[1]), z = turns_to_x(T[2]);
    eout.px[i] = x;
    eout.py[i] = y;
    eout.pz[i] = z;
    if (keys) keys[i] = cell_key_turns(T, x, y, z, ck);
    eout.vx[i] = v[0]; eout.vy[i] = v[1]; eout.vz[i] = v[2];
    if constexpr (ACC) { eout.ax[i] = a[0]; eout.ay[i] = a[1]; eout.az[i] = a[2]; }
  }
}

}  // namespace soax
