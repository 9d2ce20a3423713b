// The paper's benchmark step, Eq. 1 (Sec. 2): x += dt v per component, single precision,
// on SoA planes and on AoS records (the replica of the SoA-vs-AoS experiment of
// Sec. 2-3).  Each update is one rounded multiply and one rounded add, exactly as the
// C expression x + dt*v evaluates in float without contraction.
//
//  * k_euler_soa_fused: one pass over all six planes, four particles per thread with
//    16-byte loads and stores (36 algorithmic bytes per particle-step);
//  * k_euler_component: the paper's GPU SoA layout of work (Sec. 3.2): one kernel per
//    component, one element per thread;
//  * k_euler_aos: the paper's GPU AoS code: one thread per particle reading its record
//    (Particle<SIZE> of Listing 4: float x[3], v[3], temp[SIZE]).
#include "soax_internal.h"

namespace soax {

struct EulerPlanes {
  float* x[3];
  const float* v[3];
  int64_t n;
  float dt;
};

__global__ void __launch_bounds__(256) k_euler_soa_fused(EulerPlanes a) {
  const int64_t ng = a.n / 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += stride) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float4 x = reinterpret_cast<const float4*>(a.x[c])[g];
      const float4 v = reinterpret_cast<const float4*>(a.v[c])[g];
      x.x = __fadd_rn(x.x, __fmul_rn(a.dt, v.x));
      x.y = __fadd_rn(x.y, __fmul_rn(a.dt, v.y));
      x.z = __fadd_rn(x.z, __fmul_rn(a.dt, v.z));
      x.w = __fadd_rn(x.w, __fmul_rn(a.dt, v.w));
      reinterpret_cast<float4*>(a.x[c])[g] = x;
    }
  }
  // ragged tail (fewer than 4 particles)
  const int64_t t = ng * 4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < a.n)
    for (int c = 0; c < 3; ++c) a.x[c][t] = __fadd_rn(a.x[c][t], __fmul_rn(a.dt, a.v[c][t]));
}

__global__ void __launch_bounds__(256) k_euler_component(float* __restrict__ x, const float* __restrict__ v,
                                                         int64_t n, float dt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = __fadd_rn(x[i], __fmul_rn(dt, v[i]));
}

__global__ void __launch_bounds__(256) k_euler_aos(char* __restrict__ rec, int64_t n, int64_t R, int64_t xo,
                                                   int64_t vo, float dt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float* x = reinterpret_cast<float*>(rec + i * R + xo);
  const float* v = reinterpret_cast<const float*>(rec + i * R + vo);
#pragma unroll
  for (int c = 0; c < 3; ++c) x[c] = __fadd_rn(x[c], __fmul_rn(dt, v[c]));
}

}  // namespace soax

using namespace soax;

extern "C" int soax_euler(soax_t h, int32_t pos_field, int32_t vel_field, float dt, int32_t per_component,
                          void* stream) {
  if (int r = check_handle(h)) return r;
  if (int r = check_field(h, pos_field, SOAX_F32, 3, "soax_euler position")) return r;
  if (int r = check_field(h, vel_field, SOAX_F32, 3, "soax_euler velocity")) return r;
  if (h->n == 0) return SOAX_OK;
  EulerPlanes a;
  const int px = h->fields[pos_field].first_plane, pv = h->fields[vel_field].first_plane;
  for (int c = 0; c < 3; ++c) {
    a.x[c] = static_cast<float*>(h->planes[h->current][px + c]);
    a.v[c] = static_cast<const float*>(h->planes[h->current][pv + c]);
    if (!a.x[c] || !a.v[c]) return fail(SOAX_EUNBOUND, "soax_euler: planes not bound");
  }
  a.n = h->n;
  a.dt = dt;
  cudaStream_t s = as_stream(stream);
  if (per_component) {
    for (int c = 0; c < 3; ++c) {
      k_euler_component<<<grid_for(h->n, 256), 256, 0, s>>>(a.x[c], a.v[c], h->n, dt);
      if (int r = check_launch("soax_euler")) return r;
    }
    return SOAX_OK;
  }
  const int grid = persistent_grid((const void*)k_euler_soa_fused, 256, 0, grid_for((h->n + 3) / 4, 256));
  k_euler_soa_fused<<<grid, 256, 0, s>>>(a);
  return check_launch("soax_euler");
}

extern "C" int soax_euler_aos(void* rec, int64_t n, int64_t record_bytes, int64_t x_off, int64_t v_off, float dt,
                              void* stream) {
  if (n < 0) return fail(SOAX_EINVAL, "soax_euler_aos: n < 0");
  if (n == 0) return SOAX_OK;
  if (!rec) return fail(SOAX_EINVAL, "soax_euler_aos: NULL records");
  if ((reinterpret_cast<uintptr_t>(rec) & 3) || (record_bytes & 3) || (x_off & 3) || (v_off & 3))
    return fail(SOAX_EALIGN, "soax_euler_aos: records, record size and offsets must be multiples of 4 bytes");
  if (x_off < 0 || v_off < 0 || x_off + 12 > record_bytes || v_off + 12 > record_bytes)
    return fail(SOAX_EINVAL, "soax_euler_aos: x or v outside the record");
  k_euler_aos<<<grid_for(n, 256), 256, 0, as_stream(stream)>>>(static_cast<char*>(rec), n, record_bytes, x_off,
                                                              v_off, dt);
  return check_launch("soax_euler_aos");
}
