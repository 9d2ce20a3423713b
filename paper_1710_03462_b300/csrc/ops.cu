// Whole-array operations of the SoAx container (Sec. 4): SetToValue applied to every
// array (apply<F>(), Listing 7) and fused elementwise expressions over planes such as
// posArr(0) = velArr(1) - velArr(2) (Listing 5), evaluated in one pass per expression
// (the loop fusion of Sec. 4.2.2) instead of one pass per operator.
#include <cmath>
#include <cstring>

#include "soax_internal.h"

namespace soax {

constexpr int kMaxTerms = 8;

struct FillArgs {
  void* planes[kMaxPlanes];
  int32_t es[kMaxPlanes];
  uint64_t pattern[kMaxPlanes];  // the element's bytes, little-endian, in the low es bytes
  int nplanes;
  int64_t n;
};

__global__ void __launch_bounds__(256) k_fill(const __grid_constant__ FillArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int p = 0; p < a.nplanes; ++p) {
    const int es = a.es[p];
    // 16 bytes of the repeated element (es divides 16).
    uint64_t w = a.pattern[p];
    if (es == 1) w = (w & 0xFF) * 0x0101010101010101ull;
    else if (es == 4) w = (w & 0xFFFFFFFFull) * 0x0000000100000001ull;
    const uint4 v = make_uint4((uint32_t)w, (uint32_t)(w >> 32), (uint32_t)w, (uint32_t)(w >> 32));
    const int64_t bytes = a.n * es, n16 = bytes >> 4;
    uint4* dst = static_cast<uint4*>(a.planes[p]);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) dst[i] = v;
    unsigned char* tail = static_cast<unsigned char*>(a.planes[p]);
    for (int64_t i = (n16 << 4) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < bytes; i += stride)
      tail[i] = (unsigned char)(w >> (8 * (i % 8)));
  }
}

template <typename T>
struct LinArgs {
  T* dst;
  const T* src[kMaxTerms];
  T coef[kMaxTerms];
  T constant;
  int nterms;
  int64_t n;
};

__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T>
__global__ void __launch_bounds__(256) k_lincomb(const __grid_constant__ LinArgs<T> a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    T acc = a.constant;
    for (int k = 0; k < a.nterms; ++k) acc = fma_rn(a.coef[k], a.src[k][i], acc);
    a.dst[i] = acc;
  }
}

static bool fill_pattern(int dtype, double v, uint64_t* pat) {
  switch (dtype) {
    case SOAX_I32: {
      if (!(v == std::floor(v) && v >= -2147483648.0 && v <= 2147483647.0)) return false;
      int32_t x = (int32_t)v;
      uint32_t u;
      std::memcpy(&u, &x, 4);
      *pat = u;
      return true;
    }
    case SOAX_I64: {
      if (!(v == std::floor(v) && v >= -9223372036854775808.0 && v < 9223372036854775808.0)) return false;
      int64_t x = (int64_t)v;
      std::memcpy(pat, &x, 8);
      return true;
    }
    case SOAX_U8:
      if (!(v == std::floor(v) && v >= 0.0 && v <= 255.0)) return false;
      *pat = (uint64_t)(uint8_t)v;
      return true;
    case SOAX_F32: {
      if (std::isfinite(v) && std::fabs(v) > 3.4028234663852886e38) return false;
      float x = (float)v;
      uint32_t u;
      std::memcpy(&u, &x, 4);
      *pat = u;
      return true;
    }
    case SOAX_F64:
      std::memcpy(pat, &v, 8);
      return true;
  }
  return false;
}

}  // namespace soax

using namespace soax;

extern "C" int soax_fill(soax_t h, int32_t field, double value, void* stream) {
  if (int r = check_handle(h)) return r;
  if (field < -1 || field >= (int)h->fields.size()) return fail(SOAX_EINVAL, "soax_fill: bad field");
  FillArgs a;
  a.nplanes = 0;
  for (size_t f = 0; f < h->fields.size(); ++f) {
    if (field >= 0 && (int)f != field) continue;
    const Field& F = h->fields[f];
    uint64_t pat = 0;
    if (!fill_pattern(F.dtype, value, &pat))
      return fail(SOAX_EINVAL, "soax_fill: value not representable in field '" + F.name + "'");
    for (int c = 0; c < F.ncomp; ++c) {
      void* p = h->planes[h->current][F.first_plane + c];
      if (!p && h->n > 0) return fail(SOAX_EUNBOUND, "soax_fill: plane not bound");
      a.planes[a.nplanes] = p;
      a.es[a.nplanes] = F.esize;
      a.pattern[a.nplanes] = pat;
      ++a.nplanes;
    }
  }
  if (h->n == 0) return SOAX_OK;
  a.n = h->n;
  const int grid = persistent_grid((const void*)k_fill, 256, 0, grid_for((h->n * 8 + 15) / 16, 256));
  k_fill<<<grid, 256, 0, as_stream(stream)>>>(a);
  return check_launch("soax_fill");
}

extern "C" int soax_lincomb(soax_t h, int32_t dst_field, int32_t dst_comp, int32_t nterms, const int32_t* src_fields,
                            const int32_t* src_comps, const double* coefs, double constant, void* stream) {
  if (int r = check_handle(h)) return r;
  if (nterms < 0 || nterms > kMaxTerms) return fail(SOAX_EINVAL, "soax_lincomb: nterms must be in 0..8");
  if (nterms > 0 && (!src_fields || !src_comps || !coefs)) return fail(SOAX_EINVAL, "soax_lincomb: NULL term arrays");
  auto plane_of = [&](int f, int c, void** out) -> int {
    if (f < 0 || f >= (int)h->fields.size() || c < 0 || c >= h->fields[f].ncomp)
      return fail(SOAX_EINVAL, "soax_lincomb: bad field or component");
    *out = h->planes[h->current][h->fields[f].first_plane + c];
    if (!*out && h->n > 0) return fail(SOAX_EUNBOUND, "soax_lincomb: plane not bound");
    return SOAX_OK;
  };
  void* dst = nullptr;
  if (int r = plane_of(dst_field, dst_comp, &dst)) return r;
  const int dt = h->fields[dst_field].dtype;
  if (dt != SOAX_F32 && dt != SOAX_F64) return fail(SOAX_ESCHEMA, "soax_lincomb: planes must be f32 or f64");
  const void* src[kMaxTerms] = {};
  for (int k = 0; k < nterms; ++k) {
    void* p = nullptr;
    if (int r = plane_of(src_fields[k], src_comps[k], &p)) return r;
    if (h->fields[src_fields[k]].dtype != dt) return fail(SOAX_ESCHEMA, "soax_lincomb: all planes must share one type");
    src[k] = p;
  }
  if (h->n == 0) return SOAX_OK;
  cudaStream_t s = as_stream(stream);
  const int64_t wb = grid_for(h->n, 256);
  if (dt == SOAX_F32) {
    LinArgs<float> a;
    a.dst = static_cast<float*>(dst);
    for (int k = 0; k < nterms; ++k) {
      a.src[k] = static_cast<const float*>(src[k]);
      a.coef[k] = (float)coefs[k];
    }
    a.constant = (float)constant;
    a.nterms = nterms;
    a.n = h->n;
    k_lincomb<float><<<persistent_grid((const void*)k_lincomb<float>, 256, 0, wb), 256, 0, s>>>(a);
  } else {
    LinArgs<double> a;
    a.dst = static_cast<double*>(dst);
    for (int k = 0; k < nterms; ++k) {
      a.src[k] = static_cast<const double*>(src[k]);
      a.coef[k] = coefs[k];
    }
    a.constant = constant;
    a.nterms = nterms;
    a.n = h->n;
    k_lincomb<double><<<persistent_grid((const void*)k_lincomb<double>, 256, 0, wb), 256, 0, s>>>(a);
  }
  return check_launch("soax_lincomb");
}
