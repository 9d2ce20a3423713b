// AoS <-> SoA transposes: the bulk form of getElement / push_back (Listing 6, Sec. 4.1),
// which copy one particle between the SoA arrays and a record.
//
// Each block stages kXRecs whole records in shared memory: the record side is moved
// with 16-byte vector accesses over one contiguous byte range, the plane side with one
// coalesced access per plane element (thread t handles records t, t + 256, ...).  Bytes
// are copied exactly; SoA -> AoS zeroes the padding of every record.
#include "soax_internal.h"

namespace soax {

constexpr int kXRecs = 512;  // records per block (kXRecs * R is a multiple of 16 for any R)
constexpr int kXThreads = 256;

struct XArgs {
  void* planes[kMaxPlanes];
  int32_t es[kMaxPlanes];
  int32_t off[kMaxPlanes];  // byte offset of the component inside the record
  int nplanes;
  int64_t n;
  int64_t R;
  char* rec;
};

__global__ void __launch_bounds__(kXThreads) k_aos_to_soa(const __grid_constant__ XArgs a) {
  extern __shared__ uint4 tile4[];
  char* tile = reinterpret_cast<char*>(tile4);
  const int64_t r0 = (int64_t)blockIdx.x * kXRecs;
  const int cnt = (int)(a.n - r0 < kXRecs ? a.n - r0 : kXRecs);
  const int64_t bytes = (int64_t)cnt * a.R;
  const char* src = a.rec + r0 * a.R;
  const int64_t n16 = bytes >> 4;
  for (int64_t k = threadIdx.x; k < n16; k += kXThreads) tile4[k] = reinterpret_cast<const uint4*>(src)[k];
  for (int64_t k = (n16 << 4) + threadIdx.x; k < bytes; k += kXThreads) tile[k] = src[k];
  __syncthreads();
  for (int p = 0; p < a.nplanes; ++p) {
    const int es = a.es[p], off = a.off[p];
    for (int t = threadIdx.x; t < cnt; t += kXThreads) {
      const char* s = tile + (int64_t)t * a.R + off;
      if (es == 8)
        static_cast<unsigned long long*>(a.planes[p])[r0 + t] = *reinterpret_cast<const unsigned long long*>(s);
      else if (es == 4)
        static_cast<uint32_t*>(a.planes[p])[r0 + t] = *reinterpret_cast<const uint32_t*>(s);
      else
        static_cast<uint8_t*>(a.planes[p])[r0 + t] = *reinterpret_cast<const uint8_t*>(s);
    }
  }
}

__global__ void __launch_bounds__(kXThreads) k_soa_to_aos(const __grid_constant__ XArgs a) {
  extern __shared__ uint4 tile4[];
  char* tile = reinterpret_cast<char*>(tile4);
  const int64_t r0 = (int64_t)blockIdx.x * kXRecs;
  const int cnt = (int)(a.n - r0 < kXRecs ? a.n - r0 : kXRecs);
  const int64_t bytes = (int64_t)cnt * a.R;
  const int64_t n16 = (bytes + 15) >> 4;
  for (int64_t k = threadIdx.x; k < n16; k += kXThreads) tile4[k] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  for (int p = 0; p < a.nplanes; ++p) {
    const int es = a.es[p], off = a.off[p];
    for (int t = threadIdx.x; t < cnt; t += kXThreads) {
      char* d = tile + (int64_t)t * a.R + off;
      if (es == 8)
        *reinterpret_cast<unsigned long long*>(d) = static_cast<const unsigned long long*>(a.planes[p])[r0 + t];
      else if (es == 4)
        *reinterpret_cast<uint32_t*>(d) = static_cast<const uint32_t*>(a.planes[p])[r0 + t];
      else
        *reinterpret_cast<uint8_t*>(d) = static_cast<const uint8_t*>(a.planes[p])[r0 + t];
    }
  }
  __syncthreads();
  char* dst = a.rec + r0 * a.R;
  const int64_t f16 = bytes >> 4;
  for (int64_t k = threadIdx.x; k < f16; k += kXThreads) reinterpret_cast<uint4*>(dst)[k] = tile4[k];
  for (int64_t k = (f16 << 4) + threadIdx.x; k < bytes; k += kXThreads) dst[k] = tile[k];
}

static int make_xargs(soax_t h, void* rec, XArgs* a, const char* who, int64_t first = 0, int64_t count = -1) {
  if (int r = live_planes_bound(h, h->current)) return r;
  if (!rec) return fail(SOAX_EINVAL, std::string(who) + ": records pointer is NULL");
  if (!aligned16(rec)) return fail(SOAX_EALIGN, std::string(who) + ": records not 16-byte aligned");
  int p = 0;
  for (size_t f = 0; f < h->fields.size(); ++f)
    for (int c = 0; c < h->fields[f].ncomp; ++c, ++p) {
      a->planes[p] = static_cast<char*>(h->planes[h->current][p]) + first * h->fields[f].esize;
      a->es[p] = h->fields[f].esize;
      a->off[p] = (int32_t)(h->offsets[f] + (int64_t)c * h->fields[f].esize);
    }
  a->nplanes = h->nplanes;
  a->n = count < 0 ? h->n : count;
  a->R = h->record_bytes;
  a->rec = static_cast<char*>(rec);
  return SOAX_OK;
}

static size_t tile_smem(int64_t R) { return (size_t)((kXRecs * R + 15) / 16 * 16); }

static int set_smem_attr(const void* fn, size_t bytes) {
  if (bytes <= 48 * 1024) return SOAX_OK;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return cuda_fail(e, "transpose: shared memory attribute");
  return SOAX_OK;
}

}  // namespace soax

using namespace soax;

extern "C" int soax_aos_to_soa(soax_t h, const void* aos_dev, void* stream) {
  if (int r = check_handle(h)) return r;
  if (h->n == 0) return SOAX_OK;
  XArgs a;
  if (int r = make_xargs(h, const_cast<void*>(aos_dev), &a, "soax_aos_to_soa")) return r;
  const size_t sm = tile_smem(a.R);
  if (sm > 200 * 1024) return fail(SOAX_EUNSUPPORTED, "soax_aos_to_soa: record larger than 400 bytes");
  if (int r = set_smem_attr((const void*)k_aos_to_soa, sm)) return r;
  k_aos_to_soa<<<grid_for(h->n, kXRecs), kXThreads, sm, as_stream(stream)>>>(a);
  return check_launch("soax_aos_to_soa");
}

extern "C" int soax_soa_to_aos(soax_t h, void* aos_dev, void* stream) {
  if (int r = check_handle(h)) return r;
  if (h->n == 0) return SOAX_OK;
  XArgs a;
  if (int r = make_xargs(h, aos_dev, &a, "soax_soa_to_aos")) return r;
  const size_t sm = tile_smem(a.R);
  if (sm > 200 * 1024) return fail(SOAX_EUNSUPPORTED, "soax_soa_to_aos: record larger than 400 bytes");
  if (int r = set_smem_attr((const void*)k_soa_to_aos, sm)) return r;
  k_soa_to_aos<<<grid_for(h->n, kXRecs), kXThreads, sm, as_stream(stream)>>>(a);
  return check_launch("soax_soa_to_aos");
}

extern "C" int soax_get_element(soax_t h, int64_t i, void* rec_dev, void* stream) {
  if (int r = check_handle(h)) return r;
  if (i < 0 || i >= h->n) return fail(SOAX_EINVAL, "soax_get_element: index out of range");
  XArgs a;
  if (int r = make_xargs(h, rec_dev, &a, "soax_get_element", i, 1)) return r;
  k_soa_to_aos<<<1, kXThreads, (size_t)((a.R + 15) / 16 * 16), as_stream(stream)>>>(a);
  return check_launch("soax_get_element");
}

extern "C" int soax_set_element(soax_t h, int64_t i, const void* rec_dev, void* stream) {
  if (int r = check_handle(h)) return r;
  if (i < 0 || i >= h->n) return fail(SOAX_EINVAL, "soax_set_element: index out of range");
  XArgs a;
  if (int r = make_xargs(h, const_cast<void*>(rec_dev), &a, "soax_set_element", i, 1)) return r;
  k_aos_to_soa<<<1, kXThreads, (size_t)((a.R + 15) / 16 * 16), as_stream(stream)>>>(a);
  return check_launch("soax_set_element");
}
