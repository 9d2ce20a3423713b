// AoS <-> SoA transposes: the bulk form of getElement / push_back (Listing 6, Sec. 4.1),
// which copy one particle between the SoA arrays and a record.
//
// Each block stages kXRecs whole records in shared memory: the record side is moved
// with 16-byte vector accesses over one contiguous byte range, the plane side with one
// coalesced access per plane element (thread t handles records t, t + 256, ...), or, for
// SoA -> AoS on a full tile, with 16-byte chunks of every plane, several in flight per
// thread (the loads would otherwise wait one after another).  Bytes are copied exactly;
// SoA -> AoS zeroes the padding of every record.
#include "soax_internal.h"

namespace soax {

constexpr int kXRecs = 512;  // records per block (kXRecs * R is a multiple of 16 for any R)
constexpr int kXThreads = 256;

struct XArgs {
  void* planes[kMaxPlanes];
  int32_t es[kMaxPlanes];
  int32_t off[kMaxPlanes];  // byte offset of the component inside the record
  int32_t cpre[kMaxPlanes + 1];  // prefix of 16-byte chunks per plane in a full tile
  int nplanes;
  int64_t n;
  int64_t R;
  char* rec;
};

constexpr int kXUnroll = 8;  // 16-byte plane chunks in flight per thread (SoA -> AoS)

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

// The element path of k_soa_to_aos (a ragged tile, or one element): one load per plane
// element.
__device__ __forceinline__ void soa_tile_elements(const XArgs& a, char* tile, int64_t r0, int cnt) {
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
}

// A full tile is staged with its 16-byte units permuted within each 128-byte row (unit k
// at k ^ ((k >> 3) & 7)): the chunk scatter below writes records that are 2 to 16 apart,
// which would otherwise fall on few banks; the copy-out reads each row's units in a
// permuted order, which stays conflict-free.  Elements are naturally aligned, so none
// straddles a unit.
__device__ __forceinline__ int64_t swz(int64_t b) {
  const int64_t u = b >> 4;
  return ((u ^ ((u >> 3) & 7)) << 4) | (b & 15);
}

// Scatter the 16-byte chunk v of plane p (tile elements q*16/es ..) into the staged records.
__device__ __forceinline__ void scatter_chunk(const XArgs& a, char* tile, int p, int q, uint4 v) {
  const int es = a.es[p], off = a.off[p];
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
  if (es == 8) {
    const int t = q * 2;
    *reinterpret_cast<uint2*>(tile + swz((int64_t)t * a.R + off)) = make_uint2(w[0], w[1]);
    *reinterpret_cast<uint2*>(tile + swz((int64_t)(t + 1) * a.R + off)) = make_uint2(w[2], w[3]);
  } else if (es == 4) {
    const int t = q * 4;
#pragma unroll
    for (int e = 0; e < 4; ++e) *reinterpret_cast<uint32_t*>(tile + swz((int64_t)(t + e) * a.R + off)) = w[e];
  } else {
    const int t = q * 16;
#pragma unroll
    for (int e = 0; e < 16; ++e) tile[swz((int64_t)(t + e) * a.R + off)] = (char)(w[e >> 2] >> ((e & 3) * 8));
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
  if (cnt == kXRecs) {
    // A full tile: every plane's span (kXRecs * es bytes, 16-byte aligned) is read as
    // 16-byte chunks, kXUnroll per thread in flight before any is placed.
    const int total = a.cpre[a.nplanes];
    for (int q0 = threadIdx.x; q0 < total; q0 += kXUnroll * kXThreads) {
      uint4 v[kXUnroll];
      int pl[kXUnroll], qq[kXUnroll];
#pragma unroll
      for (int u = 0; u < kXUnroll; ++u) {
        const int q = q0 + u * kXThreads;
        pl[u] = -1;
        if (q < total) {
          int p = 0;
          while (a.cpre[p + 1] <= q) ++p;
          pl[u] = p;
          qq[u] = q - a.cpre[p];
          v[u] = reinterpret_cast<const uint4*>(static_cast<const char*>(a.planes[p]) + r0 * a.es[p])[qq[u]];
        }
      }
#pragma unroll
      for (int u = 0; u < kXUnroll; ++u)
        if (pl[u] >= 0) scatter_chunk(a, tile, pl[u], qq[u], v[u]);
    }
    __syncthreads();
    // kXRecs * R is a multiple of 128 bytes for every R, so the tile is whole rows of units.
    uint4* dst = reinterpret_cast<uint4*>(a.rec + r0 * a.R);
    for (int64_t k = threadIdx.x; k < n16; k += kXThreads) dst[k] = tile4[k ^ ((k >> 3) & 7)];
    return;
  }
  soa_tile_elements(a, tile, r0, cnt);
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
  a->cpre[0] = 0;
  for (int q = 0; q < h->nplanes; ++q) a->cpre[q + 1] = a->cpre[q] + kXRecs * a->es[q] / 16;
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
