// Removal of particles by overwriting them with the last ones (Sec. 2: the default of
// SoAx when the order of the particles does not matter; O(1) per particle instead of
// shifting the arrays).
//
// For k distinct ascending indices and the new size m = n - k: the "holes" are the
// indices below m, which come first in idx; the "movers" are the tail positions
// m..n-1 that are not removed, in ascending order; there are as many of each, and hole j
// receives mover j.
//   k_remove_mark:   flag the removed tail positions (and check idx);
//   k_remove_movers: one block lists the unflagged tail positions (block scan);
//   k_remove_gather: every plane, hole j <- mover j.
#include "soax_internal.h"

namespace soax {

constexpr int kRmThreads = 1024;

static size_t r256(size_t x) { return (x + 255) & ~size_t(255); }

struct RemoveWs {
  size_t off_flags, off_movers, off_meta, total;
};

static RemoveWs remove_plan(int64_t k) {
  RemoveWs w;
  w.off_flags = 0;
  w.off_movers = r256((size_t)k);
  w.off_meta = w.off_movers + r256((size_t)k * 4);
  w.total = w.off_meta + 256;
  return w;
}

// meta[0] = number of holes, meta[1] = 1 if idx is invalid.
__global__ void __launch_bounds__(256) k_remove_mark(const uint32_t* __restrict__ idx, int64_t k, int64_t n, int64_t m,
                                                     uint8_t* __restrict__ flags, uint32_t* meta, int* status) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  const uint32_t t = idx[j];
  if (t >= n || (j > 0 && idx[j - 1] >= t)) {
    meta[1] = 1;
    atomicExch(status, (int)SOAX_EINVAL);
    return;
  }
  if (t >= m) flags[t - m] = 1;
}

__global__ void __launch_bounds__(kRmThreads) k_remove_movers(const uint8_t* __restrict__ flags, int64_t k, int64_t m,
                                                              uint32_t* __restrict__ movers, uint32_t* meta) {
  __shared__ uint32_t scratch[kRmThreads / 32 + 1];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t per = (k + kRmThreads - 1) / kRmThreads;
  const int64_t lo = tid * per, hi = lo + per < k ? lo + per : k;
  uint32_t cnt = 0;
  for (int64_t t = lo; t < hi; ++t) cnt += flags[t] ? 0u : 1u;
  // Block exclusive scan of the per-thread counts of movers.
  uint32_t inc = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) scratch[w] = inc;
  __syncthreads();
  if (w == 0) {
    const uint32_t s = lane < kRmThreads / 32 ? scratch[lane] : 0u;
    uint32_t si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, si, o);
      if (lane >= o) si += y;
    }
    if (lane < kRmThreads / 32) scratch[lane] = si - s;
    if (lane == kRmThreads / 32 - 1) scratch[kRmThreads / 32] = si;
  }
  __syncthreads();
  uint32_t pos = scratch[w] + inc - cnt;
  for (int64_t t = lo; t < hi; ++t)
    if (!flags[t]) movers[pos++] = (uint32_t)(m + t);
  if (tid == 0) meta[0] = scratch[kRmThreads / 32];
}

struct RemoveArgs {
  void* planes[kMaxPlanes];
  int32_t es[kMaxPlanes];
  int nplanes;
  const uint32_t* idx;
  const uint32_t* movers;
  const uint32_t* meta;
  int64_t k;
};

__global__ void __launch_bounds__(256) k_remove_gather(const __grid_constant__ RemoveArgs a) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.k || a.meta[1] || j >= (int64_t)a.meta[0]) return;
  const uint32_t hole = a.idx[j], src = a.movers[j];
  for (int f = 0; f < a.nplanes; ++f) {
    const int es = a.es[f];
    if (es == 8) {
      unsigned long long* p = static_cast<unsigned long long*>(a.planes[f]);
      p[hole] = p[src];
    } else if (es == 4) {
      uint32_t* p = static_cast<uint32_t*>(a.planes[f]);
      p[hole] = p[src];
    } else {
      uint8_t* p = static_cast<uint8_t*>(a.planes[f]);
      p[hole] = p[src];
    }
  }
}

}  // namespace soax

using namespace soax;

extern "C" int soax_remove_workspace_bytes(int64_t k, size_t* bytes) {
  if (!bytes || k < 0) return fail(SOAX_EINVAL, "soax_remove_workspace_bytes: bad argument");
  *bytes = remove_plan(k).total;
  return SOAX_OK;
}

extern "C" int soax_remove(soax_t h, const uint32_t* idx, int64_t k, void* ws, size_t ws_bytes, void* stream) {
  if (int r = check_handle(h)) return r;
  if (k < 0 || k > h->n) return fail(SOAX_EINVAL, "soax_remove: k must be in 0..n");
  if (k == 0) return SOAX_OK;
  if (!idx) return fail(SOAX_EINVAL, "soax_remove: idx is NULL");
  const RemoveWs w = remove_plan(k);
  if (!ws || ws_bytes < w.total) return fail(SOAX_ENOMEM, "soax_remove: workspace too small");
  if (!aligned16(ws)) return fail(SOAX_EALIGN, "soax_remove: workspace not 16-byte aligned");
  if (int r = live_planes_bound(h, h->current)) return r;
  int* status = status_word();
  if (!status) return fail(SOAX_ECUDA, "soax_remove: status word");
  char* base = static_cast<char*>(ws);
  uint8_t* flags = reinterpret_cast<uint8_t*>(base + w.off_flags);
  uint32_t* movers = reinterpret_cast<uint32_t*>(base + w.off_movers);
  uint32_t* meta = reinterpret_cast<uint32_t*>(base + w.off_meta);
  const int64_t m = h->n - k;
  cudaStream_t s = as_stream(stream);
  cudaError_t e = cudaMemsetAsync(flags, 0, (size_t)k, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(meta, 0, 8, s);
  if (e != cudaSuccess) return cuda_fail(e, "soax_remove: memset");
  k_remove_mark<<<grid_for(k, 256), 256, 0, s>>>(idx, k, h->n, m, flags, meta, status);
  if (int r = check_launch("soax_remove: mark")) return r;
  k_remove_movers<<<1, kRmThreads, 0, s>>>(flags, k, m, movers, meta);
  if (int r = check_launch("soax_remove: movers")) return r;
  RemoveArgs a;
  for (int p = 0; p < h->nplanes; ++p) {
    a.planes[p] = h->planes[h->current][p];
    a.es[p] = h->plane_esize[p];
  }
  a.nplanes = h->nplanes;
  a.idx = idx;
  a.movers = movers;
  a.meta = meta;
  a.k = k;
  k_remove_gather<<<grid_for(k, 256), 256, 0, s>>>(a);
  if (int r = check_launch("soax_remove: gather")) return r;
  h->n = m;
  return SOAX_OK;
}
