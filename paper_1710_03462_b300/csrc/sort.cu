// Cell keys, stable LSD radix sort of (u32 key, u32 value) pairs, the permute-gather of
// every plane, and soax_sort_by_cell which chains them.
//
// The sort keeps the particle arrays in spatial order so that the step's and the
// gather's memory accesses stay local (Sec. 1 motivates SoA layouts by the spatial
// locality of memory access; the sort extends that to the particles' order).
//
// Radix sort: reduce-then-scan, least significant digit first, digits of up to 9 bits.
// Per pass: (1) every block histograms the digits of its 4096-key tile; (2) one block
// per digit turns the per-block counts into global offsets (digit-major exclusive
// scan); (3) every block ranks its tile stably (warp match + per-warp counters, in tile
// order), stages the tile in shared memory in digit order and writes each digit's run
// contiguously.  No block waits on another block, so nothing can hang.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "cell_key.cuh"
#include "soax_internal.h"

namespace soax {

constexpr int kSortBlock = 256;
constexpr int kSortWarps = kSortBlock / 32;
constexpr int kSortItems = 16;
constexpr int kTile = kSortBlock * kSortItems;  // 4096 keys per block
constexpr int kMaxDigitBits = 9;
constexpr int kMaxRadix = 1 << kMaxDigitBits;
constexpr int kScanThreads = 1024;

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct RadixPlan {
  int passes = 0, width = 0;
  int64_t nblocks = 0;
  size_t off_counts = 0, off_totals = 0, off_ak[2] = {0, 0}, off_av[2] = {0, 0}, total = 0;
};

static RadixPlan radix_plan(int64_t n, int bits) {
  RadixPlan p;
  p.passes = (bits + kMaxDigitBits - 1) / kMaxDigitBits;
  p.width = (bits + p.passes - 1) / p.passes;
  p.nblocks = (n + kTile - 1) / kTile;
  size_t off = 0;
  p.off_counts = off;
  off = align256(off + (size_t)kMaxRadix * p.nblocks * 4);
  p.off_totals = off;
  off = align256(off + (size_t)kMaxRadix * 4);
  int nalt = p.passes <= 1 ? 0 : (p.passes == 2 ? 1 : 2);
  for (int a = 0; a < nalt; ++a) {
    p.off_ak[a] = off;
    off = align256(off + (size_t)n * 4);
    p.off_av[a] = off;
    off = align256(off + (size_t)n * 4);
  }
  p.total = off;
  return p;
}

// ------------------------------------------------------------------ block scans
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive scan of one value per thread over the block; returns this thread's prefix
// and writes the block total to *total.  scratch: 33 words of shared memory.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* scratch, uint32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  uint32_t inc = warp_incl_scan(v);
  if (lane == 31) scratch[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t s = lane < nw ? scratch[lane] : 0;
    uint32_t si = warp_incl_scan(s);
    if (lane < nw) scratch[lane] = si - s;
    if (lane == nw - 1) scratch[32] = si;
  }
  __syncthreads();
  uint32_t r = scratch[w] + inc - v;
  uint32_t t = scratch[32];
  __syncthreads();
  *total = t;
  return r;
}

// ------------------------------------------------------------------ cell keys
// Four particles per thread: 16-byte loads of the positions (planes and keys are 16-byte
// aligned, so a full group of four is), one 16-byte store of the keys; the ragged end one
// by one.
constexpr int kKeyPPT = 4;

__global__ void __launch_bounds__(256) k_cell_keys(const double* __restrict__ px, const double* __restrict__ py,
                                                   const double* __restrict__ pz, int64_t n, CellKeyK ck,
                                                   uint32_t* __restrict__ keys) {
  const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kKeyPPT;
  if (i0 + kKeyPPT <= n) {
    const double2 x0 = *reinterpret_cast<const double2*>(px + i0), x1 = *reinterpret_cast<const double2*>(px + i0 + 2);
    const double2 y0 = *reinterpret_cast<const double2*>(py + i0), y1 = *reinterpret_cast<const double2*>(py + i0 + 2);
    const double2 z0 = *reinterpret_cast<const double2*>(pz + i0), z1 = *reinterpret_cast<const double2*>(pz + i0 + 2);
    *reinterpret_cast<uint4*>(keys + i0) =
        make_uint4(cell_key(x0.x, y0.x, z0.x, ck), cell_key(x0.y, y0.y, z0.y, ck), cell_key(x1.x, y1.x, z1.x, ck),
                   cell_key(x1.y, y1.y, z1.y, ck));
  } else {
    for (int64_t i = i0; i < n; ++i) keys[i] = cell_key(px[i], py[i], pz[i], ck);
  }
}

CellKeyK make_cell_key_k(int grid) {
  const double c = (double)grid / SOAX_TWO_PI_HOST;
  uint64_t cb;
  std::memcpy(&cb, &c, sizeof cb);
  CellKeyK k;
  k.cm = (cb & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  k.ce = (int)((cb >> 52) & 0x7FF);
  // c 2^54 rounded to an integer (c < 2^8 for G <= 1024, so it fits 62 bits).
  k.cfx = (uint64_t)std::llround(std::ldexp(c, 54));
  k.G = grid;
  return k;
}

// ------------------------------------------------------------------ radix passes
// gate: NULL, or a device flag; the radix kernels return at once while it is 0 (the cell
// counting sort below has done the work).
__global__ void __launch_bounds__(kSortBlock) k_radix_upsweep(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                                              uint32_t mask, int64_t nblocks,
                                                              uint32_t* __restrict__ counts,
                                                              uint32_t* __restrict__ totals, const int* gate) {
  if (gate && *gate == 0) return;
  __shared__ uint32_t hist[kMaxRadix];
  const int radix = (int)mask + 1, tid = threadIdx.x, lane = tid & 31;
  const uint32_t lt = (1u << lane) - 1;
  // One tile per block, or several when the grid is smaller than the tile count.
  for (int64_t tile = blockIdx.x; tile < nblocks; tile += gridDim.x) {
    for (int d = tid; d < radix; d += kSortBlock) hist[d] = 0;
    __syncthreads();
    const int64_t base = tile * kTile;
    // All loads first, so that their latencies overlap.
    uint32_t dg[kSortItems];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
      const int64_t i = base + (int64_t)j * kSortBlock + tid;
      dg[j] = i < n ? ((keys[i] >> shift) & mask) : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
      // Warp-aggregated increment: sorted input puts many equal digits in one warp.
      const uint32_t d = dg[j];
      const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
      if (d != 0xFFFFFFFFu && (peers & lt) == 0) atomicAdd(&hist[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int d = tid; d < radix; d += kSortBlock) {
      uint32_t c = hist[d];
      counts[(int64_t)d * nblocks + tile] = c;
      if (c) atomicAdd(&totals[d], c);
    }
    __syncthreads();
  }
}

// One block per digit d: counts[d][b] <- sum_{d' < d} totals[d'] + sum_{b' < b} counts[d][b'].
__global__ void __launch_bounds__(kScanThreads) k_radix_scan_rows(uint32_t* __restrict__ counts,
                                                                  const uint32_t* __restrict__ totals,
                                                                  int64_t nblocks, const int* gate) {
  if (gate && *gate == 0) return;
  __shared__ uint32_t scratch[33];
  const int d = blockIdx.x, tid = threadIdx.x;
  uint32_t part = 0;
  for (int k = tid; k < d; k += kScanThreads) part += totals[k];
  uint32_t base;
  block_excl_scan(part, scratch, &base);
  uint32_t* row = counts + (int64_t)d * nblocks;
  const int64_t per = (nblocks + kScanThreads - 1) / kScanThreads;
  const int64_t lo = tid * per, hi = lo + per < nblocks ? lo + per : nblocks;
  uint32_t s = 0;
  for (int64_t k = lo; k < hi; ++k) s += row[k];
  uint32_t tot;
  uint32_t excl = block_excl_scan(s, scratch, &tot) + base;
  for (int64_t k = lo; k < hi; ++k) {
    uint32_t c = row[k];
    row[k] = excl;
    excl += c;
  }
}

// LOOP: the grid may be smaller than the tile count (each block loops over tiles); without
// it every block takes exactly its own tile.
template <bool LOOP>
__global__ void __launch_bounds__(kSortBlock, 3) k_radix_downsweep(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, uint32_t* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out, int64_t n, int shift, uint32_t mask, int64_t nblocks,
    const uint32_t* __restrict__ counts, int* __restrict__ status, const int* gate) {
  if (gate && *gate == 0) return;
  extern __shared__ uint32_t sm[];
  const int radix = (int)mask + 1;
  uint32_t* wc = sm;                         // [warps][radix]: per-warp digit counts, then prefixes
  uint32_t* boff = wc + kSortWarps * radix;  // [radix]: block-local digit offsets
  uint32_t* gbase = boff + radix;            // [radix]: global offset minus local offset
  uint32_t* sk = gbase + radix;              // [tile] staged keys
  uint32_t* sv = sk + kTile;                 // [tile] staged values
  __shared__ uint32_t scratch[33];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  bool over = false;
  // One tile per block, or several when the grid is smaller than the tile count.
  for (int64_t tile = blockIdx.x; tile < nblocks; tile += gridDim.x) {
  for (int k = tid; k < kSortWarps * radix; k += kSortBlock) wc[k] = 0;
  __syncthreads();
  const int64_t tile0 = tile * kTile;
  const int tcount = (int)(n - tile0 < kTile ? n - tile0 : kTile);
  const uint32_t lt = (1u << lane) - 1;
  uint32_t kr[kSortItems], vr[kSortItems], rk[kSortItems];
  // Load the warp's 512 elements first (their latencies overlap; the ranking loop below
  // synchronises the warp, which would otherwise keep each load behind the previous
  // round).
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int li = w * (kTile / kSortWarps) + r * 32 + lane;
    const int64_t i = tile0 + li;
    kr[r] = li < tcount ? keys_in[i] : 0u;
    vr[r] = li < tcount ? (vals_in ? vals_in[i] : (uint32_t)i) : 0u;
  }
  // Stable ranking: warp w owns tile elements [w*512, (w+1)*512) in rounds of 32.
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int li = w * (kTile / kSortWarps) + r * 32 + lane;
    const bool valid = li < tcount;
    const uint32_t d = valid ? ((kr[r] >> shift) & mask) : 0xFFFFFFFFu;
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
    uint32_t rank = 0;
    if (valid) rank = wc[w * radix + d] + __popc(peers & lt);
    __syncwarp();
    if (valid && (peers & lt) == 0) wc[w * radix + d] += __popc(peers);
    __syncwarp();
    rk[r] = rank;
  }
  __syncthreads();
  // Per digit: prefix over warps, block count.
  for (int d = tid; d < radix; d += kSortBlock) {
    uint32_t run = 0;
    for (int ww = 0; ww < kSortWarps; ++ww) {
      uint32_t c = wc[ww * radix + d];
      wc[ww * radix + d] = run;
      run += c;
    }
    boff[d] = run;
  }
  __syncthreads();
  // Exclusive scan of the block's digit counts (radix <= 2 * kSortBlock).
  {
    const int d0 = 2 * tid, d1 = 2 * tid + 1;
    uint32_t c0 = d0 < radix ? boff[d0] : 0, c1 = d1 < radix ? boff[d1] : 0, tot;
    uint32_t ex = block_excl_scan(c0 + c1, scratch, &tot);
    if (d0 < radix) boff[d0] = ex;
    if (d1 < radix) boff[d1] = ex + c0;
  }
  __syncthreads();
  for (int d = tid; d < radix; d += kSortBlock) gbase[d] = counts[(int64_t)d * nblocks + tile] - boff[d];
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int li = w * (kTile / kSortWarps) + r * 32 + lane;
    if (li < tcount) {
      uint32_t d = (kr[r] >> shift) & mask;
      uint32_t lp = boff[d] + wc[w * radix + d] + rk[r];
      sk[lp] = kr[r];
      sv[lp] = vr[r];
    }
  }
  __syncthreads();
  for (int li = tid; li < tcount; li += kSortBlock) {
    uint32_t key = sk[li];
    // Only a corrupted workspace (digit offsets overwritten meanwhile) puts dest outside
    // the output: it is clamped to the last element rather than written out of bounds,
    // and recorded once per thread after the loop.
    const uint32_t raw = gbase[(key >> shift) & mask] + (uint32_t)li;
    over |= raw >= (uint32_t)n;  // n < 2^31
    const uint32_t dest = min(raw, (uint32_t)n - 1u);
    if (keys_out) keys_out[dest] = key;
    vals_out[dest] = sv[li];
  }
  if constexpr (!LOOP) break;
  __syncthreads();  // the tile's staging area and counters are free for the next tile
  }
  if (over) atomicExch(status, (int)SOAX_EINVAL);
}

static size_t downsweep_smem(int radix) { return (size_t)(kSortWarps * radix + 2 * radix + 2 * kTile) * 4; }

// ------------------------------------------------------------------ permute
struct PermArgs {
  const void* in[kMaxPlanes];
  void* out[kMaxPlanes];
  int32_t es[kMaxPlanes];
  int nplanes;
  int64_t n;     // outputs: out_f[i] for 0 <= i < n
  int64_t nsrc;  // inputs: perm entries must be < nsrc
  const uint32_t* perm;
  int* status;  // device status word: an index >= nsrc is recorded here and not read
};

__global__ void __launch_bounds__(256) k_permute(const __grid_constant__ PermArgs a) {
  const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (i0 >= a.n) return;
  if (i0 + 4 <= a.n) {
    uint4 p = *reinterpret_cast<const uint4*>(a.perm + i0);
    if (p.x >= a.nsrc || p.y >= a.nsrc || p.z >= a.nsrc || p.w >= a.nsrc) {
      // Not a permutation of 0..nsrc-1: report and gather element 0 instead.
      atomicExch(a.status, (int)SOAX_EINVAL);
      if (p.x >= a.nsrc) p.x = 0;
      if (p.y >= a.nsrc) p.y = 0;
      if (p.z >= a.nsrc) p.z = 0;
      if (p.w >= a.nsrc) p.w = 0;
    }
    for (int f = 0; f < a.nplanes; ++f) {
      const int es = a.es[f];
      if (es == 8) {
        const unsigned long long* s = static_cast<const unsigned long long*>(a.in[f]);
        unsigned long long* o = static_cast<unsigned long long*>(a.out[f]) + i0;
        unsigned long long v0 = s[p.x], v1 = s[p.y], v2 = s[p.z], v3 = s[p.w];
        reinterpret_cast<ulonglong2*>(o)[0] = make_ulonglong2(v0, v1);
        reinterpret_cast<ulonglong2*>(o)[1] = make_ulonglong2(v2, v3);
      } else if (es == 4) {
        const uint32_t* s = static_cast<const uint32_t*>(a.in[f]);
        *reinterpret_cast<uint4*>(static_cast<uint32_t*>(a.out[f]) + i0) = make_uint4(s[p.x], s[p.y], s[p.z], s[p.w]);
      } else {
        const uint8_t* s = static_cast<const uint8_t*>(a.in[f]);
        uint32_t v = (uint32_t)s[p.x] | ((uint32_t)s[p.y] << 8) | ((uint32_t)s[p.z] << 16) | ((uint32_t)s[p.w] << 24);
        *reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(a.out[f]) + i0) = v;
      }
    }
  } else {
    for (int64_t i = i0; i < a.n; ++i) {
      uint32_t p = a.perm[i];
      if (p >= a.nsrc) {
        atomicExch(a.status, (int)SOAX_EINVAL);
        p = 0;
      }
      for (int f = 0; f < a.nplanes; ++f) {
        const int es = a.es[f];
        if (es == 8)
          static_cast<unsigned long long*>(a.out[f])[i] = static_cast<const unsigned long long*>(a.in[f])[p];
        else if (es == 4)
          static_cast<uint32_t*>(a.out[f])[i] = static_cast<const uint32_t*>(a.in[f])[p];
        else
          static_cast<uint8_t*>(a.out[f])[i] = static_cast<const uint8_t*>(a.in[f])[p];
      }
    }
  }
}

// ------------------------------------------------------------------ cell counting sort
// The stable argsort of cell keys of at most 18 bits (grids up to 64^3) in one pass over
// the keys plus per-cell work, for keys that come in near cell order (the keys of the
// particles a previous sort left in cell order, after a few steps).  Every aligned
// 32-key segment of the input is cut into groups of equal keys (one warp match):
//   probe:   groups per segment on sample segments: keys in no particular order leave
//            the sort to the radix passes at once (below);
//   count:   per key d, its particle count m_d (one atomic per group), then the totals
//            of every 4096 keys;
//   scan:    bucket starts (exclusive sums of m);
//   scatter: each group reserves cnt consecutive slots of its key's bucket (one atomic)
//            and writes its indices there in lane order;
//   order:   one warp per key: every group of the bucket is one chunk of consecutive
//            slots, and chunks from different groups come from different segments
//            (disjoint, ascending index ranges), so a chunk ends where the segment of
//            the index (index / 32) changes, and the stable order of the bucket is its
//            chunks ranked by segment; each chunk's destination is the count of the
//            bucket's particles in chunks of smaller segment, and one pass moves every
//            index there.
// A key with more than kCellMaxParticles particles (found by the scan) or more than
// kCellMaxGroups chunks (found by the order kernel) does not fit the per-warp buffers:
// the gate is raised and the radix passes (behind the counting sort: in a graph's
// conditional node, or launched gated) sort instead of this sort; scatter and order
// return at once once it is raised.  Nothing waits on another block.
constexpr int kCellMaxParticles = 2048;  // per key: the per-warp chunk-id table
constexpr int kCellMaxGroups = 256;      // per key: 8 chunk keys per lane in the warp sort
constexpr int kCellChunk = 4096;         // keys per scan block
constexpr int kCellBlock = 256;
constexpr int kCellOrderWarps = 8;

struct CellSortArgs {
  const uint32_t* keys;
  int64_t n;
  uint32_t mask;           // 2^bits - 1; keys are taken modulo 2^bits, as the radix sort does
  int nb;                  // 2^bits buckets
  uint32_t* cnt;           // [nb] particle counts, then the slot cursors
  uint32_t* start;         // [nb + 1] bucket starts
  uint32_t* chunk_tot;     // [nchunks] particle totals of each 4096 keys
  int* gate;               // 0: this sort's result stands; 1: the radix passes sort
  uint32_t* probe;         // [2] sampled segments and their groups
  uint32_t* tmp;           // [n] indices in bucket order, unordered within a bucket
  uint32_t* perm;          // [n] the stable argsort
  uint32_t* skeys;         // [n] sorted keys, or NULL
};

// Segments per warp iteration in the count and scatter kernels: their key loads are in
// flight together.
constexpr int kSegBatch = 8;

// The probe: groups per segment on evenly spread sample segments (one per warp of the
// launch).  Keys in no particular order (a set never sorted) give up to 32 groups per
// segment and would overflow the order kernel's chunk tables after a full count and
// scatter; with more than kProbeGroups groups per segment on average the count raises the
// gate first and the counting sort returns at once.
constexpr int kProbeGroups = 12;
constexpr int kProbeBlocks = 148;

__global__ void __launch_bounds__(kCellBlock) k_cell_probe(const __grid_constant__ CellSortArgs a) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1;
  const int64_t nseg = (a.n + 31) / 32;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (wid >= nseg) return;  // uniform per warp
  const int64_t sg = nseg <= nw ? wid : wid * nseg / nw;
  const int64_t i = sg * 32 + lane;
  const uint32_t d = i < a.n ? (a.keys[i] & a.mask) : 0xFFFFFFFFu;
  const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
  const uint32_t lead = __ballot_sync(0xFFFFFFFFu, d != 0xFFFFFFFFu && (peers & lt) == 0);
  if (lane == 0) {
    atomicAdd(&a.probe[0], 1u);
    atomicAdd(&a.probe[1], (uint32_t)__popc(lead));
  }
}

__global__ void __launch_bounds__(kCellBlock) k_cell_count(const __grid_constant__ CellSortArgs a) {
  // Keys in no particular order: the radix passes sort (the probe's verdict, uniform).
  if (a.probe[1] > (uint32_t)kProbeGroups * a.probe[0]) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(a.gate, 1);
    return;
  }
  if (*a.gate) return;
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1;
  const int64_t nseg = (a.n + 31) / 32;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t sg0 = w0 * kSegBatch; sg0 < nseg; sg0 += wstride * kSegBatch) {
    uint32_t d[kSegBatch];
#pragma unroll
    for (int k = 0; k < kSegBatch; ++k) {
      const int64_t i = (sg0 + k) * 32 + lane;
      d[k] = i < a.n ? (a.keys[i] & a.mask) : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int k = 0; k < kSegBatch; ++k) {
      const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d[k]);
      if (d[k] != 0xFFFFFFFFu && (peers & lt) == 0) atomicAdd(&a.cnt[d[k]], (uint32_t)__popc(peers));
    }
  }
}

// One block of kScanThreads per 4096 keys: the particle total of its keys.
__global__ void __launch_bounds__(kScanThreads) k_cell_chunk_totals(const __grid_constant__ CellSortArgs a) {
  if (*a.gate) return;
  __shared__ uint32_t scratch[33];
  const int b0 = blockIdx.x * kCellChunk + threadIdx.x * 4;
  uint32_t sm = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (b0 + j < a.nb) sm += a.cnt[b0 + j];
  uint32_t tm;
  block_excl_scan(sm, scratch, &tm);
  if (threadIdx.x == 0) a.chunk_tot[blockIdx.x] = tm;
}

// One block of kScanThreads per 4096 keys: bucket starts, the slot cursors, and the gate
// for keys with more particles than the order kernel takes.
__global__ void __launch_bounds__(kScanThreads) k_cell_scan(const __grid_constant__ CellSortArgs a) {
  if (*a.gate) return;
  __shared__ uint32_t scratch[33];
  __shared__ uint32_t s_base;
  const int c = blockIdx.x, tid = threadIdx.x;
  if (tid == 0) {
    uint32_t b = 0;
    for (int k = 0; k < c; ++k) b += a.chunk_tot[k];
    s_base = b;
  }
  __syncthreads();
  const int b0 = c * kCellChunk + tid * 4;
  uint32_t m[4], sm = 0;
  bool big = false;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    m[j] = b0 + j < a.nb ? a.cnt[b0 + j] : 0u;
    big |= m[j] > (uint32_t)kCellMaxParticles;
    sm += m[j];
  }
  uint32_t tm;
  uint32_t em = block_excl_scan(sm, scratch, &tm) + s_base;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int b = b0 + j;
    if (b < a.nb) {
      a.start[b] = em;
      a.cnt[b] = em;  // the slot cursor
    }
    em += m[j];
  }
  if (c == gridDim.x - 1 && tid == blockDim.x - 1) a.start[a.nb] = em;
  if (big) atomicExch(a.gate, 1);
}

__global__ void __launch_bounds__(kCellBlock) k_cell_scatter(const __grid_constant__ CellSortArgs a) {
  if (*a.gate) return;
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1;
  const int64_t nseg = (a.n + 31) / 32;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t sg0 = w0 * kSegBatch; sg0 < nseg; sg0 += wstride * kSegBatch) {
    uint32_t d[kSegBatch], peers[kSegBatch], slot[kSegBatch];
#pragma unroll
    for (int k = 0; k < kSegBatch; ++k) {
      const int64_t i = (sg0 + k) * 32 + lane;
      d[k] = i < a.n ? (a.keys[i] & a.mask) : 0xFFFFFFFFu;
    }
    // Every group's reservation first (independent atomics, in flight together) ...
#pragma unroll
    for (int k = 0; k < kSegBatch; ++k) {
      peers[k] = __match_any_sync(0xFFFFFFFFu, d[k]);
      slot[k] = 0;
      if (d[k] != 0xFFFFFFFFu && (peers[k] & lt) == 0) slot[k] = atomicAdd(&a.cnt[d[k]], (uint32_t)__popc(peers[k]));
    }
    // ... then the indices into their slots (a slot beyond the n indices, only possible
    // if the workspace is overwritten while the sort runs, is not written).
#pragma unroll
    for (int k = 0; k < kSegBatch; ++k) {
      const uint32_t sl = __shfl_sync(0xFFFFFFFFu, slot[k], __ffs(peers[k]) - 1) + __popc(peers[k] & lt);
      if (d[k] != 0xFFFFFFFFu && sl < (uint32_t)a.n) a.tmp[sl] = (uint32_t)((sg0 + k) * 32 + lane);
    }
  }
}

// Ascending bitonic sort of 32 K values held K per lane (lane l holds positions
// l K .. l K + K - 1).
template <int K, typename T>
__device__ __forceinline__ void warp_bitonic(T (&r)[K]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int kk = 2; kk <= 32 * K; kk <<= 1) {
#pragma unroll
    for (int j = kk >> 1; j > 0; j >>= 1) {
      if (j < K) {  // both partners in this lane
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const int p = k ^ j;
          if (p > k) {
            const bool up = ((lane * K + k) & kk) == 0;
            const T x = r[k], y = r[p];
            const bool sw = up ? (x > y) : (x < y);
            r[k] = sw ? y : x;
            r[p] = sw ? x : y;
          }
        }
      } else {  // the partner in lane ^ (j / K), same register
        const int lj = j / K;
        const bool lower = (lane & lj) == 0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const T o = __shfl_xor_sync(0xFFFFFFFFu, r[k], lj);
          const bool up = ((lane * K + k) & kk) == 0;
          r[k] = (lower == up) ? (r[k] < o ? r[k] : o) : (r[k] > o ? r[k] : o);
        }
      }
    }
  }
}

// Per-warp tables of the order kernel.
struct CellWarpSmem {
  uint16_t cid[kCellMaxParticles];   // chunk of each slot
  uint16_t coff[kCellMaxGroups + 1]; // first slot of each chunk (coff[C] = m)
  uint16_t cdst[kCellMaxGroups];     // destination of each chunk's first slot
  uint32_t cseg[kCellMaxGroups];     // segment of each chunk
};

// The chunks of a bucket ranked by segment (C <= 32 K): their destinations into t.cdst.
// The sort key is (segment, chunk): 32 bits while every segment is below 2^24 - 1
// (fewer than 2^29 - 32 particles), else 64; padding is all ones, above every key.
template <int K, typename T>
__device__ __forceinline__ void cell_rank_chunks(CellWarpSmem& t, uint32_t C) {
  const int lane = threadIdx.x & 31;
  constexpr int kShift = sizeof(T) == 4 ? 8 : 16;
  constexpr T kNone = ~T(0);
  T r[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint32_t c = (uint32_t)(lane * K + k);
    r[k] = c < C ? (T)(((T)t.cseg[c] << kShift) | c) : kNone;
  }
  warp_bitonic<K, T>(r);
  uint32_t cn[K], cc[K], local = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    cc[k] = (uint32_t)(r[k] & ((T(1) << kShift) - 1));
    cn[k] = r[k] == kNone ? 0u : (uint32_t)t.coff[cc[k] + 1] - t.coff[cc[k]];
    local += cn[k];
  }
  uint32_t incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += v;
  }
  uint32_t dest = incl - local;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (cn[k]) t.cdst[cc[k]] = (uint16_t)dest;
    dest += cn[k];
  }
}

// Chunk discovery over R rows of 32 slots (v: the indices, rows r0 ..): a slot starts a
// chunk where its index's segment differs from the previous slot's.  C and carry (the
// previous row's last segment) run across calls.
template <int R>
__device__ __forceinline__ void cell_find_chunks(const uint32_t (&v)[R], uint32_t r0, uint32_t m, uint32_t& C,
                                                 uint32_t& carry, CellWarpSmem& t) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1;
#pragma unroll
  for (int b = 0; b < R; ++b) {
    const uint32_t j = (r0 + b) * 32 + lane;
    const uint32_t sg = j < m ? (v[b] >> 5) : 0xFFFFFFFFu;
    uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, sg, 1);
    if (lane == 0) prev = carry;
    const bool s0 = j < m && sg != prev;
    const uint32_t mk = __ballot_sync(0xFFFFFFFFu, s0);
    const uint32_t c = C + __popc(mk & lt) - (s0 ? 0u : 1u);  // this slot's chunk
    if (j < m && c < (uint32_t)kCellMaxGroups) {
      t.cid[j] = (uint16_t)c;
      if (s0) {
        t.coff[c] = (uint16_t)j;
        t.cseg[c] = sg;
      }
    }
    C += __popc(mk);
    carry = __shfl_sync(0xFFFFFFFFu, sg, 31);
  }
}

// Every slot of R rows (v: the indices) to its chunk's destination.
template <int R>
__device__ __forceinline__ void cell_move(const uint32_t (&v)[R], uint32_t r0, uint32_t m, const CellWarpSmem& t,
                                          uint32_t* perm) {
  const int lane = threadIdx.x & 31;
  uint32_t q[R];
#pragma unroll
  for (int b = 0; b < R; ++b) {
    const uint32_t j = (r0 + b) * 32 + lane;
    if (j < m) {
      const uint32_t c = t.cid[j];
      q[b] = (uint32_t)t.cdst[c] + (j - t.coff[c]);
    }
  }
#pragma unroll
  for (int b = 0; b < R; ++b) {
    const uint32_t j = (r0 + b) * 32 + lane;
    if (j < m) perm[q[b]] = v[b];
  }
}

template <int R>
__device__ __forceinline__ void cell_load_rows(const uint32_t* src, uint32_t r0, uint32_t m, uint32_t (&v)[R]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int b = 0; b < R; ++b) {
    const uint32_t j = (r0 + b) * 32 + lane;
    v[b] = j < m ? src[j] : 0u;
  }
}

template <typename T>
__device__ __forceinline__ void cell_rank_t(CellWarpSmem& t, uint32_t C) {
  if (C <= 32)
    cell_rank_chunks<1, T>(t, C);
  else if (C <= 64)
    cell_rank_chunks<2, T>(t, C);
  else if (C <= 128)
    cell_rank_chunks<4, T>(t, C);
  else
    cell_rank_chunks<8, T>(t, C);
}

constexpr int kOrderRowsHeld = 16;  // a bucket of up to 512 slots stays in registers
constexpr int kOrderRows = 8;       // larger buckets: rows of 32 slots loaded together

template <typename T>
__global__ void __launch_bounds__(kCellOrderWarps * 32, 3) k_cell_order(const __grid_constant__ CellSortArgs a) {
  if (*a.gate) return;
  __shared__ CellWarpSmem s_tab[kCellOrderWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  CellWarpSmem& t = s_tab[w];
  const int64_t wstride = (int64_t)gridDim.x * kCellOrderWarps;
  int64_t d = (int64_t)blockIdx.x * kCellOrderWarps + w;
  uint32_t st = 0, en = 0;
  if (d < a.nb) {
    st = a.start[d];
    en = a.start[d + 1];
  }
  for (; d < a.nb; d += wstride) {
    // The next bucket's bounds, read while this one is ordered.
    const int64_t dn = d + wstride;
    uint32_t stn = 0, enn = 0;
    if (dn < a.nb) {
      stn = a.start[dn];
      enn = a.start[dn + 1];
    }
    // Bounds outside the n slots (only possible if the workspace is overwritten while
    // the sort runs): the radix passes sort instead (uniform per warp).
    if (st > en || en > (uint32_t)a.n) {
      if (lane == 0) atomicExch(a.gate, 1);
      return;
    }
    const uint32_t m = en - st;
    if (m > 0) {
      if (a.skeys)
        for (uint32_t j = lane; j < m; j += 32) a.skeys[st + j] = (uint32_t)d;
      uint32_t C = 0, carry = 0xFFFFFFFFu;
      bool over = false;
      if (m <= 32 * kOrderRowsHeld) {
        uint32_t v[kOrderRowsHeld];
        cell_load_rows<kOrderRowsHeld>(a.tmp + st, 0, m, v);
        cell_find_chunks<kOrderRowsHeld>(v, 0, m, C, carry, t);
        over = C > (uint32_t)kCellMaxGroups;
        if (!over) {
          if (lane == 0) t.coff[C] = (uint16_t)m;
          __syncwarp();
          cell_rank_t<T>(t, C);
          __syncwarp();
          cell_move<kOrderRowsHeld>(v, 0, m, t, a.perm + st);
        }
      } else {
        for (uint32_t r0 = 0; r0 * 32 < m; r0 += kOrderRows) {
          uint32_t v[kOrderRows];
          cell_load_rows<kOrderRows>(a.tmp + st, r0, m, v);
          cell_find_chunks<kOrderRows>(v, r0, m, C, carry, t);
        }
        over = C > (uint32_t)kCellMaxGroups;
        if (!over) {
          if (lane == 0) t.coff[C] = (uint16_t)m;
          __syncwarp();
          cell_rank_t<T>(t, C);
          __syncwarp();
          for (uint32_t r0 = 0; r0 * 32 < m; r0 += kOrderRows) {
            uint32_t v[kOrderRows];
            cell_load_rows<kOrderRows>(a.tmp + st, r0, m, v);
            cell_move<kOrderRows>(v, r0, m, t, a.perm + st);
          }
        }
      }
      if (over) {  // beyond the warp's tables: the radix passes sort
        if (lane == 0) atomicExch(a.gate, 1);
        return;
      }
      __syncwarp();
    }
    st = stn;
    en = enn;
  }
}

static int key_bits_for_grid(int G) {
  uint32_t maxkey = (uint32_t)G * G * G - 1;
  int b = 0;
  while (b < 32 && (maxkey >> b)) ++b;
  return b < 1 ? 1 : b;
}

struct SortWs {
  size_t off_keys, off_skeys, off_perm, off_radix, total;
  RadixPlan rp;
  // The cell counting sort (grids up to 64^3): its zeroed header (gate, counts, chunk
  // totals), the bucket starts, and its index array, which shares the radix region (the
  // radix passes only run, gated, after the counting sort is done).
  bool cell = false;
  int bits = 0, nb = 0, nchunks = 0;
  size_t off_hdr = 0, hdr_bytes = 0, off_start = 0, off_tmp = 0;
};

constexpr int kCellMaxBits = 18;

static SortWs sort_ws_plan(int64_t n, int G) {
  SortWs w;
  size_t off = 0;
  w.off_keys = off;
  off = align256(off + (size_t)n * 4);
  w.off_skeys = off;
  off = align256(off + (size_t)n * 4);
  w.off_perm = off;
  off = align256(off + (size_t)n * 4);
  w.bits = key_bits_for_grid(G);
  w.rp = radix_plan(n, w.bits);
  w.cell = w.bits <= kCellMaxBits;
  if (w.cell) {
    w.nb = 1 << w.bits;
    w.nchunks = (w.nb + kCellChunk - 1) / kCellChunk;
    w.off_hdr = off;  // gate and probe counters (256 B), cnt[nb], chunk totals[nchunks]
    w.hdr_bytes = 256 + (size_t)w.nb * 4 + (size_t)w.nchunks * 4;
    off = align256(off + w.hdr_bytes);
    w.off_start = off;
    off = align256(off + (size_t)(w.nb + 1) * 4);
  }
  w.off_radix = off;
  size_t tail = w.rp.total;
  if (w.cell) {
    w.off_tmp = off;
    if ((size_t)n * 4 > tail) tail = (size_t)n * 4;
  }
  w.total = off + tail;
  return w;
}

static int find_position_field(soax_t h) {
  for (size_t f = 0; f < h->fields.size(); ++f)
    if (h->fields[f].tag == 'P' && h->fields[f].dtype == SOAX_F64 && h->fields[f].ncomp == 3) return (int)f;
  return -1;
}

}  // namespace soax

using namespace soax;

extern "C" int soax_cell_keys(soax_t h, int32_t pos_field, int32_t grid, uint32_t* keys, void* stream) {
  if (int r = check_handle(h)) return r;
  if (int r = check_field(h, pos_field, SOAX_F64, 3, "soax_cell_keys position")) return r;
  if (grid < 1 || grid > 1024) return fail(SOAX_EINVAL, "soax_cell_keys: grid must be in 1..1024");
  if (h->n == 0) return SOAX_OK;
  if (!keys) return fail(SOAX_EINVAL, "soax_cell_keys: keys is NULL");
  if (!aligned16(keys)) return fail(SOAX_EALIGN, "soax_cell_keys: keys not 16-byte aligned");
  const int fp = h->fields[pos_field].first_plane;
  const double* px = (const double*)h->planes[h->current][fp];
  const double* py = (const double*)h->planes[h->current][fp + 1];
  const double* pz = (const double*)h->planes[h->current][fp + 2];
  if (!px || !py || !pz) return fail(SOAX_EUNBOUND, "soax_cell_keys: position planes not bound");
  k_cell_keys<<<grid_for((h->n + kKeyPPT - 1) / kKeyPPT, 256), 256, 0, as_stream(stream)>>>(px, py, pz, h->n,
                                                                                              make_cell_key_k(grid), keys);
  return check_launch("soax_cell_keys");
}

extern "C" int soax_radix_workspace_bytes(int64_t n, int32_t key_bits, size_t* bytes) {
  if (!bytes) return fail(SOAX_EINVAL, "soax_radix_workspace_bytes: NULL");
  if (n < 0 || n >= (int64_t(1) << 31)) return fail(SOAX_EINVAL, "soax_radix_workspace_bytes: n out of range");
  if (key_bits < 1 || key_bits > 32) return fail(SOAX_EINVAL, "soax_radix_workspace_bytes: key_bits in 1..32");
  *bytes = radix_plan(n, key_bits).total;
  return SOAX_OK;
}

namespace soax {
static int radix_sort_gated(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out, uint32_t* vals_out,
                            int64_t n, int32_t key_bits, void* ws, size_t ws_bytes, void* stream, const int* gate);
}  // namespace soax

extern "C" int soax_radix_sort_pairs(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                                     uint32_t* vals_out, int64_t n, int32_t key_bits, void* ws, size_t ws_bytes,
                                     void* stream) {
  return soax::radix_sort_gated(keys_in, vals_in, keys_out, vals_out, n, key_bits, ws, ws_bytes, stream, nullptr);
}

namespace soax {
// The downsweep's shared memory above 48 KB and the largest carveout, set once per device.
static int radix_prepare() {
  static std::mutex mu;
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return SOAX_OK;
  std::lock_guard<std::mutex> lk(mu);
  if (attr_set[dev]) return SOAX_OK;
  for (const void* fn : {(const void*)k_radix_downsweep<false>, (const void*)k_radix_downsweep<true>}) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)downsweep_smem(kMaxRadix));
    // Prefer shared memory over L1 so that three 53 KB blocks fit on an SM.
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return cuda_fail(e, "soax_radix_sort_pairs: smem attribute");
  }
  attr_set[dev] = true;
  return SOAX_OK;
}

// The radix sort; gate as for the kernels (NULL: always sort).
static int radix_sort_gated(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out, uint32_t* vals_out,
                            int64_t n, int32_t key_bits, void* ws, size_t ws_bytes, void* stream, const int* gate) {
  if (n < 0 || n >= (int64_t(1) << 31)) return fail(SOAX_EINVAL, "soax_radix_sort_pairs: n out of range");
  if (key_bits < 1 || key_bits > 32) return fail(SOAX_EINVAL, "soax_radix_sort_pairs: key_bits in 1..32");
  if (n == 0) return SOAX_OK;
  if (!keys_in || !vals_out || !ws) return fail(SOAX_EINVAL, "soax_radix_sort_pairs: NULL pointer");
  if (!aligned16(keys_in) || !aligned16(vals_in) || !aligned16(keys_out) || !aligned16(vals_out) || !aligned16(ws))
    return fail(SOAX_EALIGN, "soax_radix_sort_pairs: pointers must be 16-byte aligned");
  if (keys_out == keys_in || (vals_in && vals_out == vals_in) || (const uint32_t*)vals_out == keys_in)
    return fail(SOAX_EINVAL, "soax_radix_sort_pairs: outputs must not alias inputs");
  RadixPlan p = radix_plan(n, key_bits);
  if (ws_bytes < p.total) return fail(SOAX_ENOMEM, "soax_radix_sort_pairs: workspace too small");
  if (int r = radix_prepare()) return r;
  char* w = static_cast<char*>(ws);
  uint32_t* counts = reinterpret_cast<uint32_t*>(w + p.off_counts);
  uint32_t* totals = reinterpret_cast<uint32_t*>(w + p.off_totals);
  uint32_t* ak[2] = {reinterpret_cast<uint32_t*>(w + p.off_ak[0]), reinterpret_cast<uint32_t*>(w + p.off_ak[1])};
  uint32_t* av[2] = {reinterpret_cast<uint32_t*>(w + p.off_av[0]), reinterpret_cast<uint32_t*>(w + p.off_av[1])};
  cudaStream_t s = as_stream(stream);
  int* status = status_word();
  if (!status) return fail(SOAX_ECUDA, "soax_radix_sort_pairs: status word");
  for (int pass = 0; pass < p.passes; ++pass) {
    const int shift = pass * p.width;
    const int width = key_bits - shift < p.width ? key_bits - shift : p.width;
    const uint32_t mask = (uint32_t)((1u << width) - 1);
    const int radix = (int)mask + 1;
    const bool last = pass == p.passes - 1;
    const uint32_t* kin = pass == 0 ? keys_in : ak[(pass - 1) & 1];
    const uint32_t* vin = pass == 0 ? vals_in : av[(pass - 1) & 1];
    uint32_t* kout = last ? keys_out : ak[pass & 1];
    uint32_t* vout = last ? vals_out : av[pass & 1];
    cudaError_t e = cudaMemsetAsync(totals, 0, (size_t)radix * 4, s);
    if (e != cudaSuccess) return cuda_fail(e, "soax_radix_sort_pairs: memset");
    // Gated (behind the cell counting sort, usually with nothing to do): grids that fill
    // the GPU once, each block looping over tiles, so that returning at once costs little.
    const unsigned gu = gate ? (unsigned)persistent_grid((const void*)k_radix_upsweep, kSortBlock, 0, p.nblocks)
                             : (unsigned)p.nblocks;
    const unsigned gd = gate ? (unsigned)persistent_grid((const void*)k_radix_downsweep<true>, kSortBlock,
                                                         downsweep_smem(radix), p.nblocks)
                             : (unsigned)p.nblocks;
    k_radix_upsweep<<<gu, kSortBlock, 0, s>>>(kin, n, shift, mask, p.nblocks, counts, totals, gate);
    if (int r = check_launch("radix upsweep")) return r;
    k_radix_scan_rows<<<radix, kScanThreads, 0, s>>>(counts, totals, p.nblocks, gate);
    if (int r = check_launch("radix scan")) return r;
    if (gate)
      k_radix_downsweep<true><<<gd, kSortBlock, downsweep_smem(radix), s>>>(kin, vin, kout, vout, n, shift, mask,
                                                                           p.nblocks, counts, status, gate);
    else
      k_radix_downsweep<false><<<gd, kSortBlock, downsweep_smem(radix), s>>>(kin, vin, kout, vout, n, shift, mask,
                                                                            p.nblocks, counts, status, gate);
    if (int r = check_launch("radix downsweep")) return r;
  }
  return SOAX_OK;
}
}  // namespace soax

namespace soax {

// Particles [i0, i0 + cnt) of the other buffer set from the live set through perm
// (out_f[i] = in_f[perm[i]], perm indexed like the particles); the live set does not
// flip.  i0 a multiple of 4 (aligned vector access of perm and of the outputs); both
// buffer sets bound and perm 16-byte aligned (the caller checks).
int permute_range(soax_t h, const uint32_t* perm, int64_t i0, int64_t cnt, void* stream) {
  const int src = h->current, dst = src ^ 1;
  if (cnt <= 0) return SOAX_OK;
  if (i0 % 4 != 0) return fail(SOAX_EINVAL, "permute_range: first index not a multiple of 4");
  PermArgs a;
  for (int p = 0; p < h->nplanes; ++p) {
    a.in[p] = h->planes[src][p];
    a.out[p] = static_cast<char*>(h->planes[dst][p]) + i0 * h->plane_esize[p];
    a.es[p] = h->plane_esize[p];
  }
  a.nplanes = h->nplanes;
  a.n = cnt;
  a.nsrc = h->n;
  a.perm = perm + i0;
  a.status = status_word();
  if (!a.status) return fail(SOAX_ECUDA, "soax_permute: status word");
  k_permute<<<grid_for((cnt + 3) / 4, 256), 256, 0, as_stream(stream)>>>(a);
  return check_launch("soax_permute");
}

// Byte offsets of the cell-key region and of the permutation in a workspace of
// soax_sort_workspace_bytes bytes (the key region takes a caller's keys, as in
// soax_sort_by_cell).
void sort_ws_regions(int64_t n, int grid, size_t* off_keys, size_t* off_perm) {
  const SortWs w = sort_ws_plan(n, grid);
  *off_keys = w.off_keys;
  *off_perm = w.off_perm;
}

}  // namespace soax

extern "C" int soax_permute(soax_t h, const uint32_t* perm, void* stream) {
  if (int r = check_handle(h)) return r;
  const int src = h->current, dst = src ^ 1;
  if (h->n == 0) {
    h->current = dst;
    return SOAX_OK;
  }
  if (!perm) return fail(SOAX_EINVAL, "soax_permute: perm is NULL");
  if (!aligned16(perm)) return fail(SOAX_EALIGN, "soax_permute: perm not 16-byte aligned");
  if (int r = live_planes_bound(h, src)) return r;
  if (int r = live_planes_bound(h, dst)) return r;
  if (int r = soax::permute_range(h, perm, 0, h->n, stream)) return r;
  h->current = dst;
  return SOAX_OK;
}

extern "C" int soax_sort_workspace_bytes(soax_t h, int32_t grid, size_t* bytes) {
  if (int r = check_handle(h)) return r;
  if (!bytes) return fail(SOAX_EINVAL, "soax_sort_workspace_bytes: NULL");
  if (grid < 1 || grid > 1024) return fail(SOAX_EINVAL, "soax_sort_workspace_bytes: grid must be in 1..1024");
  *bytes = sort_ws_plan(h->n, grid).total;
  return SOAX_OK;
}

extern "C" int soax_sort_results(soax_t h, int32_t grid, void* ws, size_t ws_bytes, uint32_t** sorted_keys,
                                 uint32_t** perm) {
  if (int r = check_handle(h)) return r;
  if (grid < 1 || grid > 1024) return fail(SOAX_EINVAL, "soax_sort_results: grid must be in 1..1024");
  SortWs w = sort_ws_plan(h->n, grid);
  if (!ws || ws_bytes < w.total) return fail(SOAX_ENOMEM, "soax_sort_results: workspace too small");
  if (sorted_keys) *sorted_keys = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + w.off_skeys);
  if (perm) *perm = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + w.off_perm);
  return SOAX_OK;
}

namespace soax {

static CellSortArgs cell_args(int64_t n, const SortWs& w, char* base, const uint32_t* keys, uint32_t* skeys,
                              uint32_t* perm) {
  CellSortArgs a;
  a.keys = keys;
  a.n = n;
  a.mask = (uint32_t)(w.nb - 1);
  a.nb = w.nb;
  a.gate = reinterpret_cast<int*>(base + w.off_hdr);
  a.probe = reinterpret_cast<uint32_t*>(base + w.off_hdr + 16);
  a.cnt = reinterpret_cast<uint32_t*>(base + w.off_hdr + 256);
  a.chunk_tot = a.cnt + w.nb;
  a.start = reinterpret_cast<uint32_t*>(base + w.off_start);
  a.tmp = reinterpret_cast<uint32_t*>(base + w.off_tmp);
  a.perm = perm;
  a.skeys = skeys;
  return a;
}

// The counting passes of the cell sort on stream s: zeroed header, probe, count, chunk
// totals, bucket scan, scatter, per-key order (each raises the gate for keys it cannot
// take and returns at once once it is raised).
static int cell_counting_passes(const CellSortArgs& a, const SortWs& w, char* base, cudaStream_t s) {
  const int64_t n = a.n;
  cudaError_t e = cudaMemsetAsync(base + w.off_hdr, 0, w.hdr_bytes, s);
  if (e != cudaSuccess) return cuda_fail(e, "cell sort: memset");
  const int64_t seg_blocks = ((n + 31) / 32 + kSegBatch * (kCellBlock / 32) - 1) / (kSegBatch * (kCellBlock / 32));
  k_cell_probe<<<kProbeBlocks, kCellBlock, 0, s>>>(a);
  if (int r = check_launch("cell sort: probe")) return r;
  const int gc = persistent_grid((const void*)k_cell_count, kCellBlock, 0, seg_blocks);
  k_cell_count<<<gc, kCellBlock, 0, s>>>(a);
  if (int r = check_launch("cell sort: count")) return r;
  k_cell_chunk_totals<<<w.nchunks, kScanThreads, 0, s>>>(a);
  if (int r = check_launch("cell sort: chunk totals")) return r;
  k_cell_scan<<<w.nchunks, kScanThreads, 0, s>>>(a);
  if (int r = check_launch("cell sort: scan")) return r;
  const int gs = persistent_grid((const void*)k_cell_scatter, kCellBlock, 0, seg_blocks);
  k_cell_scatter<<<gs, kCellBlock, 0, s>>>(a);
  if (int r = check_launch("cell sort: scatter")) return r;
  // Chunk sort keys of 32 bits while every segment (index / 32) is below 2^24 - 1 (so no
  // key reaches the all-ones padding value).
  const bool narrow = n <= (int64_t(1) << 29) - 64;
  const void* ko = narrow ? (const void*)k_cell_order<uint32_t> : (const void*)k_cell_order<unsigned long long>;
  const int go = persistent_grid(ko, kCellOrderWarps * 32, 0, (w.nb + kCellOrderWarps - 1) / kCellOrderWarps);
  if (narrow)
    k_cell_order<uint32_t><<<go, kCellOrderWarps * 32, 0, s>>>(a);
  else
    k_cell_order<unsigned long long><<<go, kCellOrderWarps * 32, 0, s>>>(a);
  return check_launch("cell sort: order");
}

// Opens the body of the graph's conditional node (the radix passes) when the counting
// passes raised the gate.
__global__ void k_cell_decide(const int* __restrict__ gate, cudaGraphConditionalHandle h) {
  if (threadIdx.x == 0) cudaGraphSetConditional(h, *gate != 0 ? 1u : 0u);
}

// The cell sort as one CUDA graph per set of pointers and sizes: the counting passes, a
// one-thread kernel that reads the gate, and the radix passes in the body of an IF node
// that runs only when the gate is up.  Launched as streams of kernels, the radix passes
// sit behind the counting sort gated (six launches that return at once, ~16 us at 16.7M
// keys); in the graph they are not launched at all, and the graph's kernels follow one
// another with shorter gaps.
struct CellGraphKey {
  unsigned long long ctx;
  const uint32_t* keys;
  uint32_t* skeys;
  uint32_t* perm;
  void* ws;
  int64_t n;
  int grid;
  bool operator==(const CellGraphKey& o) const {
    return ctx == o.ctx && keys == o.keys && skeys == o.skeys && perm == o.perm && ws == o.ws && n == o.n &&
           grid == o.grid;
  }
};

struct CellGraph {
  CellGraphKey key;
  cudaGraphExec_t exec;  // NULL: building failed, launch the kernels on the stream
};

constexpr size_t kCellGraphCache = 8;
static std::mutex g_cell_graph_mu;
static std::vector<CellGraph> g_cell_graphs;  // most recently used first
static int64_t g_cell_graphs_built = 0, g_cell_graphs_failed = 0;
thread_local bool t_cell_graph_off = false;

// Captures the graph on a private stream.  Any failure leaves *out NULL.
static void build_cell_graph(const CellSortArgs& a, const SortWs& w, char* base, cudaGraphExec_t* out) {
  *out = nullptr;
  if (radix_prepare() != SOAX_OK) return;  // function attributes before the capture
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return;
  cudaGraph_t g = nullptr;
  cudaGraphConditionalHandle hnd;
  bool ok = cudaGraphCreate(&g, 0) == cudaSuccess &&
            cudaGraphConditionalHandleCreate(&hnd, g, 0, cudaGraphCondAssignDefault) == cudaSuccess &&
            cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  bool capturing = ok;
  cudaGraphNodeParams cp = {};
  if (ok) ok = cell_counting_passes(a, w, base, cs) == SOAX_OK;
  if (ok) {
    k_cell_decide<<<1, 32, 0, cs>>>(a.gate, hnd);
    ok = cudaGetLastError() == cudaSuccess;
  }
  if (ok) {
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    cudaGraphNode_t cn;
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hnd;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    ok = cudaStreamGetCaptureInfo(cs, &st, nullptr, nullptr, &deps, nullptr, &nd) == cudaSuccess &&
         st == cudaStreamCaptureStatusActive &&
         cudaGraphAddNode(&cn, g, deps, nullptr, nd, &cp) == cudaSuccess &&
         cudaStreamUpdateCaptureDependencies(cs, &cn, nullptr, 1, cudaStreamSetCaptureDependencies) == cudaSuccess;
  }
  if (capturing) {
    cudaGraph_t done = nullptr;
    ok = cudaStreamEndCapture(cs, &done) == cudaSuccess && ok;
  }
  if (ok) {  // the body: the radix passes, ungated
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    ok = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
         cudaSuccess;
    if (ok) {
      ok = radix_sort_gated(a.keys, nullptr, a.skeys, a.perm, a.n, w.bits, base + w.off_radix, w.rp.total, cs,
                            nullptr) == SOAX_OK;
      cudaGraph_t done = nullptr;
      ok = cudaStreamEndCapture(cs, &done) == cudaSuccess && ok;
    }
  }
  if (ok) ok = cudaGraphInstantiate(out, g, 0) == cudaSuccess;
  if (!ok) *out = nullptr;
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  cudaGetLastError();  // a failed build falls back to the stream form, leaving no error behind
}

// Launches the cached graph for these pointers and sizes (built on first use) on s; sets
// *launched to false when there is none (its build failed).  The launch happens under
// the cache's lock, so another thread cannot evict and destroy the graph in between.
static int cell_graph_launch(const CellSortArgs& a, const SortWs& w, char* base, int grid, cudaStream_t s,
                             bool* launched) {
  *launched = false;
  const CellGraphKey key{current_context_id(), a.keys, a.skeys, a.perm, base, a.n, grid};
  std::lock_guard<std::mutex> lk(g_cell_graph_mu);
  cudaGraphExec_t ex = nullptr;
  bool found = false;
  for (size_t i = 0; i < g_cell_graphs.size(); ++i) {
    if (g_cell_graphs[i].key == key) {
      const CellGraph hit = g_cell_graphs[i];
      g_cell_graphs.erase(g_cell_graphs.begin() + i);
      g_cell_graphs.insert(g_cell_graphs.begin(), hit);
      ex = hit.exec;
      found = true;
      break;
    }
  }
  if (!found) {
    CellGraph gnew{key, nullptr};
    build_cell_graph(a, w, base, &gnew.exec);
    ++(gnew.exec ? g_cell_graphs_built : g_cell_graphs_failed);
    if (g_cell_graphs.size() >= kCellGraphCache) {
      // An executable graph still running is freed when it completes.
      if (g_cell_graphs.back().exec) cudaGraphExecDestroy(g_cell_graphs.back().exec);
      g_cell_graphs.pop_back();
    }
    g_cell_graphs.insert(g_cell_graphs.begin(), gnew);
    ex = gnew.exec;
  }
  if (!ex) return SOAX_OK;
  const cudaError_t e = cudaGraphLaunch(ex, s);
  if (e != cudaSuccess) return cuda_fail(e, "cell sort: graph launch");
  *launched = true;
  return SOAX_OK;
}

// Whether the calling thread's cell sorts launch their kernels on the stream instead of
// a graph (for callers that must not create graphs); returns the previous setting.
bool set_cell_graph_off(bool off) {
  const bool prev = t_cell_graph_off;
  t_cell_graph_off = off;
  return prev;
}

// The stable argsort of n cell keys on a grid^3 grid into perm (and the sorted keys into
// skeys unless NULL), in the workspace laid out by sort_ws_plan: the cell counting sort
// for grids up to 64^3 (the radix passes behind it for keys it cannot take: in the body
// of a graph's conditional node, or gated on the stream when the caller's stream is
// being captured or graphs are off), the radix sort alone beyond.
static int cell_argsort(const uint32_t* keys, uint32_t* skeys, uint32_t* perm, int64_t n, int grid, void* ws,
                        void* stream) {
  const SortWs w = sort_ws_plan(n, grid);
  char* base = static_cast<char*>(ws);
  if (!w.cell)
    return radix_sort_gated(keys, nullptr, skeys, perm, n, w.bits, base + w.off_radix, w.rp.total, stream, nullptr);
  if (!aligned16(keys)) return fail(SOAX_EALIGN, "cell sort: keys not 16-byte aligned");
  const CellSortArgs a = cell_args(n, w, base, keys, skeys, perm);
  cudaStream_t s = as_stream(stream);
  cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
  if (!t_cell_graph_off && cudaStreamIsCapturing(s, &cst) == cudaSuccess && cst == cudaStreamCaptureStatusNone) {
    bool launched = false;
    if (int r = cell_graph_launch(a, w, base, grid, s, &launched)) return r;
    if (launched) return SOAX_OK;
  }
  if (int r = cell_counting_passes(a, w, base, s)) return r;
  return radix_sort_gated(keys, nullptr, skeys, perm, n, w.bits, base + w.off_radix, w.rp.total, stream, a.gate);
}

}  // namespace soax

// The sort of the given keys and the permute-gather (soax_sort_by_cell after its key
// pass).  keys may lie in the workspace's own key region.
static int sort_by_keys_impl(soax_t h, int32_t grid, const uint32_t* keys, void* ws, void* stream) {
  const SortWs w = sort_ws_plan(h->n, grid);
  char* base = static_cast<char*>(ws);
  uint32_t* skeys = reinterpret_cast<uint32_t*>(base + w.off_skeys);
  uint32_t* perm = reinterpret_cast<uint32_t*>(base + w.off_perm);
  if (int r = cell_argsort(keys, skeys, perm, h->n, grid, ws, stream)) return r;
  return soax_permute(h, perm, stream);
}

extern "C" int soax_sort_perm(soax_t h, int32_t grid, const uint32_t* keys, void* ws, size_t ws_bytes,
                              void* stream) {
  if (int r = check_handle(h)) return r;
  if (grid < 1 || grid > 1024) return fail(SOAX_EINVAL, "soax_sort_perm: grid must be in 1..1024");
  const SortWs w = sort_ws_plan(h->n, grid);
  if (h->n == 0) return SOAX_OK;
  if (!keys) return fail(SOAX_EINVAL, "soax_sort_perm: keys is NULL");
  if (!aligned16(keys)) return fail(SOAX_EALIGN, "soax_sort_perm: keys not 16-byte aligned");
  if (!ws || ws_bytes < w.total) return fail(SOAX_ENOMEM, "soax_sort_perm: workspace too small");
  if (!aligned16(ws)) return fail(SOAX_EALIGN, "soax_sort_perm: workspace not 16-byte aligned");
  char* base = static_cast<char*>(ws);
  return cell_argsort(keys, nullptr, reinterpret_cast<uint32_t*>(base + w.off_perm), h->n, grid, ws, stream);
}

extern "C" int soax_sort_by_keys(soax_t h, int32_t grid, const uint32_t* keys, void* ws, size_t ws_bytes,
                                 void* stream) {
  if (int r = check_handle(h)) return r;
  if (grid < 1 || grid > 1024) return fail(SOAX_EINVAL, "soax_sort_by_keys: grid must be in 1..1024");
  const SortWs w = sort_ws_plan(h->n, grid);
  if (h->n == 0) return SOAX_OK;
  if (!keys) return fail(SOAX_EINVAL, "soax_sort_by_keys: keys is NULL");
  if (!aligned16(keys)) return fail(SOAX_EALIGN, "soax_sort_by_keys: keys not 16-byte aligned");
  if (!ws || ws_bytes < w.total) return fail(SOAX_ENOMEM, "soax_sort_by_keys: workspace too small");
  if (!aligned16(ws)) return fail(SOAX_EALIGN, "soax_sort_by_keys: workspace not 16-byte aligned");
  if (int r = live_planes_bound(h, h->current)) return r;
  if (int r = live_planes_bound(h, h->current ^ 1)) return r;
  return sort_by_keys_impl(h, grid, keys, ws, stream);
}

extern "C" int soax_sort_by_cell(soax_t h, int32_t grid, void* ws, size_t ws_bytes, void* stream) {
  if (int r = check_handle(h)) return r;
  if (grid < 1 || grid > 1024) return fail(SOAX_EINVAL, "soax_sort_by_cell: grid must be in 1..1024");
  const int pf = find_position_field(h);
  if (pf < 0) return fail(SOAX_ESCHEMA, "soax_sort_by_cell: no f64 x 3 field tagged 'P'");
  SortWs w = sort_ws_plan(h->n, grid);
  if (h->n == 0) return SOAX_OK;
  if (!ws || ws_bytes < w.total) return fail(SOAX_ENOMEM, "soax_sort_by_cell: workspace too small");
  if (!aligned16(ws)) return fail(SOAX_EALIGN, "soax_sort_by_cell: workspace not 16-byte aligned");
  if (int r = live_planes_bound(h, h->current)) return r;
  if (int r = live_planes_bound(h, h->current ^ 1)) return r;
  uint32_t* keys = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + w.off_keys);
  if (int r = soax_cell_keys(h, pf, grid, keys, stream)) return r;
  return sort_by_keys_impl(h, grid, keys, ws, stream);
}

extern "C" int soax_sort_graph_counts(int64_t* built, int64_t* failed) {
  if (!built || !failed) return soax::fail(SOAX_EINVAL, "soax_sort_graph_counts: NULL");
  std::lock_guard<std::mutex> lk(soax::g_cell_graph_mu);
  *built = soax::g_cell_graphs_built;
  *failed = soax::g_cell_graphs_failed;
  return SOAX_OK;
}
