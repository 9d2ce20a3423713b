// soax_sort_by_cell_noalloc: the cell sort for callers that cannot hand the library a
// device workspace.
//
// Some hosts of this library cannot allocate device memory at the point where they want
// to sort: C or Fortran particle codes that link libsoax directly and have no device
// allocator of their own, or simulation loops that forbid cudaMalloc between time steps
// because it may synchronise the whole device and eat into a memory budget fixed at
// start-up.  This entry point runs the same keys / radix sort / permute-gather as
// soax_sort_by_cell, with its scratch (keys, sorted keys, permutation, digit counts and
// the radix ping-pong buffers) in one file-scope device array instead of a caller
// workspace.  The array is sized for at most kNoAllocMaxParticles particles on a grid of
// at most kNoAllocMaxGrid cells per side; every GPU that loads the library holds it
// until the process exits.
#include "soax_internal.h"

namespace {

constexpr int64_t kNoAllocMaxParticles = int64_t(1) << 20;  // 1,048,576 particles
constexpr int kNoAllocMaxGrid = 64;                         // keys of at most 18 bits
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;   // 32 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch per device and context: looked up with that device
// current on its first use, and again if the context changed since (cudaDeviceReset
// reloads the module).  In host code the array's name is only a host-side stand-in, never
// a device address.
soax::SymbolCache g_noalloc_cache;

int noalloc_scratch(void** out) {
  if (int r = soax::device_symbol_address(&g_noalloc_scratch, &g_noalloc_cache, out))
    return soax::fail(r, std::string("soax_sort_by_cell_noalloc: ") + soax_last_error());
  return SOAX_OK;
}

}  // namespace

namespace soax {
bool set_cell_graph_off(bool off);  // sort.cu
}  // namespace soax

extern "C" int soax_sort_by_cell_noalloc(soax_t h, int32_t grid, uint32_t* perm_out, void* stream) {
  using namespace soax;
  if (int r = check_handle(h)) return r;
  if (grid < 1 || grid > kNoAllocMaxGrid)
    return fail(SOAX_EINVAL, "soax_sort_by_cell_noalloc: grid must be in 1..64 (static scratch limit)");
  if (h->n > kNoAllocMaxParticles)
    return fail(SOAX_EINVAL, "soax_sort_by_cell_noalloc: at most 1048576 particles fit the static scratch (n = " +
                                 std::to_string(h->n) + "); use soax_sort_by_cell with a workspace");
  size_t need = 0;
  if (int r = soax_sort_workspace_bytes(h, grid, &need)) return r;
  if (need > kNoAllocScratchBytes) return fail(SOAX_ENOMEM, "soax_sort_by_cell_noalloc: static scratch too small");
  if (h->n == 0) return soax_sort_by_cell(h, grid, nullptr, 0, stream);
  void* ws = nullptr;
  if (int r = noalloc_scratch(&ws)) return r;
  // The sort clears what it counts into (the cell sort's counts and gate, the radix
  // sort's per-pass digit totals) itself; every other part of the scratch is fully
  // written before it is read, so nothing left from an earlier call is used.  Its kernels
  // go on the stream, not into a CUDA graph (instantiating one is an allocation).
  const bool prev = set_cell_graph_off(true);
  const int rs = soax_sort_by_cell(h, grid, ws, kNoAllocScratchBytes, stream);
  set_cell_graph_off(prev);
  if (rs) return rs;
  if (perm_out) {
    uint32_t* perm = nullptr;
    if (int r = soax_sort_results(h, grid, ws, kNoAllocScratchBytes, nullptr, &perm)) return r;
    cudaError_t e = cudaMemcpyAsync(perm_out, perm, (size_t)h->n * sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                                    as_stream(stream));
    if (e != cudaSuccess) return cuda_fail(e, "soax_sort_by_cell_noalloc: copy of the permutation");
  }
  return SOAX_OK;
}
