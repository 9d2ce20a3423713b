// Host-side internals shared by the library's translation units (not installed).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/soax.h"

#define SOAX_TWO_PI_HOST 6.283185307179586  // binary64 nearest to 2pi

namespace soax {

constexpr int kMaxPlanes = 64;
constexpr int kMaxFields = 32;

struct Field {
  std::string name;
  int dtype;
  int ncomp;
  char tag;
  int esize;        // bytes per scalar
  int first_plane;  // index of component 0 in the plane table
};

}  // namespace soax

struct soax_s {
  int64_t n = 0;         // current number of particles
  int64_t capacity = 0;  // n at creation: every bound plane holds this many elements
  std::vector<soax::Field> fields;
  int nplanes = 0;
  void* planes[2][soax::kMaxPlanes] = {};
  int plane_esize[soax::kMaxPlanes] = {};
  int current = 0;
  int64_t record_bytes = 0;
  std::vector<int64_t> offsets;  // AoS byte offset of each field
};

namespace soax {

// Error reporting: sets the thread's last-error message and returns code.
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
// Check the launch that was just made (cudaGetLastError).
int check_launch(const char* what);

int dtype_size(int dtype);
// Id of the calling thread's current CUDA context (0 if none or unknown).
unsigned long long current_context_id();
// Per-device cache of a __device__ variable's address, valid for one context.
struct SymbolCache {
  static constexpr int kDevices = 64;
  std::mutex mu;
  void* ptr[kDevices] = {};
  unsigned long long ctx[kDevices] = {};
};
// Device address of a __device__ variable on the current device: looked up with
// cudaGetSymbolAddress on the first call for that device and again whenever the current
// context is not the one the cached address was taken in (after cudaDeviceReset the
// module is loaded again and the variable may move).  The lookup can load the module, so
// the first call on a device belongs before any stream capture.
int device_symbol_address(const void* symbol, SymbolCache* cache, void** out);
// Device address of this device's status word, or null.
int* status_word();
bool aligned16(const void* p);

// Validation helpers used by several entry points.
int check_handle(soax_t h);
int check_field(soax_t h, int f, int dtype, int ncomp, const char* role);
int live_planes_bound(soax_t h, int buf);

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline int grid_for(int64_t work_items, int block) {
  int64_t g = (work_items + block - 1) / block;
  return (int)(g < 1 ? 1 : g);
}

struct EnsArgs;
struct FlowK;
// Grid of a persistent kernel: resident blocks per SM x SMs, at most work_blocks.
int persistent_grid(const void* kern, int block, size_t smem, int64_t work_blocks);
// Validate fl against h's schema and fill the kernel arguments for buffer set buf.
int make_ens_args(soax_t h, const soax_flow* fl, int buf, EnsArgs* e, FlowK* f, const char* who);

}  // namespace soax
