// Handle management, schema validation, AoS layout and status reporting.
#include <cstring>
#include <mutex>
#include <new>
#include <set>

#include "soax_internal.h"

namespace {
thread_local std::string g_last_error;
// Per-device status word: a device-side check that fails stores its code here.
__device__ int g_status_word;
}  // namespace

namespace soax {

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(SOAX_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, what);
  return SOAX_OK;
}

int dtype_size(int dtype) {
  switch (dtype) {
    case SOAX_I32: return 4;
    case SOAX_I64: return 8;
    case SOAX_U8: return 1;
    case SOAX_F32: return 4;
    case SOAX_F64: return 8;
    default: return 0;
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

unsigned long long current_context_id() {
  // cuCtxGetCurrent and cuCtxGetId through the runtime's driver entry points (no link
  // against libcuda).  A context's id is unique for the life of the process, so a device
  // whose primary context was destroyed and created again (cudaDeviceReset) gets a new id.
  typedef int (*get_current_t)(void**);
  typedef int (*get_id_t)(void*, unsigned long long*);
  static get_current_t get_current = nullptr;
  static get_id_t get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<get_current_t>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<get_id_t>(f);
  });
  if (!get_current || !get_id) return 0;
  void* ctx = nullptr;
  if (get_current(&ctx) != 0 || !ctx) return 0;
  unsigned long long id = 0;
  if (get_id(ctx, &id) != 0) return 0;
  return id;
}

int device_symbol_address(const void* symbol, SymbolCache* cache, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= SymbolCache::kDevices) return fail(SOAX_EUNSUPPORTED, "device index >= 64");
  std::lock_guard<std::mutex> lk(cache->mu);
  unsigned long long id = current_context_id();
  if (id == 0 || cache->ctx[dev] != id || !cache->ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, symbol);
    if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress");
    cache->ptr[dev] = p;
    cache->ctx[dev] = current_context_id();  // the lookup makes the primary context current
  }
  *out = cache->ptr[dev];
  return SOAX_OK;
}

int* status_word() {
  static SymbolCache cache;
  void* p = nullptr;
  if (device_symbol_address(&g_status_word, &cache, &p) != SOAX_OK) return nullptr;
  return static_cast<int*>(p);
}

int check_handle(soax_t h) {
  if (!h) return fail(SOAX_EINVAL, "null handle");
  return SOAX_OK;
}

int check_field(soax_t h, int f, int dtype, int ncomp, const char* role) {
  if (f < 0 || f >= (int)h->fields.size())
    return fail(SOAX_ESCHEMA, std::string(role) + ": field index out of range");
  const Field& F = h->fields[f];
  if (F.dtype != dtype || F.ncomp != ncomp)
    return fail(SOAX_ESCHEMA, std::string(role) + ": field '" + F.name + "' has the wrong type or ncomp");
  return SOAX_OK;
}

int live_planes_bound(soax_t h, int buf) {
  if (h->n == 0) return SOAX_OK;
  for (int p = 0; p < h->nplanes; ++p)
    if (!h->planes[buf][p])
      return fail(SOAX_EUNBOUND, "plane " + std::to_string(p) + " of buffer " + std::to_string(buf) + " is not bound");
  return SOAX_OK;
}

}  // namespace soax

using namespace soax;

extern "C" int soax_version(void) { return 1; }

extern "C" const char* soax_last_error(void) { return g_last_error.c_str(); }

extern "C" int soax_create(const soax_field_desc* fields, int32_t nfields, int64_t n, soax_t* out) {
  if (!out) return fail(SOAX_EINVAL, "soax_create: out is NULL");
  *out = nullptr;
  if (n < 0 || n >= (int64_t(1) << 31)) return fail(SOAX_EINVAL, "soax_create: n out of range [0, 2^31)");
  if (nfields < 1 || nfields > kMaxFields || !fields) return fail(SOAX_ESCHEMA, "soax_create: need 1..32 fields");
  soax_s* h = new (std::nothrow) soax_s();
  if (!h) return fail(SOAX_EINVAL, "soax_create: out of host memory");
  h->n = n;
  h->capacity = n;
  std::set<std::string> names;
  int plane = 0;
  for (int f = 0; f < nfields; ++f) {
    const soax_field_desc& d = fields[f];
    int es = dtype_size(d.dtype);
    if (!d.name || !d.name[0] || std::strlen(d.name) > 31 || es == 0 || d.ncomp < 1 || d.ncomp > 16) {
      delete h;
      return fail(SOAX_ESCHEMA, "soax_create: field " + std::to_string(f) + " is malformed");
    }
    if (!names.insert(d.name).second) {
      delete h;
      return fail(SOAX_ESCHEMA, std::string("soax_create: duplicate field name '") + d.name + "'");
    }
    if (plane + d.ncomp > kMaxPlanes) {
      delete h;
      return fail(SOAX_ESCHEMA, "soax_create: more than 64 planes");
    }
    Field F{d.name, d.dtype, d.ncomp, d.tag, es, plane};
    for (int c = 0; c < d.ncomp; ++c) h->plane_esize[plane + c] = es;
    plane += d.ncomp;
    h->fields.push_back(F);
  }
  h->nplanes = plane;
  // Natural C struct layout (Listing 1 / Listing 4).
  int64_t off = 0, maxal = 1;
  for (const Field& F : h->fields) {
    int64_t al = F.esize;
    if (al > maxal) maxal = al;
    off = (off + al - 1) / al * al;
    h->offsets.push_back(off);
    off += al * F.ncomp;
  }
  h->record_bytes = (off + maxal - 1) / maxal * maxal;
  *out = h;
  return SOAX_OK;
}

namespace soax {
void release_host_pipe(const soax_s* h);  // host_step.cu: the events of soax_step_host
}

extern "C" int soax_destroy(soax_t h) {
  if (h) soax::release_host_pipe(h);
  delete h;
  return SOAX_OK;
}

extern "C" int soax_size(soax_t h, int64_t* n, int32_t* nfields, int32_t* nplanes) {
  if (int e = check_handle(h)) return e;
  if (n) *n = h->n;
  if (nfields) *nfields = (int32_t)h->fields.size();
  if (nplanes) *nplanes = h->nplanes;
  return SOAX_OK;
}

extern "C" int soax_set_size(soax_t h, int64_t n) {
  if (int e = check_handle(h)) return e;
  if (n < 0 || n > h->capacity)
    return fail(SOAX_EINVAL, "soax_set_size: n must be in 0..capacity (" + std::to_string(h->capacity) + ")");
  h->n = n;
  return SOAX_OK;
}

extern "C" int soax_bind(soax_t h, int32_t field, int32_t comp, int32_t buf, void* dev_ptr) {
  if (int e = check_handle(h)) return e;
  if (field < 0 || field >= (int)h->fields.size()) return fail(SOAX_EINVAL, "soax_bind: bad field");
  if (comp < 0 || comp >= h->fields[field].ncomp) return fail(SOAX_EINVAL, "soax_bind: bad component");
  if (buf != 0 && buf != 1) return fail(SOAX_EINVAL, "soax_bind: buf must be 0 or 1");
  if (!dev_ptr && h->n > 0) return fail(SOAX_EINVAL, "soax_bind: NULL pointer");
  if (!aligned16(dev_ptr)) return fail(SOAX_EALIGN, "soax_bind: pointer not 16-byte aligned");
  h->planes[buf][h->fields[field].first_plane + comp] = dev_ptr;
  return SOAX_OK;
}

extern "C" int soax_copy_plane(soax_t h, int32_t field, int32_t comp, void* host, int32_t to_device, void* stream) {
  if (int e = check_handle(h)) return e;
  if (field < 0 || field >= (int)h->fields.size()) return fail(SOAX_EINVAL, "soax_copy_plane: bad field");
  if (comp < 0 || comp >= h->fields[field].ncomp) return fail(SOAX_EINVAL, "soax_copy_plane: bad component");
  if (to_device != 0 && to_device != 1) return fail(SOAX_EINVAL, "soax_copy_plane: to_device must be 0 or 1");
  if (h->n == 0) return SOAX_OK;
  if (!host) return fail(SOAX_EINVAL, "soax_copy_plane: host is NULL");
  const int p = h->fields[field].first_plane + comp;
  void* dev = h->planes[h->current][p];
  if (!dev) return fail(SOAX_EINVAL, "soax_copy_plane: plane not bound");
  const size_t bytes = (size_t)h->n * (size_t)h->plane_esize[p];
  const cudaError_t e = to_device ? cudaMemcpyAsync(dev, host, bytes, cudaMemcpyHostToDevice, as_stream(stream))
                                  : cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, as_stream(stream));
  return e == cudaSuccess ? SOAX_OK : cuda_fail(e, "soax_copy_plane");
}

extern "C" int soax_current(soax_t h, int32_t* buf) {
  if (int e = check_handle(h)) return e;
  if (!buf) return fail(SOAX_EINVAL, "soax_current: NULL");
  *buf = h->current;
  return SOAX_OK;
}

extern "C" int soax_set_current(soax_t h, int32_t buf) {
  if (int e = check_handle(h)) return e;
  if (buf != 0 && buf != 1) return fail(SOAX_EINVAL, "soax_set_current: buf must be 0 or 1");
  h->current = buf;
  return SOAX_OK;
}

extern "C" int soax_aos_layout(soax_t h, int64_t* record_bytes, int64_t* field_offsets) {
  if (int e = check_handle(h)) return e;
  if (record_bytes) *record_bytes = h->record_bytes;
  if (field_offsets)
    for (size_t f = 0; f < h->fields.size(); ++f) field_offsets[f] = h->offsets[f];
  return SOAX_OK;
}

extern "C" int soax_sync(void* stream) {
  cudaError_t e = cudaStreamSynchronize(as_stream(stream));
  if (e != cudaSuccess) return cuda_fail(e, "soax_sync");
  int s = 0;
  e = cudaMemcpyFromSymbol(&s, g_status_word, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "soax_sync: status read");
  if (s != 0) {
    int zero = 0;
    e = cudaMemcpyToSymbol(g_status_word, &zero, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "soax_sync: status clear");
    return fail(s, "soax_sync: a device-side check failed (status " + std::to_string(s) + ")");
  }
  return SOAX_OK;
}
