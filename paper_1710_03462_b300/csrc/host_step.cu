// soax_step_host: one sort interval (fused steps with cell keys, stable cell sort,
// permute-gather of every plane) of a particle set held in host memory, streamed through
// the device in pieces of consecutive particles.
//
// Three streams: the uploads (host -> live planes) on up, the steps, the sort and the
// gathers on the compute stream, the downloads (other buffer set -> host) on down.  Piece
// c is stepped as soon as its upload has landed (event up[c]), and downloaded as soon as
// its gather has run (event gathered[c]), so the device time of the steps hides under
// the uploads and the two link directions work at once; only the sort and the first
// piece's gather sit between the last upload and the first download.  The next call's
// upload of a piece waits for this call's download of the same particles (event down[c]):
// the host buffer is the same, and so is the device range (the gather target is the
// next call's live set).
#include <algorithm>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "../../include/soax_host.h"
#include "soax_internal.h"
#include "step_core.cuh"

namespace soax {

int permute_range(soax_t h, const uint32_t* perm, int64_t i0, int64_t cnt, void* stream);  // sort.cu
void sort_ws_regions(int64_t n, int grid, size_t* off_keys, size_t* off_perm);             // sort.cu

namespace {

constexpr int kDefaultChunks = 16;
constexpr int kMaxChunks = 1024;
constexpr int64_t kChunkAlign = 16;  // particles: every piece starts 16-byte aligned in every plane

// The events of a handle's pipeline and the pieces of its last call.
struct Pipe {
  int dev = -1;
  cudaEvent_t start = nullptr;
  std::vector<cudaEvent_t> up, gathered, down;
  std::vector<int64_t> lo, hi;  // the last call's pieces: [lo[c], hi[c])
  bool pending = false;         // that call's downloads may still be in flight
  // A call made with defer leaves its downloads to the next call (interleaved with its
  // uploads) or to soax_step_host_finish: where they go, where they come from, and how
  // many of its pieces have been enqueued.
  bool deferred = false;
  std::vector<void*> dhost;
  int dbuf = 0;
  size_t ndone = 0;
};

std::mutex g_mu;
std::unordered_map<const soax_s*, Pipe> g_pipes;

void destroy_events(Pipe& p) {
  if (p.start) cudaEventDestroy(p.start);
  for (auto* v : {&p.up, &p.gathered, &p.down})
    for (cudaEvent_t e : *v)
      if (e) cudaEventDestroy(e);
  p.start = nullptr;
  p.up.clear();
  p.gathered.clear();
  p.down.clear();
}

int make_event(cudaEvent_t* e) {
  const cudaError_t err = cudaEventCreateWithFlags(e, cudaEventDisableTiming);
  return err == cudaSuccess ? SOAX_OK : cuda_fail(err, "soax_step_host: event");
}

// At least nchunks events of each kind on the current device.  Events are only added
// (an earlier call's waits may still name them), or all replaced when the device changed.
int ensure_events(Pipe& p, int nchunks) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cuda_fail(cudaGetLastError(), "soax_step_host: device");
  if (p.dev != dev) {
    destroy_events(p);
    p.pending = false;  // the earlier call ran on another device's streams
    p.dev = dev;
  }
  if (!p.start)
    if (int r = make_event(&p.start)) return r;
  while ((int)p.up.size() < nchunks) {
    cudaEvent_t a = nullptr, b = nullptr, c = nullptr;
    if (int r = make_event(&a)) return r;
    if (int r = make_event(&b)) return cudaEventDestroy(a), r;
    if (int r = make_event(&c)) return cudaEventDestroy(a), cudaEventDestroy(b), r;
    p.up.push_back(a);
    p.gathered.push_back(b);
    p.down.push_back(c);
  }
  return SOAX_OK;
}

// Piece boundaries 0 = cut[0] < cut[1] < ... < cut[C] = n, every inner one a multiple of
// kChunkAlign.  The first piece's download and the last piece's upload each run with the
// other link direction idle, and the last piece's step sits before the sort: with four or
// more pieces those two are a quarter of the others.
std::vector<int64_t> plan_pieces(int64_t n, int64_t want) {
  const int64_t units = (n + kChunkAlign - 1) / kChunkAlign;
  if (want > units) want = units;
  std::vector<int64_t> w(want, 4);
  if (want >= 4) w.front() = w.back() = 1;
  int64_t total = 0;
  for (int64_t x : w) total += x;
  std::vector<int64_t> cut{0};
  int64_t acc = 0;
  for (int64_t i = 0; i < want; ++i) {
    acc += w[i];
    int64_t c = (units * acc + total / 2) / total * kChunkAlign;
    if (c > n) c = n;
    if (c > cut.back()) cut.push_back(c);
  }
  if (cut.back() != n) cut.push_back(n);
  return cut;
}

// The handle restricted to particles [i0, i0 + cnt) in both buffer sets: the same
// schema, plane pointers advanced by i0 elements.
soax_s view(const soax_s& h, int64_t i0, int64_t cnt) {
  soax_s v;
  v.n = v.capacity = cnt;
  v.fields = h.fields;
  v.nplanes = h.nplanes;
  v.current = h.current;
  v.record_bytes = h.record_bytes;
  v.offsets = h.offsets;
  for (int p = 0; p < h.nplanes; ++p) {
    v.plane_esize[p] = h.plane_esize[p];
    for (int b = 0; b < 2; ++b)
      v.planes[b][p] = h.planes[b][p] ? static_cast<char*>(h.planes[b][p]) + i0 * h.plane_esize[p] : nullptr;
  }
  return v;
}

int copy(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind, void* s) {
  const cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind, as_stream(s));
  return e == cudaSuccess ? SOAX_OK : cuda_fail(e, "soax_step_host: copy");
}

int record(cudaEvent_t e, void* s) {
  const cudaError_t err = cudaEventRecord(e, as_stream(s));
  return err == cudaSuccess ? SOAX_OK : cuda_fail(err, "soax_step_host: event record");
}

int wait(void* s, cudaEvent_t e) {
  const cudaError_t err = cudaStreamWaitEvent(as_stream(s), e, 0);
  return err == cudaSuccess ? SOAX_OK : cuda_fail(err, "soax_step_host: stream wait");
}

// The download of piece j of a deferred call: after its gather, into its host planes.
int download_piece(soax_t h, Pipe& P, size_t j, void* down) {
  const int64_t a = P.lo[j], cnt = P.hi[j] - P.lo[j];
  if (int r = wait(down, P.gathered[j])) return r;
  for (int p = 0; p < h->nplanes; ++p) {
    const size_t es = (size_t)h->plane_esize[p];
    if (int r = copy(static_cast<char*>(P.dhost[p]) + a * es, static_cast<const char*>(h->planes[P.dbuf][p]) + a * es,
                     cnt * es, cudaMemcpyDeviceToHost, down))
      return r;
  }
  return record(P.down[j], down);
}

// Enqueue what is left of a deferred call's downloads.
int flush_deferred(soax_t h, Pipe& P, void* down) {
  for (; P.ndone < P.lo.size(); ++P.ndone)
    if (int r = download_piece(h, P, P.ndone, down)) return r;
  P.deferred = false;
  return SOAX_OK;
}

int step_host(soax_t h, void* const* host, const soax_flow* fl, int32_t nsteps, int32_t grid, int32_t nchunks,
              int32_t defer, void* ws, size_t ws_bytes, void* stream, void* up, void* down) {
  const char* who = "soax_step_host";
  if (int r = check_handle(h)) return r;
  if (nsteps < 0) return fail(SOAX_EINVAL, std::string(who) + ": nsteps < 0");
  if (grid < 1 || grid > 1024) return fail(SOAX_EINVAL, std::string(who) + ": grid must be in 1..1024");
  if (nchunks < 0 || nchunks > kMaxChunks)
    return fail(SOAX_EINVAL, std::string(who) + ": nchunks must be in 0.." + std::to_string(kMaxChunks));
  if (defer != 0 && defer != 1) return fail(SOAX_EINVAL, std::string(who) + ": defer must be 0 or 1");
  EnsArgs e;
  FlowK f;
  if (int r = make_ens_args(h, fl, h->current, &e, &f, who)) return r;
  const int64_t n = h->n;
  if (n == 0) {  // nothing moves; the live set flips as after soax_permute
    {
      std::lock_guard<std::mutex> lk(g_mu);
      auto it = g_pipes.find(h);
      if (it != g_pipes.end() && it->second.deferred)
        if (int r = flush_deferred(h, it->second, down)) return r;
    }
    h->current ^= 1;
    return SOAX_OK;
  }
  if (!host) return fail(SOAX_EINVAL, std::string(who) + ": host is NULL");
  for (int p = 0; p < h->nplanes; ++p)
    if (!host[p]) return fail(SOAX_EINVAL, std::string(who) + ": host plane " + std::to_string(p) + " is NULL");
  size_t need = 0;
  if (int r = soax_sort_workspace_bytes(h, grid, &need)) return r;
  if (!ws || ws_bytes < need) return fail(SOAX_ENOMEM, std::string(who) + ": workspace too small");
  if (!aligned16(ws)) return fail(SOAX_EALIGN, std::string(who) + ": workspace not 16-byte aligned");
  if (int r = live_planes_bound(h, h->current)) return r;
  if (int r = live_planes_bound(h, h->current ^ 1)) return r;

  const std::vector<int64_t> cut = plan_pieces(n, nchunks ? nchunks : kDefaultChunks);
  const int C = (int)cut.size() - 1;

  std::lock_guard<std::mutex> lk(g_mu);
  Pipe& P = g_pipes[h];
  if (int r = ensure_events(P, C)) return r;
  size_t off_keys = 0, off_perm = 0;
  sort_ws_regions(n, grid, &off_keys, &off_perm);
  uint32_t* keys = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + off_keys);
  const uint32_t* perm = reinterpret_cast<const uint32_t*>(static_cast<char*>(ws) + off_perm);
  const int live = h->current, other = live ^ 1;

  // From here on a failure leaves part of the call enqueued: the next call then waits
  // for every download event (their latest records) before any upload.
  auto failed = [&P](int r) {
    P.lo.assign(P.down.size(), 0);
    P.hi.assign(P.down.size(), INT64_MAX);
    P.pending = true;
    P.deferred = false;
    return r;
  };
  // The previous call's deferred downloads interleave with this call's uploads only when
  // both cut the set the same way; otherwise they are all enqueued first.
  const bool interleave = P.deferred && P.lo.size() == (size_t)C &&
                          std::equal(P.lo.begin(), P.lo.end(), cut.begin());
  if (P.deferred && !interleave)
    if (int r = flush_deferred(h, P, down)) return failed(r);

  // Work already on stream (e.g. the last use of these planes) comes first.
  if (int r = record(P.start, stream)) return failed(r);
  if (int r = wait(up, P.start)) return failed(r);

  // 1. Upload and step piece by piece.
  for (int c = 0; c < C; ++c) {
    const int64_t a = cut[c], cnt = cut[c + 1] - cut[c];
    if (interleave) {
      // The previous call's download of this piece, held back until this call's upload
      // two pieces earlier has landed: the two directions then move together, piece by
      // piece, instead of the downloads running ahead and the uploads finishing alone.
      if (c >= 2)
        if (int r = wait(down, P.up[c - 2])) return failed(r);
      if (int r = download_piece(h, P, (size_t)c, down)) return failed(r);
      P.ndone = (size_t)c + 1;
    }
    if (P.pending)
      for (size_t j = 0; j < P.lo.size(); ++j)
        if (P.lo[j] < a + cnt && a < P.hi[j])
          if (int r = wait(up, P.down[j])) return failed(r);
    for (int p = 0; p < h->nplanes; ++p) {
      const size_t es = (size_t)h->plane_esize[p];
      if (int r = copy(static_cast<char*>(h->planes[live][p]) + a * es, static_cast<const char*>(host[p]) + a * es,
                       cnt * es, cudaMemcpyHostToDevice, up))
        return failed(r);
    }
    if (int r = record(P.up[c], up)) return failed(r);
    if (int r = wait(stream, P.up[c])) return failed(r);
    soax_s v = view(*h, a, cnt);
    if (int r = soax_step_fused_keys(&v, fl, nsteps, grid, keys + a, stream)) return failed(r);
  }

  // 2. The permutation that sorts every key.
  if (int r = soax_sort_perm(h, grid, keys, ws, ws_bytes, stream)) return failed(r);

  // 3. Gather piece by piece, and download each piece (now, or deferred).
  P.lo.assign(cut.begin(), cut.end() - 1);
  P.hi.assign(cut.begin() + 1, cut.end());
  P.dhost.assign(host, host + h->nplanes);
  P.dbuf = other;
  P.ndone = 0;
  P.deferred = false;
  for (int c = 0; c < C; ++c) {
    if (int r = permute_range(h, perm, cut[c], cut[c + 1] - cut[c], stream)) return failed(r);
    if (int r = record(P.gathered[c], stream)) return failed(r);
    if (!defer) {
      if (int r = download_piece(h, P, (size_t)c, down)) return failed(r);
      P.ndone = (size_t)c + 1;
    }
  }
  // stream does not wait for the downloads: the next call's start event on stream must
  // not hold its uploads behind this call's downloads (they overlap them, piece by
  // piece).  The host planes are final once down_stream has passed the call (with defer,
  // the next call or soax_step_host_finish).
  P.deferred = defer != 0;
  P.pending = true;
  h->current = other;
  return SOAX_OK;
}

int step_host_finish(soax_t h, void* down) {
  if (int r = check_handle(h)) return r;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_pipes.find(h);
  if (it == g_pipes.end() || !it->second.deferred) return SOAX_OK;
  Pipe& P = it->second;
  if (int r = flush_deferred(h, P, down)) {
    P.lo.assign(P.down.size(), 0);
    P.hi.assign(P.down.size(), INT64_MAX);
    P.deferred = false;
    return r;
  }
  return SOAX_OK;
}

}  // namespace

// Called by soax_destroy: the handle's events go with it.
void release_host_pipe(const soax_s* h) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_pipes.find(h);
  if (it == g_pipes.end()) return;
  destroy_events(it->second);
  g_pipes.erase(it);
}

}  // namespace soax

extern "C" int soax_step_host(soax_t h, void* const* host, const soax_flow* fl, int32_t nsteps, int32_t grid,
                              int32_t nchunks, int32_t defer, void* ws, size_t ws_bytes, void* stream,
                              void* up_stream, void* down_stream) {
  return soax::step_host(h, host, fl, nsteps, grid, nchunks, defer, ws, ws_bytes, stream, up_stream, down_stream);
}

extern "C" int soax_step_host_finish(soax_t h, void* down_stream) { return soax::step_host_finish(h, down_stream); }
