// Checkpointed forward and hand-written adjoint of the midpoint-RK2 step, and the
// minimum-image loss that seeds it.
//
// Every particle is independent, so one thread owns one particle for the whole
// computation.  The forward keeps the particle in registers for all K steps, with the
// arithmetic of soax_step_fused (position as fixed-point turns T between steps), and
// writes its state (T, v) every C steps (checkpoint j = state before step j*C).  The
// reverse walks the segments backwards: it recomputes a segment from its checkpoint with
// the same per-step function (so the states are bit-identical), pushing the C states on
// a per-particle stack in the workspace (coalesced [step][plane][particle] layout), then
// applies the reverse step C times.  Parameter gradients are reduced in a fixed order
// (per-block tree, then one block over the block partials), so the result is
// bit-reproducible.
#include <cmath>
#include <mutex>

#include "soax_internal.h"
#include "step_fused.cuh"

namespace soax {

constexpr int kAdjBlock = 256;      // the reverse (2 blocks per SM with the scaled tables)
constexpr int kAdjFwdBlock = 512;   // the forward (2 blocks per SM with the scaled tables)
constexpr int kLossBlock = 256;

TurnsK make_turns_k(double dt, double umax);
TurnsK make_turns_k(const soax_flow* fl, const FlowK& f, int nsteps);
double amplitude_bound(const soax_flow* fl);

__host__ __device__ static inline size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct AdjWs {
  size_t state_bytes, off_partials, off_ckpt, off_stack, total;
  int nck;
};

static AdjWs adj_plan(int64_t n, int K, int C) {
  AdjWs w;
  w.state_bytes = a256((size_t)n * 24) + a256((size_t)n * 12);
  w.nck = (int)(((int64_t)K + C - 1) / C);
  const size_t nb_adj = (size_t)((n + kAdjBlock - 1) / kAdjBlock);
  const size_t nb_loss = (size_t)((n + kLossBlock - 1) / kLossBlock);
  w.off_partials = 0;
  w.off_ckpt = a256((nb_adj * 4 > nb_loss ? nb_adj * 4 : nb_loss) * 8 + 8);
  w.off_stack = w.off_ckpt + (size_t)w.nck * w.state_bytes;
  w.total = w.off_stack + (size_t)(K < C ? K : C) * w.state_bytes;
  return w;
}

// A stored state: the position as fixed-point turns (3 u64 planes) and the velocity.
struct StateRef {
  uint64_t* T[3];
  float* v[3];
};

__device__ __forceinline__ StateRef state_at(char* base, size_t sb, int64_t n, int j) {
  char* p = base + (size_t)j * sb;
  StateRef r;
  uint64_t* ts = reinterpret_cast<uint64_t*>(p);
  float* vs = reinterpret_cast<float*>(p + a256((size_t)n * 24));
  for (int c = 0; c < 3; ++c) {
    r.T[c] = ts + (size_t)c * n;
    r.v[c] = vs + (size_t)c * n;
  }
  return r;
}

// One step of the forward and of the recompute alike (soax_step_fused's choice of path,
// so the same bits).
template <bool ACC, class Trig>
__device__ __forceinline__ void adj_step(const StepC& k, const TurnsK& tk, const Trig& tg, bool fast, uint64_t T[3],
                                         float v[3], float a[3]) {
  if (fast && near_shift(k, v))
    rk2_step_turns<ACC, true>(k, tk, tg, T, v, a);
  else
    rk2_step_turns<ACC, false>(k, tk, tg, T, v, a);
}

// The forward's K steps from (T, v), writing the state before every C-th step as a
// checkpoint.  SAFE: every step is known to be within the shift series (no check).
template <bool ACC, bool SAFE, class Trig>
__device__ __forceinline__ void forward_segments(const StepC& k, const TurnsK& tk, const Trig& tg, bool fast, int K,
                                                 int C, char* ckpt, size_t sb, int64_t n, int64_t i, uint64_t T[3],
                                                 float v[3], float a[3]) {
  int seg = 0;
  for (int64_t s0 = 0; s0 < K; s0 += C, ++seg) {
    StateRef r = state_at(ckpt, sb, n, seg);
    for (int c = 0; c < 3; ++c) {
      r.T[c][i] = T[c];
      r.v[c][i] = v[c];
    }
    const int len = (K - s0 < C) ? (int)(K - s0) : C;
    for (int j = 0; j < len; ++j) {
      if constexpr (SAFE)
        rk2_step_turns<ACC, true>(k, tk, tg, T, v, a);
      else
        adj_step<ACC>(k, tk, tg, fast, T, v, a);
    }
  }
}

template <bool ACC>
__global__ void __launch_bounds__(kAdjFwdBlock, 2) k_adj_forward(EnsArgs e, FlowK f, TurnsK tk, int K, int C,
                                                                  char* ckpt, size_t sb) {
  extern __shared__ float4 s_tab3[];
  load_scaled_trig_tables(s_tab3, ff_from2(e.Af), ff_from2(e.Bf), ff_from2(e.Cf));
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= e.n) return;
  const StepC k = make_stepc(e, f);
  const TrigScaled tg{s_tab3};
  const bool fast = fast_positions(k, tk);
  uint64_t T[3] = {to_turns(e.px[i]), to_turns(e.py[i]), to_turns(e.pz[i])};
  float v[3] = {e.vx[i], e.vy[i], e.vz[i]}, a[3] = {0.f, 0.f, 0.f};
  // All K steps within the shift series (TurnsK::vsafe for K steps): no check per step.
  if (fast && fmaxf(fabsf(v[0]), fmaxf(fabsf(v[1]), fabsf(v[2]))) <= tk.vsafe)
    forward_segments<ACC, true>(k, tk, tg, fast, K, C, ckpt, sb, e.n, i, T, v, a);
  else
    forward_segments<ACC, false>(k, tk, tg, fast, K, C, ckpt, sb, e.n, i, T, v, a);
  e.px[i] = turns_to_x(T[0]);
  e.py[i] = turns_to_x(T[1]);
  e.pz[i] = turns_to_x(T[2]);
  e.vx[i] = v[0]; e.vy[i] = v[1]; e.vz[i] = v[2];
  if constexpr (ACC) {
    if (K > 0) { e.ax[i] = a[0]; e.ay[i] = a[1]; e.az[i] = a[2]; }
  }
}

// binary64 <-> float pair (once per particle, outside the step loop).
__device__ __forceinline__ ff d2ff(double d) {
  const float h = __double2float_rn(d);
  return ff{h, __double2float_rn(d - (double)h)};
}
__device__ __forceinline__ double ff2d(ff a) { return (double)a.h + (double)a.l; }

struct AdjIO {
  const double* xbK[3];
  const double* vbK[3];  // all null: zero
  double* xb0[3];
  double* vb0[3];
};

// Fixed-order block reduction of NV doubles per thread into out[0..NV) (thread 0).
template <int NV, int BLOCK>
__device__ __forceinline__ void block_reduce_fixed(double (&v)[NV], double* out) {
  __shared__ double red[NV][BLOCK];
  for (int k = 0; k < NV; ++k) red[k][threadIdx.x] = v[k];
  __syncthreads();
  for (int w = BLOCK / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int k = 0; k < NV; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < NV; ++k) out[k] = red[k][0];
}

// The recompute's step when some coordinate is beyond the shift series, and the
// reverse's sines and cosines in that case: rare, and out of line, which keeps the
// reverse kernel's code (recompute and reverse alternate within each block) small
// enough for the instruction cache.
template <class Trig>
__device__ __noinline__ void recompute_step_far(const StepC& k, const TurnsK& tk, const Trig& tg, uint64_t* T,
                                               float* v) {
  uint64_t t[3] = {T[0], T[1], T[2]};
  float w[3] = {v[0], v[1], v[2]}, a[3];
  rk2_step_turns<false, false>(k, tk, tg, t, w, a);
  for (int c = 0; c < 3; ++c) {
    T[c] = t[c];
    v[c] = w[c];
  }
}

template <class Trig>
__device__ __noinline__ void reverse_trig_far(const StepC& k, const TurnsK& tk, const Trig& tg, const uint64_t* T,
                                             const float* v, ff* P0, ff* Q0, ff* P1, ff* Q1) {
  const uint64_t t[3] = {T[0], T[1], T[2]};
  const float w[3] = {v[0], v[1], v[2]};
  ff a0[3], b0[3], a1[3], b1[3];
  step_trig_turns<false>(k, tk, tg, t, w, a0, b0, a1, b1);
  for (int c = 0; c < 3; ++c) {
    P0[c] = a0[c];
    Q0[c] = b0[c];
    P1[c] = a1[c];
    Q1[c] = b1[c];
  }
}

// Amplitudes at least this large in magnitude take the reverse on the amplitude-scaled
// tables (the parameter gradients come out multiplied by their amplitude and are divided
// once per particle); a smaller or zero amplitude takes the plain table.
constexpr double kScaledReverseMinAmp = 0x1p-20;

// SCALED: the three amplitude-scaled tables (96 KB, the forward's: the recompute reads the
// same entries); otherwise the plain table (32 KB), scaled per lookup in the recompute
// (the same bits) and read unscaled by the reverse.
template <bool SCALED>
__global__ void __launch_bounds__(kAdjBlock, 2) k_adj_reverse(EnsArgs e, FlowK f, TurnsK tk, int K, int C, int nck,
                                                             char* ckpt, char* stack, size_t sb, AdjIO io,
                                                             double* partials) {
  extern __shared__ float4 s_tab[];
  if constexpr (SCALED)
    load_scaled_trig_tables(s_tab, ff_from2(e.Af), ff_from2(e.Bf), ff_from2(e.Cf));
  else
    load_trig_table(s_tab);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double th[4] = {0.0, 0.0, 0.0, 0.0};
  if (i < e.n) {
    const StepC k = make_stepc(e, f, i);
    const TrigScaled tsc{s_tab};
    const TrigUnscaled tun = trig_unscaled(s_tab, e);  // amp = (B, C, A)
    const TrigPlain tpl{s_tab};
    const bool fast = fast_positions(k, tk);
    ff xb[3], vb[3], G[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    for (int c = 0; c < 3; ++c) {
      xb[c] = d2ff(io.xbK[c][i]);
      vb[c] = io.vbK[0] ? d2ff(io.vbK[c][i]) : ff{0.f, 0.f};
    }
    float a[3];
    for (int seg = nck - 1; seg >= 0; --seg) {
      const int s0 = seg * C, len = (K - s0 < C) ? K - s0 : C;
      StateRef ck = state_at(ckpt, sb, e.n, seg);
      uint64_t T[3];
      float v[3];
      for (int c = 0; c < 3; ++c) {
        T[c] = ck.T[c][i];
        v[c] = ck.v[c][i];
      }
      for (int j = 0; j < len; ++j) {
        StateRef st = state_at(stack, sb, e.n, j);
        for (int c = 0; c < 3; ++c) {
          st.T[c][i] = T[c];
          st.v[c][i] = v[c];
        }
        if constexpr (SCALED) {
          if (fast && near_shift(k, v))
            rk2_step_turns<false, true>(k, tk, tsc, T, v, a);
          else
            recompute_step_far(k, tk, tsc, T, v);
        } else {
          if (fast && near_shift(k, v))
            rk2_step_turns<false, true>(k, tk, tun, T, v, a);
          else
            recompute_step_far(k, tk, tun, T, v);
        }
      }
      for (int j = len - 1; j >= 0; --j) {
        StateRef st = state_at(stack, sb, e.n, j);
        for (int c = 0; c < 3; ++c) {
          T[c] = st.T[c][i];
          v[c] = st.v[c][i];
        }
        ff P0[3], Q0[3], P1[3], Q1[3];
        if constexpr (SCALED) {
          if (near_shift(k, v))
            step_trig_turns<true>(k, tk, tsc, T, v, P0, Q0, P1, Q1);
          else
            reverse_trig_far(k, tk, tsc, T, v, P0, Q0, P1, Q1);
        } else {
          if (near_shift(k, v))
            step_trig_turns<true>(k, tk, tpl, T, v, P0, Q0, P1, Q1);
          else
            reverse_trig_far(k, tk, tpl, T, v, P0, Q0, P1, Q1);
        }
        rk2_reverse_core<SCALED>(k, tun.amp, P0, Q0, P1, Q1, v, xb, vb, G);
      }
    }
    for (int c = 0; c < 3; ++c) {
      io.xb0[c][i] = ff2d(xb[c]);
      io.vb0[c][i] = ff2d(vb[c]);
    }
    // SCALED: G[0..2] = A dL/dA, B dL/dB, C dL/dC.  dL/dtau = -s^2 dL/ds = -s^2 dt G[3].
    th[0] = SCALED ? ff2d(G[0]) / e.A : ff2d(G[0]);
    th[1] = SCALED ? ff2d(G[1]) / e.B : ff2d(G[1]);
    th[2] = SCALED ? ff2d(G[2]) / e.C : ff2d(G[2]);
    th[3] = -ff2d(ff_mul(ff_mul(k.s, k.s), k.dt)) * ff2d(G[3]);
  }
  block_reduce_fixed<4, kAdjBlock>(th, partials + 4 * (size_t)blockIdx.x);
}

// One block: out[k] = scale * sum over b of partials[b*width + k], in a fixed order.
__global__ void __launch_bounds__(256) k_reduce_partials(const double* partials, int64_t nblocks, int width,
                                                         double scale, double* out) {
  __shared__ double red[256];
  for (int k = 0; k < width; ++k) {
    double s = 0.0;
    for (int64_t b = threadIdx.x; b < nblocks; b += 256) s += partials[b * width + k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = red[0] * scale;
    __syncthreads();
  }
}

struct LossIO {
  const double* x[3];
  const double* xt[3];
  double* xb[3];  // null: not wanted
};

__global__ void __launch_bounds__(kLossBlock) k_minimage_loss(LossIO io, int64_t n, double two_over_n,
                                                              double* partials) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double l[1] = {0.0};
  if (i < n) {
    const double half = 0.5 * SOAX_TWO_PI;
    for (int c = 0; c < 3; ++c) {
      double d = io.x[c][i] - io.xt[c][i];
      if (d > half)
        d -= SOAX_TWO_PI;
      else if (d < -half)
        d += SOAX_TWO_PI;
      l[0] += d * d;
      if (io.xb[0]) io.xb[c][i] = two_over_n * d;
    }
  }
  block_reduce_fixed<1, kLossBlock>(l, partials + blockIdx.x);
}

// Dynamic shared memory above 48 KB and the largest carveout for the forward, once per
// device.
static int prepare_adj_kernels() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return cuda_fail(cudaGetLastError(), "soax adjoint: device");
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return SOAX_OK;
  for (const void* fn : {(const void*)k_adj_forward<true>, (const void*)k_adj_forward<false>,
                         (const void*)k_adj_reverse<true>, (const void*)k_adj_reverse<false>}) {
    cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kScaledTrigBytes);
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (err != cudaSuccess) return cuda_fail(err, "soax adjoint: kernel attributes");
  }
  done[dev] = true;
  return SOAX_OK;
}

static int check_ptrs3(const void* const* p, bool allow_null, const char* what) {
  if (!p) return allow_null ? SOAX_OK : fail(SOAX_EINVAL, std::string(what) + " is NULL");
  for (int c = 0; c < 3; ++c) {
    if (!p[c]) return fail(SOAX_EINVAL, std::string(what) + ": NULL plane");
    if (!aligned16(p[c])) return fail(SOAX_EALIGN, std::string(what) + ": plane not 16-byte aligned");
  }
  return SOAX_OK;
}

static int adj_common(soax_t h, const soax_flow* fl, int32_t K, int32_t C, void* ws, size_t ws_bytes, EnsArgs* e,
                      FlowK* f, AdjWs* w, const char* who) {
  if (int r = check_handle(h)) return r;
  if (K < 0 || C < 1) return fail(SOAX_EINVAL, std::string(who) + ": K >= 0 and ckpt_every >= 1 required");
  if (int r = make_ens_args(h, fl, h->current, e, f, who)) return r;
  if (fl->tau_field >= 0) return fail(SOAX_EUNSUPPORTED, std::string(who) + ": per-particle tau is not differentiated");
  *w = adj_plan(h->n, K, C);
  if (h->n > 0 && (!ws || ws_bytes < w->total)) return fail(SOAX_ENOMEM, std::string(who) + ": workspace too small");
  if (!aligned16(ws)) return fail(SOAX_EALIGN, std::string(who) + ": workspace not 16-byte aligned");
  return SOAX_OK;
}

}  // namespace soax

using namespace soax;

extern "C" int soax_adjoint_workspace_bytes(soax_t h, int32_t K, int32_t ckpt_every, size_t* bytes) {
  if (int r = check_handle(h)) return r;
  if (!bytes || K < 0 || ckpt_every < 1) return fail(SOAX_EINVAL, "soax_adjoint_workspace_bytes: bad argument");
  *bytes = adj_plan(h->n, K, ckpt_every).total;
  return SOAX_OK;
}

extern "C" int soax_step_checkpointed(soax_t h, const soax_flow* fl, int32_t K, int32_t ckpt_every, void* ws,
                                      size_t ws_bytes, void* stream) {
  EnsArgs e;
  FlowK f;
  AdjWs w;
  if (int r = adj_common(h, fl, K, ckpt_every, ws, ws_bytes, &e, &f, &w, "soax_step_checkpointed")) return r;
  if (h->n == 0 || K == 0) return SOAX_OK;
  if (int r = prepare_adj_kernels()) return r;
  const auto kern = e.ax ? k_adj_forward<true> : k_adj_forward<false>;
  kern<<<grid_for(h->n, kAdjFwdBlock), kAdjFwdBlock, kScaledTrigBytes, as_stream(stream)>>>(
      e, f, make_turns_k(fl, f, K), K, ckpt_every, static_cast<char*>(ws) + w.off_ckpt,
      w.state_bytes);
  return check_launch("soax_step_checkpointed");
}

extern "C" int soax_step_adjoint(soax_t h, const soax_flow* fl, int32_t K, int32_t ckpt_every, void* ws,
                                 size_t ws_bytes, const double* const* xbarK, const double* const* vbarK,
                                 double* const* xbar0, double* const* vbar0, double* grad, void* stream) {
  EnsArgs e;
  FlowK f;
  AdjWs w;
  if (int r = adj_common(h, fl, K, ckpt_every, ws, ws_bytes, &e, &f, &w, "soax_step_adjoint")) return r;
  if (!grad) return fail(SOAX_EINVAL, "soax_step_adjoint: grad is NULL");
  cudaStream_t s = as_stream(stream);
  if (h->n == 0) {
    cudaError_t ce = cudaMemsetAsync(grad, 0, 4 * sizeof(double), s);
    return ce == cudaSuccess ? SOAX_OK : cuda_fail(ce, "soax_step_adjoint: memset");
  }
  if (int r = check_ptrs3((const void* const*)xbarK, false, "xbarK")) return r;
  if (int r = check_ptrs3((const void* const*)vbarK, true, "vbarK")) return r;
  if (int r = check_ptrs3((const void* const*)xbar0, false, "xbar0")) return r;
  if (int r = check_ptrs3((const void* const*)vbar0, false, "vbar0")) return r;
  AdjIO io;
  for (int c = 0; c < 3; ++c) {
    io.xbK[c] = xbarK[c];
    io.vbK[c] = vbarK ? vbarK[c] : nullptr;
    io.xb0[c] = xbar0[c];
    io.vb0[c] = vbar0[c];
  }
  char* base = static_cast<char*>(ws);
  double* partials = reinterpret_cast<double*>(base + w.off_partials);
  const int nb = grid_for(h->n, kAdjBlock);
  if (int r = prepare_adj_kernels()) return r;
  const bool scaled = std::fabs(fl->A) >= kScaledReverseMinAmp && std::fabs(fl->B) >= kScaledReverseMinAmp &&
                      std::fabs(fl->C) >= kScaledReverseMinAmp;
  const auto rev = scaled ? k_adj_reverse<true> : k_adj_reverse<false>;
  const size_t smem = scaled ? (size_t)kScaledTrigBytes : SOAX_TRIG_TABLE_SIZE * sizeof(float4);
  rev<<<nb, kAdjBlock, smem, s>>>(e, f, make_turns_k(fl->dt, amplitude_bound(fl)), K, ckpt_every, w.nck,
                                        base + w.off_ckpt, base + w.off_stack, w.state_bytes, io, partials);
  if (int r = check_launch("soax_step_adjoint")) return r;
  k_reduce_partials<<<1, 256, 0, s>>>(partials, nb, 4, 1.0, grad);
  return check_launch("soax_step_adjoint: reduce");
}

extern "C" int soax_minimage_loss(soax_t h, int32_t pos_field, const double* const* xtgt, double* loss,
                                  double* const* xbar, void* ws, size_t ws_bytes, void* stream) {
  if (int r = check_handle(h)) return r;
  if (int r = check_field(h, pos_field, SOAX_F64, 3, "soax_minimage_loss position")) return r;
  if (!loss) return fail(SOAX_EINVAL, "soax_minimage_loss: loss is NULL");
  if (h->n == 0) return fail(SOAX_EINVAL, "soax_minimage_loss: no particles");
  if (int r = check_ptrs3((const void* const*)xtgt, false, "xtgt")) return r;
  if (int r = check_ptrs3((const void* const*)xbar, true, "xbar")) return r;
  const int nb = grid_for(h->n, kLossBlock);
  if (!ws || ws_bytes < (size_t)nb * 8) return fail(SOAX_ENOMEM, "soax_minimage_loss: workspace too small");
  if (!aligned16(ws)) return fail(SOAX_EALIGN, "soax_minimage_loss: workspace not 16-byte aligned");
  LossIO io;
  const int fp = h->fields[pos_field].first_plane;
  for (int c = 0; c < 3; ++c) {
    io.x[c] = (const double*)h->planes[h->current][fp + c];
    if (!io.x[c]) return fail(SOAX_EUNBOUND, "soax_minimage_loss: position not bound");
    io.xt[c] = xtgt[c];
    io.xb[c] = xbar ? xbar[c] : nullptr;
  }
  double* partials = static_cast<double*>(ws);
  cudaStream_t s = as_stream(stream);
  k_minimage_loss<<<nb, kLossBlock, 0, s>>>(io, h->n, 2.0 / (double)h->n, partials);
  if (int r = check_launch("soax_minimage_loss")) return r;
  k_reduce_partials<<<1, 256, 0, s>>>(partials, nb, 1, 1.0 / (double)h->n, loss);
  return check_launch("soax_minimage_loss: reduce");
}
