/*
 * soax_oracle.c -- plain, slow, obviously-correct CPU oracle for the SoA particle
 * hot path (test infrastructure only).
 *
 * Only the tests, __graft_entry__.smoke() and the CPU-baseline leg of bench.py may load
 * this library.  The product path never calls it; it shares no code, header or constant
 * with the CUDA library.
 *
 * Everything is IEEE binary64 unless stated, compiled with -ffp-contract=off so that
 * every a*b+c below is two roundings unless written as fma().  Sine and cosine are the C
 * library's.  Threads only split the particle range; every particle's arithmetic is
 * the same sequential code whatever the thread count.
 *
 * What is computed, and where it comes from:
 *  - Eq. 1 (Sec. 2) is the paper's advection x += dt*v.  The step here generalises it
 *    to inertial particles, dx/dt = v, dv/dt = (u(x) - v)/tau, in the ABC flow
 *        u(x,y,z) = (A sin z + C cos y,  B sin x + A cos z,  C sin y + B cos x),
 *    integrated by the explicit midpoint (RK2) rule; positions live on the periodic
 *    box [0, 2pi)^3 and are wrapped once per step.  Positions are f64, velocities are
 *    stored as f32 (rounded once per step), as in the record {int id; double pos[3];
 *    float vel[3]} of the program summary.  Neither the RK2 rule, the flow nor the
 *    wrap is in the paper; they are the workload's definition and the readings are
 *    listed in the design notes.
 *  - The AoS record (Listing 1, Listing 4, Sec. 1-2) is the C struct of the schema's
 *    fields in order with natural alignment.  Transposes copy bytes (Listing 6,
 *    Sec. 4.1: getElement / push_back, done for every particle).
 *  - The cell sort is not in the paper; Sec. 1 motivates it (spatial locality of memory
 *    access).  key = (iz*G + iy)*G + ix with i = min((int)(x * (G/2pi)), G-1); the
 *    order is the stable ascending order of keys; the permutation is applied to every
 *    array, as apply<F>() does for all SoA arrays (Listing 7, Sec. 4.2.1).
 *  - The adjoint is reverse-mode differentiation of the step sequence, written out by
 *    hand, with all forward states kept in memory (no checkpointing: this is the
 *    definition the checkpointed GPU version must reproduce).
 *
 * Parity pins for each function are in tests/test_oracle_*.py.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TWO_PI 6.283185307179586 /* nearest binary64 to 2pi, 0x401921FB54442D18 */

/* ---------------------------------------------------------------- flow (ABC) */
static void abc_flow(double A, double B, double C, const double x[3], double u[3]) {
  u[0] = A * sin(x[2]) + C * cos(x[1]);
  u[1] = B * sin(x[0]) + A * cos(x[2]);
  u[2] = C * sin(x[1]) + B * cos(x[0]);
}

void orc_flow(double A, double B, double C, int64_t n, const double* x, const double* y,
              const double* z, double* ux, double* uy, double* uz) {
  for (int64_t i = 0; i < n; ++i) {
    double p[3] = {x[i], y[i], z[i]}, u[3];
    abc_flow(A, B, C, p, u);
    ux[i] = u[0]; uy[i] = u[1]; uz[i] = u[2];
  }
}

static double wrap_once(double x) {
  if (x >= ORC_TWO_PI) return x - ORC_TWO_PI;
  if (x < 0.0) return x + ORC_TWO_PI;
  return x;
}

/* One midpoint-RK2 step of one particle.  v is the f64 value of the stored velocity;
 * vnew_f64 receives v + dt*a2 before any f32 rounding; a2_out receives a2. */
static void rk2_core(double A, double B, double C, double inv_tau, double dt,
                     double x[3], const double v[3], double vnew_f64[3], double a2_out[3]) {
  double hdt = 0.5 * dt;
  double u0[3], u1[3], a1[3], xm[3], vm[3], a2[3];
  abc_flow(A, B, C, x, u0);
  for (int c = 0; c < 3; ++c) a1[c] = (u0[c] - v[c]) * inv_tau;
  for (int c = 0; c < 3; ++c) xm[c] = fma(hdt, v[c], x[c]);
  for (int c = 0; c < 3; ++c) vm[c] = v[c] + hdt * a1[c];
  abc_flow(A, B, C, xm, u1);
  for (int c = 0; c < 3; ++c) a2[c] = (u1[c] - vm[c]) * inv_tau;
  for (int c = 0; c < 3; ++c) x[c] = wrap_once(fma(dt, vm[c], x[c]));
  for (int c = 0; c < 3; ++c) vnew_f64[c] = v[c] + dt * a2[c];
  for (int c = 0; c < 3; ++c) a2_out[c] = a2[c];
}

/* ------------------------------------------------------------ threading helper */
typedef void (*range_fn)(void* ctx, int64_t lo, int64_t hi);
typedef struct { range_fn fn; void* ctx; int64_t lo, hi; } range_job;
static void* range_thread(void* p) {
  range_job* j = (range_job*)p;
  j->fn(j->ctx, j->lo, j->hi);
  return NULL;
}
static void parallel_for(int64_t n, int nthreads, range_fn fn, void* ctx) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (n < 1024 || nthreads == 1) { fn(ctx, 0, n); return; }
  pthread_t th[256];
  range_job jobs[256];
  int ok[256];
  int64_t chunk = (n + nthreads - 1) / nthreads;
  int used = 0;
  for (int t = 0; t < nthreads; ++t) {
    int64_t lo = t * chunk, hi = lo + chunk < n ? lo + chunk : n;
    if (lo >= hi) break;
    jobs[t].fn = fn; jobs[t].ctx = ctx; jobs[t].lo = lo; jobs[t].hi = hi;
    ok[t] = pthread_create(&th[t], NULL, range_thread, &jobs[t]) == 0;
    if (!ok[t]) fn(ctx, lo, hi);
    used = t + 1;
  }
  for (int t = 0; t < used; ++t)
    if (ok[t]) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------- SoA step */
typedef struct {
  double *px, *py, *pz;
  float *vx, *vy, *vz;
  float *ax, *ay, *az;      /* may be NULL */
  const float* mass;        /* may be NULL: then tau is uniform */
  double A, B, C, tau, tau_scale, dt;
  int nsteps;
} soa_ctx;

static void soa_range(void* p, int64_t lo, int64_t hi) {
  soa_ctx* c = (soa_ctx*)p;
  for (int64_t i = lo; i < hi; ++i) {
    double tau = c->mass ? c->tau_scale * (double)c->mass[i] : c->tau;
    double inv_tau = 1.0 / tau;
    double x[3] = {c->px[i], c->py[i], c->pz[i]};
    float vf[3] = {c->vx[i], c->vy[i], c->vz[i]};
    float af[3] = {0, 0, 0};
    for (int s = 0; s < c->nsteps; ++s) {
      double v[3] = {vf[0], vf[1], vf[2]}, vn[3], a2[3];
      rk2_core(c->A, c->B, c->C, inv_tau, c->dt, x, v, vn, a2);
      for (int k = 0; k < 3; ++k) { vf[k] = (float)vn[k]; af[k] = (float)a2[k]; }
    }
    c->px[i] = x[0]; c->py[i] = x[1]; c->pz[i] = x[2];
    c->vx[i] = vf[0]; c->vy[i] = vf[1]; c->vz[i] = vf[2];
    if (c->ax && c->nsteps > 0) { c->ax[i] = af[0]; c->ay[i] = af[1]; c->az[i] = af[2]; }
  }
}

/* Advance n particles nsteps steps in place (SoA planes).  ax/ay/az may be NULL; mass
 * may be NULL (then tau is used), else tau_i = tau_scale * mass_i. */
void orc_step_soa(int64_t n, double* px, double* py, double* pz, float* vx, float* vy,
                  float* vz, float* ax, float* ay, float* az, const float* mass, double A,
                  double B, double C, double tau, double tau_scale, double dt, int nsteps,
                  int nthreads) {
  soa_ctx c = {px, py, pz, vx, vy, vz, ax, ay, az, mass, A, B, C, tau, tau_scale, dt, nsteps};
  parallel_for(n, nthreads, soa_range, &c);
}

/* ------------------------------------------------------------- AoS step */
typedef struct {
  uint8_t* rec;
  int64_t rb, pos_off, vel_off, acc_off, mass_off;
  double A, B, C, tau, tau_scale, dt;
  int nsteps;
} aos_ctx;

static void aos_range(void* p, int64_t lo, int64_t hi) {
  aos_ctx* c = (aos_ctx*)p;
  for (int64_t i = lo; i < hi; ++i) {
    uint8_t* r = c->rec + i * c->rb;
    double x[3];
    float vf[3], af[3] = {0, 0, 0}, m = 0.f;
    memcpy(x, r + c->pos_off, sizeof x);
    memcpy(vf, r + c->vel_off, sizeof vf);
    if (c->mass_off >= 0) memcpy(&m, r + c->mass_off, sizeof m);
    double tau = c->mass_off >= 0 ? c->tau_scale * (double)m : c->tau;
    double inv_tau = 1.0 / tau;
    for (int s = 0; s < c->nsteps; ++s) {
      double v[3] = {vf[0], vf[1], vf[2]}, vn[3], a2[3];
      rk2_core(c->A, c->B, c->C, inv_tau, c->dt, x, v, vn, a2);
      for (int k = 0; k < 3; ++k) { vf[k] = (float)vn[k]; af[k] = (float)a2[k]; }
    }
    memcpy(r + c->pos_off, x, sizeof x);
    memcpy(r + c->vel_off, vf, sizeof vf);
    if (c->acc_off >= 0 && c->nsteps > 0) memcpy(r + c->acc_off, af, sizeof af);
  }
}

/* Same step on AoS records of rb bytes: f64 pos[3] at pos_off, f32 vel[3] at vel_off,
 * optional f32 acc[3] at acc_off and f32 mass at mass_off (-1 = absent). */
void orc_step_aos(int64_t n, uint8_t* rec, int64_t rb, int64_t pos_off, int64_t vel_off,
                  int64_t acc_off, int64_t mass_off, double A, double B, double C, double tau,
                  double tau_scale, double dt, int nsteps, int nthreads) {
  aos_ctx c = {rec, rb, pos_off, vel_off, acc_off, mass_off, A, B, C, tau, tau_scale, dt, nsteps};
  parallel_for(n, nthreads, aos_range, &c);
}

/* One step of one particle, exposing the f64 value of v + dt*a2 before its f32
 * rounding (used to audit velocities that straddle an f32 rounding midpoint). */
void orc_step_one_detail(double A, double B, double C, double tau, double dt, double* x3,
                         const float* v3, double* vnew_f64, double* a2) {
  double v[3] = {v3[0], v3[1], v3[2]};
  rk2_core(A, B, C, 1.0 / tau, dt, x3, v, vnew_f64, a2);
}

/* FP64-state forward (velocity never rounded to f32): used for finite differences
 * and the FP64 adjoint. */
typedef struct {
  double *px, *py, *pz, *vx, *vy, *vz;
  double A, B, C, tau, dt;
  int nsteps;
} f64state_ctx;

static void f64state_range(void* p, int64_t lo, int64_t hi) {
  f64state_ctx* c = (f64state_ctx*)p;
  double inv_tau = 1.0 / c->tau;
  for (int64_t i = lo; i < hi; ++i) {
    double x[3] = {c->px[i], c->py[i], c->pz[i]}, v[3] = {c->vx[i], c->vy[i], c->vz[i]};
    for (int s = 0; s < c->nsteps; ++s) {
      double vn[3], a2[3];
      rk2_core(c->A, c->B, c->C, inv_tau, c->dt, x, v, vn, a2);
      v[0] = vn[0]; v[1] = vn[1]; v[2] = vn[2];
    }
    c->px[i] = x[0]; c->py[i] = x[1]; c->pz[i] = x[2];
    c->vx[i] = v[0]; c->vy[i] = v[1]; c->vz[i] = v[2];
  }
}

void orc_step_f64state(int64_t n, double* px, double* py, double* pz, double* vx, double* vy,
                       double* vz, double A, double B, double C, double tau, double dt,
                       int nsteps, int nthreads) {
  f64state_ctx c = {px, py, pz, vx, vy, vz, A, B, C, tau, dt, nsteps};
  parallel_for(n, nthreads, f64state_range, &c);
}

/* ------------------------------------------------------------- cell keys */
void orc_cell_keys(int64_t n, const double* px, const double* py, const double* pz, int G,
                   uint32_t* keys) {
  double c = (double)G / ORC_TWO_PI;
  for (int64_t i = 0; i < n; ++i) {
    int ix = (int)(px[i] * c), iy = (int)(py[i] * c), iz = (int)(pz[i] * c);
    if (ix > G - 1) ix = G - 1;
    if (iy > G - 1) iy = G - 1;
    if (iz > G - 1) iz = G - 1;
    keys[i] = (uint32_t)(((int64_t)iz * G + iy) * G + ix);
  }
}

/* ------------------------------------------------------- stable sort, permute */
typedef struct { uint32_t key; uint32_t idx; } kv_pair;
static int kv_cmp(const void* a, const void* b) {
  const kv_pair* p = (const kv_pair*)a;
  const kv_pair* q = (const kv_pair*)b;
  if (p->key != q->key) return p->key < q->key ? -1 : 1;
  return p->idx < q->idx ? -1 : (p->idx > q->idx);
}

/* perm = the stable ascending argsort of keys: ordering by (key, original index) makes
 * the order unique.  sorted_keys may be NULL.  Returns 0, or -1 on allocation failure. */
int orc_stable_argsort(int64_t n, const uint32_t* keys, uint32_t* perm, uint32_t* sorted_keys) {
  kv_pair* t = (kv_pair*)malloc((size_t)(n > 0 ? n : 1) * sizeof(kv_pair));
  if (!t) return -1;
  for (int64_t i = 0; i < n; ++i) { t[i].key = keys[i]; t[i].idx = (uint32_t)i; }
  qsort(t, (size_t)n, sizeof(kv_pair), kv_cmp);
  for (int64_t i = 0; i < n; ++i) {
    perm[i] = t[i].idx;
    if (sorted_keys) sorted_keys[i] = t[i].key;
  }
  free(t);
  return 0;
}

/* out_f[i] = in_f[perm[i]] for each of nplanes planes of elem_bytes[f] bytes per element. */
void orc_permute(int64_t n, int nplanes, const void* const* in, void* const* out,
                 const int32_t* elem_bytes, const uint32_t* perm) {
  for (int f = 0; f < nplanes; ++f) {
    const uint8_t* src = (const uint8_t*)in[f];
    uint8_t* dst = (uint8_t*)out[f];
    int64_t e = elem_bytes[f];
    for (int64_t i = 0; i < n; ++i) memcpy(dst + i * e, src + (int64_t)perm[i] * e, (size_t)e);
  }
}

/* ------------------------------------------------------------- AoS layout */
/* Natural C layout of a struct whose members are, in order, arrays of ncomp[f]
 * scalars of elem_bytes[f] bytes: each member starts at the next multiple of its scalar
 * size; the record size is rounded up to the largest scalar size. */
int64_t orc_aos_layout(int nfields, const int32_t* elem_bytes, const int32_t* ncomp,
                       int64_t* offsets) {
  int64_t off = 0, maxal = 1;
  for (int f = 0; f < nfields; ++f) {
    int64_t al = elem_bytes[f];
    if (al > maxal) maxal = al;
    off = (off + al - 1) / al * al;
    offsets[f] = off;
    off += al * ncomp[f];
  }
  return (off + maxal - 1) / maxal * maxal;
}

/* planes: one pointer per (field, component) in schema order.  Padding bytes of every
 * record are written as zero. */
void orc_soa_to_aos(int64_t n, int nfields, const int32_t* elem_bytes, const int32_t* ncomp,
                    const void* const* planes, uint8_t* rec) {
  int64_t offs[64];
  int64_t rb = orc_aos_layout(nfields, elem_bytes, ncomp, offs);
  memset(rec, 0, (size_t)(n * rb));
  int p = 0;
  for (int f = 0; f < nfields; ++f)
    for (int c = 0; c < ncomp[f]; ++c, ++p) {
      const uint8_t* src = (const uint8_t*)planes[p];
      int64_t e = elem_bytes[f];
      for (int64_t i = 0; i < n; ++i) memcpy(rec + i * rb + offs[f] + c * e, src + i * e, (size_t)e);
    }
}

void orc_aos_to_soa(int64_t n, int nfields, const int32_t* elem_bytes, const int32_t* ncomp,
                    const uint8_t* rec, void* const* planes) {
  int64_t offs[64];
  int64_t rb = orc_aos_layout(nfields, elem_bytes, ncomp, offs);
  int p = 0;
  for (int f = 0; f < nfields; ++f)
    for (int c = 0; c < ncomp[f]; ++c, ++p) {
      uint8_t* dst = (uint8_t*)planes[p];
      int64_t e = elem_bytes[f];
      for (int64_t i = 0; i < n; ++i) memcpy(dst + i * e, rec + i * rb + offs[f] + c * e, (size_t)e);
    }
}

/* ------------------------------------------------------------- adjoint */
/* Reverse of one midpoint step (x, v) -> (x', v') given adjoints xb, vb of (x', v'),
 * which are overwritten with the adjoints of (x, v).  The f32 storage rounding of v'
 * and the periodic wrap are treated as the identity.  th[0..3] accumulate the
 * derivatives with respect to (A, B, C, tau). */
static void rk2_reverse(double A, double B, double C, double tau, double dt, const double x[3],
                        const double v[3], double xb[3], double vb[3], double th[4]) {
  double s = 1.0 / tau, hdt = 0.5 * dt;
  double u0[3], a1[3], xm[3], vm[3], u1[3];
  abc_flow(A, B, C, x, u0);
  for (int c = 0; c < 3; ++c) a1[c] = (u0[c] - v[c]) * s;
  for (int c = 0; c < 3; ++c) xm[c] = fma(hdt, v[c], x[c]);
  for (int c = 0; c < 3; ++c) vm[c] = v[c] + hdt * a1[c];
  abc_flow(A, B, C, xm, u1);

  /* x' = x + dt*vm ; v' = v + dt*a2 */
  double a2b[3], vmb[3], ub1[3], xmb[3], a1b[3], ub0[3];
  double sb = 0.0; /* adjoint of s = 1/tau */
  for (int c = 0; c < 3; ++c) a2b[c] = dt * vb[c];
  /* a2 = (u1 - vm)*s */
  for (int c = 0; c < 3; ++c) {
    ub1[c] = a2b[c] * s;
    vmb[c] = dt * xb[c] - a2b[c] * s;
    sb += a2b[c] * (u1[c] - vm[c]);
  }
  /* u1 = u(xm): xm_bar = J(xm)^T ub1 ; theta_bar += (du/dtheta)^T ub1 */
  {
    double sx = sin(xm[0]), cx = cos(xm[0]), sy = sin(xm[1]), cy = cos(xm[1]);
    double sz = sin(xm[2]), cz = cos(xm[2]);
    xmb[0] = B * cx * ub1[1] - B * sx * ub1[2];
    xmb[1] = -C * sy * ub1[0] + C * cy * ub1[2];
    xmb[2] = A * cz * ub1[0] - A * sz * ub1[1];
    th[0] += sz * ub1[0] + cz * ub1[1];
    th[1] += sx * ub1[1] + cx * ub1[2];
    th[2] += cy * ub1[0] + sy * ub1[2];
  }
  /* vm = v + hdt*a1 ; xm = x + hdt*v ; v' = v + ... ; x' = x + ... */
  for (int c = 0; c < 3; ++c) {
    a1b[c] = hdt * vmb[c];
    vb[c] = vb[c] + vmb[c] + hdt * xmb[c];
    xb[c] = xb[c] + xmb[c];
  }
  /* a1 = (u0 - v)*s */
  for (int c = 0; c < 3; ++c) {
    ub0[c] = a1b[c] * s;
    vb[c] -= a1b[c] * s;
    sb += a1b[c] * (u0[c] - v[c]);
  }
  {
    double sx = sin(x[0]), cx = cos(x[0]), sy = sin(x[1]), cy = cos(x[1]);
    double sz = sin(x[2]), cz = cos(x[2]);
    xb[0] += B * cx * ub0[1] - B * sx * ub0[2];
    xb[1] += -C * sy * ub0[0] + C * cy * ub0[2];
    xb[2] += A * cz * ub0[0] - A * sz * ub0[1];
    th[0] += sz * ub0[0] + cz * ub0[1];
    th[1] += sx * ub0[1] + cx * ub0[2];
    th[2] += cy * ub0[0] + sy * ub0[2];
  }
  /* s = 1/tau: d s / d tau = -1/tau^2 = -s*s */
  th[3] += -sb * s * s;
}

typedef struct {
  int64_t n;
  const double *x0[3], *xt[3];
  const float* v0f[3];
  const double* v0d[3];
  double A, B, C, tau, dt;
  int K, f32v;
  double *xb0[3], *vb0[3], *contrib;
} adj_ctx;

static double min_image(double d) {
  /* ((d + pi) mod 2pi) - pi with the mathematical (non-negative) modulus */
  double t = fmod(d + 0.5 * ORC_TWO_PI, ORC_TWO_PI);
  if (t < 0) t += ORC_TWO_PI;
  return t - 0.5 * ORC_TWO_PI;
}

static void adj_range(void* p, int64_t lo, int64_t hi) {
  adj_ctx* c = (adj_ctx*)p;
  int K = c->K;
  double* xs = (double*)malloc(sizeof(double) * 6 * (size_t)(K + 1));
  if (!xs) return;
  for (int64_t i = lo; i < hi; ++i) {
    double x[3], v[3];
    for (int k = 0; k < 3; ++k) {
      x[k] = c->x0[k][i];
      v[k] = c->f32v ? (double)c->v0f[k][i] : c->v0d[k][i];
    }
    double inv_tau = 1.0 / c->tau;
    for (int s = 0; s < K; ++s) {
      for (int k = 0; k < 3; ++k) { xs[6 * s + k] = x[k]; xs[6 * s + 3 + k] = v[k]; }
      double vn[3], a2[3];
      rk2_core(c->A, c->B, c->C, inv_tau, c->dt, x, v, vn, a2);
      for (int k = 0; k < 3; ++k) v[k] = c->f32v ? (double)(float)vn[k] : vn[k];
    }
    double xb[3], vb[3] = {0, 0, 0}, th[4] = {0, 0, 0, 0}, l = 0.0;
    for (int k = 0; k < 3; ++k) {
      double d = min_image(x[k] - c->xt[k][i]);
      l += d * d;
      xb[k] = 2.0 * d / (double)c->n;
    }
    for (int s = K - 1; s >= 0; --s)
      rk2_reverse(c->A, c->B, c->C, c->tau, c->dt, &xs[6 * s], &xs[6 * s + 3], xb, vb, th);
    for (int k = 0; k < 3; ++k) { c->xb0[k][i] = xb[k]; c->vb0[k][i] = vb[k]; }
    for (int k = 0; k < 4; ++k) c->contrib[5 * i + k] = th[k];
    c->contrib[5 * i + 4] = l;
  }
  free(xs);
}

/* Loss L = (1/n) sum_p |d_p|^2, d the minimum image of x_K - x_target, and its gradient
 * with respect to x0, v0 and (A, B, C, tau) after K steps.  f32v != 0: the velocity is
 * stored as f32 after each step (v0 read from v0f); f32v == 0: FP64 state (v0 read
 * from v0d).  grad[0..3] = dL/d(A,B,C,tau), summed over particles in index order.
 * Returns 0, or -1 on allocation failure. */
int orc_adjoint(int64_t n, const double* x0, const double* y0, const double* z0,
                const float* v0x_f, const float* v0y_f, const float* v0z_f, const double* v0x_d,
                const double* v0y_d, const double* v0z_d, const double* xtx, const double* xty,
                const double* xtz, double A, double B, double C, double tau, double dt, int K,
                int f32v, double* xb0x, double* xb0y, double* xb0z, double* vb0x, double* vb0y,
                double* vb0z, double* grad, double* loss, int nthreads) {
  double* contrib = (double*)calloc((size_t)(n > 0 ? n : 1) * 5, sizeof(double));
  if (!contrib) return -1;
  adj_ctx c;
  memset(&c, 0, sizeof c);
  c.n = n;
  c.x0[0] = x0; c.x0[1] = y0; c.x0[2] = z0;
  c.xt[0] = xtx; c.xt[1] = xty; c.xt[2] = xtz;
  c.v0f[0] = v0x_f; c.v0f[1] = v0y_f; c.v0f[2] = v0z_f;
  c.v0d[0] = v0x_d; c.v0d[1] = v0y_d; c.v0d[2] = v0z_d;
  c.A = A; c.B = B; c.C = C; c.tau = tau; c.dt = dt; c.K = K; c.f32v = f32v;
  c.xb0[0] = xb0x; c.xb0[1] = xb0y; c.xb0[2] = xb0z;
  c.vb0[0] = vb0x; c.vb0[1] = vb0y; c.vb0[2] = vb0z;
  c.contrib = contrib;
  parallel_for(n, nthreads, adj_range, &c);
  double g[4] = {0, 0, 0, 0}, l = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    for (int k = 0; k < 4; ++k) g[k] += contrib[5 * i + k];
    l += contrib[5 * i + 4];
  }
  for (int k = 0; k < 4; ++k) grad[k] = g[k];
  *loss = l / (double)n;
  free(contrib);
  return 0;
}

/* ------------------------------------------------------------- Euler (Eq. 1) */
/* The paper's own benchmark step, x += dt*v per component in single precision. */
void orc_euler_f32(int64_t n, float* x, const float* v, float dt) {
  for (int64_t i = 0; i < n; ++i) x[i] = x[i] + dt * v[i];
}

/* The same step on AoS records of rb bytes with f32 x[3] at x_off and f32 v[3] at
 * v_off (the Particle<SIZE> record of Listing 4: x, v, then SIZE padding floats). */
void orc_euler_aos_f32(int64_t n, uint8_t* rec, int64_t rb, int64_t x_off, int64_t v_off, float dt) {
  for (int64_t i = 0; i < n; ++i) {
    float x[3], v[3];
    memcpy(x, rec + i * rb + x_off, sizeof x);
    memcpy(v, rec + i * rb + v_off, sizeof v);
    for (int c = 0; c < 3; ++c) x[c] = x[c] + dt * v[c];
    memcpy(rec + i * rb + x_off, x, sizeof x);
  }
}

/* ------------------------------------------------ whole-array operations (Sec. 4) */
/* SetToValue applied to one array (Listing 7): every element of a plane of elem_bytes
 * bytes and type code tcode (0 i32, 1 i64, 2 u8, 3 f32, 4 f64) set to value. */
void orc_fill(int64_t n, void* plane, int tcode, double value) {
  for (int64_t i = 0; i < n; ++i) {
    switch (tcode) {
      case 0: ((int32_t*)plane)[i] = (int32_t)value; break;
      case 1: ((int64_t*)plane)[i] = (int64_t)value; break;
      case 2: ((uint8_t*)plane)[i] = (uint8_t)value; break;
      case 3: ((float*)plane)[i] = (float)value; break;
      default: ((double*)plane)[i] = value; break;
    }
  }
}

/* dst = constant + sum_k coef_k src_k, element by element, accumulated left to right with
 * one fused multiply-add per term (acc = fma(coef_k, src_k, acc)), in the planes' type
 * (all f32 when is_f32, else all f64; coefficients and constant rounded to it).  The
 * expression of Listing 5, posArr(0) = velArr(1) - velArr(2), is constant 0 and
 * coefficients (1, -1). */
void orc_lincomb(int64_t n, int is_f32, void* dst, int nterms, const void* const* src, const double* coef,
                 double constant) {
  for (int64_t i = 0; i < n; ++i) {
    if (is_f32) {
      float acc = (float)constant;
      for (int k = 0; k < nterms; ++k) acc = fmaf((float)coef[k], ((const float*)src[k])[i], acc);
      ((float*)dst)[i] = acc;
    } else {
      double acc = constant;
      for (int k = 0; k < nterms; ++k) acc = fma(coef[k], ((const double*)src[k])[i], acc);
      ((double*)dst)[i] = acc;
    }
  }
}

/* Removal by overwriting with the last particles (Sec. 2: a particle is removed by
 * overwriting it with the last one, the default of SoAx when the order does not
 * matter).  For k distinct ascending indices and m = n - k: the removed positions below
 * m ("holes", ascending) receive the particles at the positions m..n-1 that are not
 * removed (ascending), one each, in every plane; nothing else moves.  For k = 1 this is
 * exactly "overwrite with the last".  Returns m. */
int64_t orc_remove(int64_t n, int nplanes, void* const* planes, const int32_t* elem_bytes, const uint32_t* idx,
                   int64_t k) {
  int64_t m = n - k;
  uint8_t* removed = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  if (!removed) return -1;
  for (int64_t j = 0; j < k; ++j) removed[idx[j]] = 1;
  int64_t src = m;
  for (int64_t j = 0; j < k && idx[j] < (uint32_t)m; ++j) {
    while (removed[src]) ++src;  /* next surviving tail particle */
    for (int f = 0; f < nplanes; ++f) {
      uint8_t* p = (uint8_t*)planes[f];
      int64_t e = elem_bytes[f];
      memcpy(p + (int64_t)idx[j] * e, p + src * e, (size_t)e);
    }
    ++src;
  }
  free(removed);
  return m;
}

/* ------------------------------------------------- general expressions (Sec. 4.2) */
/* An expression over whole arrays (the expression templates of Sec. 4.2, e.g. Listing
 * 5's posArr(0) = velArr(1) - velArr(2)), written as a postfix program evaluated element
 * by element on a stack of values of the compute type (binary32 when is_f32, else
 * binary64).  Operation codes (op[j]):
 *   0 LOAD  push source j converted to the compute type (as a C cast: exact for every
 *           source type in binary64 except i64 beyond 2^53; rounded to nearest in
 *           binary32 for i32, i64 and f64 sources)
 *   1 CONST push value[j] rounded to the compute type
 *   2 ADD, 3 SUB, 4 MUL, 5 DIV: pop b, pop a, push a op b, correctly rounded
 *   6 NEG, 7 ABS, 8 SQRT (correctly rounded): pop a, push f(a)
 *   9 MIN, 10 MAX: pop b, pop a, push (a < b ? a : b), (a > b ? a : b)
 *  11 FMA: pop c, pop b, pop a, push a*b+c with one rounding
 * The result (the one value left) is stored into dst, rounded to the destination type
 * (dst_is_f32) when that is narrower.  src_tcode[j] is the type code of source j (0 i32,
 * 1 i64, 2 u8, 3 f32, 4 f64); src[j] is unused unless op[j] is LOAD.  The program is
 * assumed valid (the library checks its own before any launch). */
static double expr_load_d(const void* p, int t, int64_t i) {
  switch (t) {
    case 0: return (double)((const int32_t*)p)[i];
    case 1: return (double)((const int64_t*)p)[i];
    case 2: return (double)((const uint8_t*)p)[i];
    case 3: return (double)((const float*)p)[i];
    default: return ((const double*)p)[i];
  }
}

static float expr_load_f(const void* p, int t, int64_t i) {
  switch (t) {
    case 0: return (float)((const int32_t*)p)[i];
    case 1: return (float)((const int64_t*)p)[i];
    case 2: return (float)((const uint8_t*)p)[i];
    case 3: return ((const float*)p)[i];
    default: return (float)((const double*)p)[i];
  }
}

void orc_expr(int64_t n, int is_f32, int nops, const int32_t* op, const double* value, const void* const* src,
              const int32_t* src_tcode, void* dst, int dst_is_f32) {
  for (int64_t i = 0; i < n; ++i) {
    if (is_f32) {
      float st[64];
      int sp = 0;
      for (int j = 0; j < nops; ++j) {
        float a, b, c;
        switch (op[j]) {
          case 0: st[sp++] = expr_load_f(src[j], src_tcode[j], i); break;
          case 1: st[sp++] = (float)value[j]; break;
          case 2: b = st[--sp]; a = st[--sp]; st[sp++] = a + b; break;
          case 3: b = st[--sp]; a = st[--sp]; st[sp++] = a - b; break;
          case 4: b = st[--sp]; a = st[--sp]; st[sp++] = a * b; break;
          case 5: b = st[--sp]; a = st[--sp]; st[sp++] = a / b; break;
          case 6: a = st[--sp]; st[sp++] = -a; break;
          case 7: a = st[--sp]; st[sp++] = fabsf(a); break;
          case 8: a = st[--sp]; st[sp++] = sqrtf(a); break;
          case 9: b = st[--sp]; a = st[--sp]; st[sp++] = a < b ? a : b; break;
          case 10: b = st[--sp]; a = st[--sp]; st[sp++] = a > b ? a : b; break;
          default: c = st[--sp]; b = st[--sp]; a = st[--sp]; st[sp++] = fmaf(a, b, c); break;
        }
      }
      if (dst_is_f32) ((float*)dst)[i] = st[0];
      else ((double*)dst)[i] = (double)st[0];
    } else {
      double st[64];
      int sp = 0;
      for (int j = 0; j < nops; ++j) {
        double a, b, c;
        switch (op[j]) {
          case 0: st[sp++] = expr_load_d(src[j], src_tcode[j], i); break;
          case 1: st[sp++] = value[j]; break;
          case 2: b = st[--sp]; a = st[--sp]; st[sp++] = a + b; break;
          case 3: b = st[--sp]; a = st[--sp]; st[sp++] = a - b; break;
          case 4: b = st[--sp]; a = st[--sp]; st[sp++] = a * b; break;
          case 5: b = st[--sp]; a = st[--sp]; st[sp++] = a / b; break;
          case 6: a = st[--sp]; st[sp++] = -a; break;
          case 7: a = st[--sp]; st[sp++] = fabs(a); break;
          case 8: a = st[--sp]; st[sp++] = sqrt(a); break;
          case 9: b = st[--sp]; a = st[--sp]; st[sp++] = a < b ? a : b; break;
          case 10: b = st[--sp]; a = st[--sp]; st[sp++] = a > b ? a : b; break;
          default: c = st[--sp]; b = st[--sp]; a = st[--sp]; st[sp++] = fma(a, b, c); break;
        }
      }
      if (dst_is_f32) ((float*)dst)[i] = (float)st[0];
      else ((double*)dst)[i] = st[0];
    }
  }
}
