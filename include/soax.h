/*
 * soax.h -- C ABI of libsoax, a B300 (sm_103a) library for heterogeneous particle
 * records stored as a Structure of Arrays (SoA).
 *
 * The container follows the paper's SoAx (Sec. 4): a particle type is a list of
 * attributes, each an N-dimensional array of one scalar type with a one-character tag
 * (SOAX_ATTRIBUTE(name, 'C') and the attribute tuple of Listing 5); the SoA holds one
 * device array ("plane") per attribute component (posArr(d) in Listing 5).  Here the
 * schema is a runtime value instead of a C++ type.
 *
 * Conventions for every call:
 *  - Return value: SOAX_OK (0) or a negative soax_status.  No exception or abort crosses
 *    this boundary.  soax_last_error() gives a message for the calling thread.
 *  - Host-side validation (null pointers, schema, alignment, sizes) happens before any
 *    launch; a failed validation launches nothing and changes nothing.
 *  - Ownership: the library owns only the host-side handle.  Particle planes, shadow
 *    planes, AoS buffers, keys, permutations and workspaces are device memory owned by
 *    the caller (e.g. PyTorch tensors), and must stay valid while work that uses them is
 *    in flight.  No call allocates device memory for data; the cell sort keeps a CUDA
 *    graph per set of buffers, which the driver instantiates on the first such call
 *    (see soax_sort_by_cell).
 *  - Streams: every compute call is asynchronous on the given cudaStream_t (passed as
 *    void*; NULL = the legacy default stream) on the calling thread's current device.
 *    Calls do not synchronise with the host, except soax_sync(), soax_autotune() and
 *    the first soax_step_batched() call for a new plan (documented there).
 *  - Device-side errors set a per-device status word that soax_sync() reports and
 *    clears.
 *  - Plane layout: plane (f, c) of field f holds component c of every particle,
 *    contiguous, element i at byte offset i*elem_size.  Every plane and AoS buffer must
 *    be 16-byte aligned (SOAX_EALIGN otherwise).
 */
#ifndef SOAX_H
#define SOAX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SOAX_OK = 0,
  SOAX_EINVAL = -1,       /* bad argument (null pointer, negative size, bad index)  */
  SOAX_ESCHEMA = -2,      /* schema is malformed or lacks a field the call needs      */
  SOAX_EALIGN = -3,       /* a device pointer is not 16-byte aligned                  */
  SOAX_ECUDA = -4,        /* a CUDA runtime call or kernel launch failed              */
  SOAX_ETIMEOUT = -5,     /* a bounded device-side wait gave up (see soax_sync)       */
  SOAX_ENOMEM = -6,       /* the caller's workspace is smaller than required          */
  SOAX_EUNSUPPORTED = -7, /* valid request this build does not implement              */
  SOAX_EUNBOUND = -8      /* a plane the call needs has not been bound                */
} soax_status;

/* Scalar types of an attribute (Sec. 4.1: id<int,1>, pos<double,3>, mass<float,1>). */
typedef enum { SOAX_I32 = 0, SOAX_I64 = 1, SOAX_U8 = 2, SOAX_F32 = 3, SOAX_F64 = 4 } soax_dtype;

/* One attribute: SOAX_ATTRIBUTE(name, tag) with type<dtype, ncomp> (Listing 5).
 * name: NUL-terminated, 1..31 chars, unique in the schema (copied at create).
 * ncomp: 1..16.  tag: free descriptive character; soax_sort_by_cell uses the field
 * tagged 'P' (f64 x 3) as the position. */
typedef struct {
  const char* name;
  int32_t dtype;
  int32_t ncomp;
  char tag;
} soax_field_desc;

typedef struct soax_s* soax_t;

/* Parameters of the inertial-particle step in the ABC flow
 *   u(x,y,z) = (A sin z + C cos y, B sin x + A cos z, C sin y + B cos x),
 *   dx/dt = v, dv/dt = (u(x) - v)/tau,
 * integrated by the explicit midpoint rule with time step dt on the periodic box
 * [0, 2pi)^3.  This generalises the paper's Euler advection x += dt*v (Eq. 1, Sec. 2). */
typedef struct {
  double A, B, C;    /* flow amplitudes (finite)                                   */
  double tau;        /* uniform response time, used when tau_field < 0 (> 0)       */
  double dt;         /* time step (> 0)                                            */
  double tau_scale;  /* tau_i = tau_scale * (double)field[tau_field][i]            */
  int32_t tau_field; /* index of an f32 x 1 field (e.g. mass), or -1                */
  int32_t pos_field; /* index of the f64 x 3 position field                        */
  int32_t vel_field; /* index of the f32 x 3 velocity field                        */
  int32_t acc_field; /* index of an f32 x 3 field that receives the last stage
                        acceleration of the last step, or -1                        */
} soax_flow;

/* Launch shape of the batched step.  parts_per_thread: 1, 2 or 4 particles per thread;
 * block: 64..512, a multiple of 32; vec_bits: 64 or 128 (width of each plane load; the
 * fused form loads each plane once and ignores it); fuse_steps: 0 = one launch and one
 * pass over memory per step (soax_step's arithmetic), 1 = all nsteps of the call in
 * registers in one launch (soax_step_fused's arithmetic). */
typedef struct {
  int32_t parts_per_thread;
  int32_t block;
  int32_t vec_bits;
  int32_t fuse_steps;
} soax_tune;

/* ------------------------------------------------------------------ handles */

/* Library ABI version (currently 1). */
int soax_version(void);

/* Message for the last failed call on this thread ("" if none).  The pointer stays
 * valid until the next call on this thread. */
const char* soax_last_error(void);

/* Build a handle for n particles (0 <= n < 2^31) with the given schema
 * (Listing 5: Soax<ArrayTypes> soax(42)).  Host only; allocates no device memory.
 * SOAX_ESCHEMA on a malformed schema (bad dtype, ncomp out of range, duplicate or empty
 * name, more than 32 fields or 64 planes). */
int soax_create(const soax_field_desc* fields, int32_t nfields, int64_t n, soax_t* out);

/* Release a handle (host memory only; bound planes are not freed).  NULL is accepted. */
int soax_destroy(soax_t h);

/* Number of particles, fields, and planes of a handle (any output may be NULL). */
int soax_size(soax_t h, int64_t* n, int32_t* nfields, int32_t* nplanes);

/* resize (Listing 5) within the capacity given to soax_create: the particle count
 * becomes n (0 <= n <= capacity, SOAX_EINVAL otherwise); elements n.. of the planes are
 * left as they are (new elements hold whatever the buffers held). */
int soax_set_size(soax_t h, int64_t n);

/* Attach caller-owned device memory to plane (field, comp) of buffer set buf
 * (0 = primary, 1 = shadow used as the destination of soax_sort_by_cell).  dev_ptr
 * must hold capacity (the n given to soax_create) elements of the field's type and be
 * 16-byte aligned (SOAX_EALIGN). */
int soax_bind(soax_t h, int32_t field, int32_t comp, int32_t buf, void* dev_ptr);

/* Which buffer set (0 or 1) currently holds the particles.  soax_sort_by_cell and
 * soax_permute flip it; soax_set_current sets it. */
int soax_current(soax_t h, int32_t* buf);

/* Copy plane (field, comp) of the live buffer set (its first n elements, n x the
 * element size bytes) from host memory to the device (to_device = 1) or back
 * (to_device = 0), as one cudaMemcpyAsync on stream.  host must stay valid until the
 * copy has run; it is asynchronous for page-locked (pinned) host memory, otherwise the
 * call returns when the copy is done.  SOAX_EINVAL for a bad field, component or
 * direction, a NULL host pointer (n > 0) or an unbound plane; SOAX_ECUDA if the copy
 * cannot be enqueued. */
int soax_copy_plane(soax_t h, int32_t field, int32_t comp, void* host, int32_t to_device, void* stream);
int soax_set_current(soax_t h, int32_t buf);

/* Natural C layout of the AoS record of this schema (the structs of Listing 1 and 4):
 * fields in schema order, each at the next multiple of its scalar size, the size rounded
 * up to the largest scalar size.  field_offsets receives nfields values (may be NULL). */
int soax_aos_layout(soax_t h, int64_t* record_bytes, int64_t* field_offsets);

/* ------------------------------------------------------------- transposes */

/* Bulk getElement (Listing 6, Sec. 4.1): copy n AoS records (layout from
 * soax_aos_layout, 16-byte aligned device buffer) into the live planes, byte for byte;
 * padding bytes are ignored.  Records of up to 400 bytes (SOAX_EUNSUPPORTED beyond). */
int soax_aos_to_soa(soax_t h, const void* aos_dev, void* stream);

/* Bulk push_back (Listing 6): copy the live planes into n AoS records, byte for byte,
 * padding bytes written as 0. */
int soax_soa_to_aos(soax_t h, void* aos_dev, void* stream);

/* getElement / push_back for one particle (Listing 6): copy particle i (0 <= i < n) of
 * the live planes into one AoS record at rec_dev (16-byte aligned device memory of
 * soax_aos_layout's record size; padding written as 0), or the record into particle i.
 * push_back = soax_set_size(h, n + 1) then soax_set_element(h, n, rec). */
int soax_get_element(soax_t h, int64_t i, void* rec_dev, void* stream);
int soax_set_element(soax_t h, int64_t i, const void* rec_dev, void* stream);

/* Workspace bytes soax_remove needs for k removals. */
int soax_remove_workspace_bytes(int64_t k, size_t* bytes);

/* Remove the k particles at the distinct ascending indices idx (device u32, all < n) by
 * overwriting them with the last particles (Sec. 2: a particle is removed by overwriting
 * it with the last one when the order does not matter): the removed positions below
 * n - k, ascending, receive the particles of positions n - k .. n - 1 that are not
 * removed, ascending; nothing else moves.  The size becomes n - k at once for later
 * calls.  If idx is not ascending, distinct and in
 * range, nothing is moved and the kernel records SOAX_EINVAL for soax_sync (the size
 * still drops by k). */
int soax_remove(soax_t h, const uint32_t* idx, int64_t k, void* ws, size_t ws_bytes, void* stream);

/* -------------------------------------------------------------------- step */

/* Advance every particle nsteps (>= 0) midpoint-RK2 steps in place on the live planes:
 *   a1 = (u(x) - v)/tau,  xm = x + dt/2 v,  vm = v + dt/2 a1,  a2 = (u(xm) - vm)/tau,
 *   x' = x + dt vm (wrapped once into [0, 2pi)),  v' = v + dt a2 rounded to f32,
 * with f64-accurate arithmetic (v is promoted from f32).  One pass over the planes per
 * step; each step is one kernel launch (capturable in a CUDA graph).
 * Defining passages: Eq. 1 (Sec. 2), the per-particle update of position from velocity
 * that this step generalises to an inertial particle with a second-order integrator;
 * Listing 4's commentary (Sec. 2) names temporary Runge-Kutta positions and velocities
 * as typical particle data.  The paper gives no RK2 scheme: the midpoint rule, the ABC
 * flow and tau are this library's workload definition, stated above. */
int soax_step(soax_t h, const soax_flow* fl, int32_t nsteps, void* stream);

/* The same nsteps (>= 0) midpoint-RK2 steps as soax_step in ONE pass over the planes:
 * each particle is loaded once, advanced nsteps steps in registers and stored once, so
 * the planes move once per call instead of once per step (one kernel launch).  The
 * velocity arithmetic is soax_step's, including the f32 rounding of v after every step.
 * Between steps the position is held as a 64-bit fixed-point fraction of a turn,
 * frac(x / 2pi) 2^64 (resolution 2^-64 turn = 3.4e-19 rad, finer than binary64 at
 * x >= 2^-8), instead of being rounded to binary64 every step; it is rounded to binary64
 * once at the end, wrapped into [0, 2pi).  Results therefore agree with soax_step to
 * within a few binary64 ulps per step, not bit for bit.  Positions on entry must lie in
 * [0, 8) (soax_step's output always does).  Tau and acceleration fields as for
 * soax_step; acc receives the last step's a2.
 * Defining passages: Eq. 1 (Sec. 2) as for soax_step; the single pass over all arrays is
 * the loop fusion of the expression templates (Sec. 4.2, 4.2.2), applied across time
 * steps. */
int soax_step_fused(soax_t h, const soax_flow* fl, int32_t nsteps, void* stream);

/* soax_step_fused that also writes the cell keys of the final positions (the flow's
 * position field) on a grid^3 grid into keys (n u32, 16-byte aligned, caller-owned),
 * bit-identical to soax_cell_keys on the result, as the particles are stored: the sort
 * that follows (soax_sort_by_keys) needs no key pass over the positions.  grid in
 * 1..1024.  nsteps = 0 writes the keys of the current positions.
 * Defining passages: Eq. 1 (Sec. 2) for the steps; the keys serve spatial locality of
 * memory access (Sec. 1; the cache analysis of Sec. 2). */
int soax_step_fused_keys(soax_t h, const soax_flow* fl, int32_t nsteps, int32_t grid, uint32_t* keys,
                         void* stream);

/* soax_permute(h, perm) followed by soax_step_fused_keys(h, fl, nsteps, grid, keys) in
 * ONE pass: particle i of the other buffer set becomes particle perm[i] of the live set,
 * its position and velocity advanced nsteps steps on the way and its other fields copied;
 * then the live set flips.  Same bits as the two calls.  perm: n u32 (a permutation of
 * 0..n-1, 16-byte aligned; an entry >= n is not read, particle 0 is used instead and
 * SOAX_EINVAL is recorded for soax_sync), e.g. the permutation soax_sort_perm left in a
 * sort workspace, so that a cell sort's gather costs no pass of its own.  grid = 0: no
 * keys (keys ignored); else keys as for soax_step_fused_keys.  Both buffer sets must be
 * bound.
 * Defining passages: apply-to-all-arrays (Listing 7, Sec. 4.2.1) for the gather of every
 * field; Eq. 1 (Sec. 2) for the steps; spatial locality (Sec. 1) for the cell order. */
int soax_permute_step_fused(soax_t h, const uint32_t* perm, const soax_flow* fl, int32_t nsteps, int32_t grid,
                            uint32_t* keys, void* stream);

/* The same step, bit-identical per particle, on AoS records in place (layout from
 * soax_aos_layout; the flow's field indices refer to this handle's schema).
 * Defining passages: the AoS records of Listings 1 and 4 and the AoS-versus-SoA
 * comparison of Sec. 2 and Sec. 3.2, with soax_step's arithmetic. */
int soax_step_aos(soax_t h, void* aos_dev, const soax_flow* fl, int32_t nsteps, void* stream);

/* ------------------------------------------------------------- cell sort */

/* keys[i] = (iz*G + iy)*G + ix of the live position field pos_field, with
 * i_d = min((int)(x_d * (G/2pi)), G-1) computed in binary64 (G/2pi rounded once).
 * grid G in 1..1024; keys: n u32, 16-byte aligned.
 * Defining passages: spatial locality of memory access (Sec. 1) and the cache analysis
 * of Sec. 2; the paper defines no cell grid, which is this library's definition above. */
int soax_cell_keys(soax_t h, int32_t pos_field, int32_t grid, uint32_t* keys, void* stream);

/* Workspace bytes soax_radix_sort_pairs needs for n keys of key_bits significant bits. */
int soax_radix_workspace_bytes(int64_t n, int32_t key_bits, size_t* bytes);

/* Stable ascending LSD radix sort of (key, value) pairs by the low key_bits (1..32) bits
 * of key.  vals_in may be NULL (then value i = i, i.e. vals_out is the stable argsort).
 * keys_out may be NULL (sorted keys not wanted).  Inputs are not modified; outputs must
 * not alias inputs.  All arrays hold n u32 and are 16-byte aligned; ws holds
 * soax_radix_workspace_bytes bytes.
 * Defining passages: none in the paper (it has no sort); the ordering step behind the
 * spatial locality of Sec. 1.  A scatter destination outside the output (only possible
 * if the workspace is overwritten while the sort runs) is clamped to the last element
 * and SOAX_EINVAL is recorded for soax_sync. */
int soax_radix_sort_pairs(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                          uint32_t* vals_out, int64_t n, int32_t key_bits, void* ws,
                          size_t ws_bytes, void* stream);

/* out_f[i] = in_f[perm[i]] for every plane of every field, from the live buffer set to
 * the other one (apply-to-all-arrays, Listing 7), then flip the live set.  perm should be
 * a permutation of 0..n-1; an entry >= n is not read (element 0 is gathered instead) and
 * the kernel records SOAX_EINVAL in the device status word, which the next soax_sync
 * returns. */
int soax_permute(soax_t h, const uint32_t* perm, void* stream);

/* Workspace bytes soax_sort_by_cell needs. */
int soax_sort_workspace_bytes(soax_t h, int32_t grid, size_t* bytes);

/* Cell keys of the field tagged 'P' on a grid^3 grid, stable sort, permute-gather of all
 * fields into the shadow set, flip.  The sorted keys and the permutation are left in the
 * workspace (soax_sort_results gives their addresses).
 * The sort (here and in soax_sort_by_keys, soax_sort_perm): for grids up to 64^3 a
 * counting sort that exploits keys in near-cell order, launched as one CUDA graph whose
 * conditional node runs the LSD radix passes only for keys the counting sort cannot take
 * (more than 2048 particles or 256 runs in one cell, keys in no particular order).  The
 * graph is built on the first call for a set of (keys, sorted keys, permutation,
 * workspace, n, grid) and kept (the eight most recent sets per process); on a stream
 * that is being captured into a graph, the same kernels are launched into the capture
 * with the radix passes gated behind them.  Larger grids: the radix passes alone.  Every
 * form gives the same stable permutation.
 * Defining passages: spatial locality (Sec. 1, Sec. 2's cache analysis) for the order;
 * apply-to-all-arrays (Listing 7, Sec. 4.2.1) for the gather of every field. */
int soax_sort_by_cell(soax_t h, int32_t grid, void* ws, size_t ws_bytes, void* stream);
int soax_sort_results(soax_t h, int32_t grid, void* ws, size_t ws_bytes, uint32_t** sorted_keys,
                      uint32_t** perm);

/* soax_sort_by_cell with its key pass done already: stable radix sort of the given keys
 * (n u32, each < grid^3, as soax_cell_keys or soax_step_fused_keys write them; only their
 * low bits up to grid^3 - 1 are sorted), permute-gather of all fields into the shadow
 * set, flip.  ws as for soax_sort_by_cell (soax_sort_results gives the sorted keys and
 * the permutation in it); keys must not overlap ws's sorted-key, permutation or radix
 * regions.  Defining passages: as for soax_sort_by_cell. */
int soax_sort_by_keys(soax_t h, int32_t grid, const uint32_t* keys, void* ws, size_t ws_bytes, void* stream);

/* soax_sort_by_keys without the permute-gather: the stable permutation that sorts keys
 * is left in ws (soax_sort_results gives its address; the sorted keys are not written);
 * no particle moves.  Pair it with soax_permute_step_fused, or soax_permute.
 * Defining passages: as for soax_sort_by_cell (the order only). */
int soax_sort_perm(soax_t h, int32_t grid, const uint32_t* keys, void* ws, size_t ws_bytes, void* stream);

/* How many cell-sort graphs this process has built (*built) and how many builds failed
 * (*failed: those sets of buffers launch the same kernels on the stream instead, with
 * the radix passes gated).  A diagnostic for callers and tests; see soax_sort_by_cell.
 * Defining passages: as for soax_sort_by_cell. */
int soax_sort_graph_counts(int64_t* built, int64_t* failed);

/* soax_sort_by_cell without a caller workspace.  The paper has no counterpart: this is
 * for hosts that cannot allocate device memory where they sort -- C or Fortran codes
 * linking the library with no device allocator of their own, or time-step loops that
 * forbid cudaMalloc because it can synchronise the device and breaks a memory budget
 * fixed at start-up.  Same keys, radix sort and permute-gather as soax_sort_by_cell,
 * with the scratch in a static device array of 32 MiB that every GPU loading the
 * library holds until exit; this call allocates nothing.  Limits: n <= 1048576 and
 * grid in 1..64 (SOAX_EINVAL otherwise, before any device work).  perm_out: n u32 on
 * the device receiving the permutation, or NULL.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current, and a call
 * looks it up again if the device's context has changed since (after cudaDeviceReset the
 * array may sit elsewhere); make the first call, and the first after a reset, before any
 * stream capture.  All calls share the one array and it keeps the
 * last call's contents (every part is rewritten before use): calls that overlap on the
 * GPU, on any stream or thread, race and corrupt each other. */
int soax_sort_by_cell_noalloc(soax_t h, int32_t grid, uint32_t* perm_out, void* stream);

/* ------------------------------------------------- whole-array operations */

/* SetToValue applied to every array (apply<F>(), Listing 7): every element of every
 * plane of field (or of all fields when field == -1) of the live set becomes value,
 * converted to the field's type as a C cast would.  SOAX_EINVAL (nothing written) if
 * value is not exactly representable in an integer field, or overflows an f32 field. */
int soax_fill(soax_t h, int32_t field, double value, void* stream);

/* Fused elementwise expression over planes of the live set (the expression templates
 * of Sec. 4.2, e.g. posArr(0) = velArr(1) - velArr(2) of Listing 5), one pass:
 *   dst[i] = constant + sum_k coefs[k] * src_k[i],
 * accumulated left to right with one fused multiply-add per term, in the planes' type
 * (all planes f32, or all f64; coefficients rounded to it).  nterms in 0..8; src_fields,
 * src_comps and coefs are host arrays of nterms entries; dst may be one of the sources. */
int soax_lincomb(soax_t h, int32_t dst_field, int32_t dst_comp, int32_t nterms, const int32_t* src_fields,
                 const int32_t* src_comps, const double* coefs, double constant, void* stream);

/* One operation of a whole-array expression (soax_expr): a postfix program evaluated
 * element by element on a stack of values of the compute type. */
typedef enum {
  SOAX_EXPR_LOAD = 0,  /* push element i of plane (field, comp) of the live set, converted
                          to the compute type as a C cast would (rounded to nearest)     */
  SOAX_EXPR_CONST = 1, /* push value, rounded to the compute type                        */
  SOAX_EXPR_ADD = 2,   /* pop b, pop a, push a + b (one IEEE rounding; SUB, MUL, DIV alike) */
  SOAX_EXPR_SUB = 3,
  SOAX_EXPR_MUL = 4,
  SOAX_EXPR_DIV = 5,
  SOAX_EXPR_NEG = 6,   /* pop a, push -a                                                 */
  SOAX_EXPR_ABS = 7,   /* pop a, push |a|                                                */
  SOAX_EXPR_SQRT = 8,  /* pop a, push sqrt(a), correctly rounded                         */
  SOAX_EXPR_MIN = 9,   /* pop b, pop a, push (a < b ? a : b)                             */
  SOAX_EXPR_MAX = 10,  /* pop b, pop a, push (a > b ? a : b)                             */
  SOAX_EXPR_FMA = 11   /* pop c, pop b, pop a, push a*b + c with one rounding            */
} soax_expr_opcode;

typedef struct {
  int32_t op;     /* soax_expr_opcode                          */
  int32_t field;  /* SOAX_EXPR_LOAD: field index; else ignored  */
  int32_t comp;   /* SOAX_EXPR_LOAD: component; else ignored    */
  int32_t pad;
  double value;   /* SOAX_EXPR_CONST: the constant; else ignored */
} soax_expr_op;

/* General whole-array expression, one pass over the planes it reads and writes (the
 * expression templates of Sec. 4.2 -- posArr(0) = velArr(1) - velArr(2) in Listing 5 --
 * with the loop fusion of Sec. 4.2.2, as a program chosen at run time): for every
 * particle i, run the postfix program prog[0..nops-1] with element i of each loaded plane
 * and store the one value left into plane (dst_field, dst_comp), rounded to its type.
 * Sources may have any type (mixed-type expressions); the arithmetic runs in
 * compute_dtype (SOAX_F32 or SOAX_F64), every operation rounded as IEEE 754 specifies
 * (no contraction: a*b + c is two roundings unless written as SOAX_EXPR_FMA).  The
 * destination must be an f32 or f64 field and may also be a source.  Limits: nops in
 * 1..64, at most 16 loads, stack depth at most 16; the program must never pop an empty
 * stack and must leave exactly one value (SOAX_EINVAL otherwise, before any launch). */
int soax_expr(soax_t h, int32_t dst_field, int32_t dst_comp, const soax_expr_op* prog, int32_t nops,
              int32_t compute_dtype, void* stream);

/* ------------------------------------------------- Euler step (Eq. 1) */

/* The paper's benchmark step x += dt*v (Eq. 1, Sec. 2) in single precision on the live
 * f32 x 3 fields pos_field and vel_field (each update one rounded multiply and one
 * rounded add).  per_component = 0: one fused pass over all six planes;
 * per_component = 1: three launches, one per component, one element per thread (the
 * paper's GPU SoA benchmark, Sec. 3.2). */
int soax_euler(soax_t h, int32_t pos_field, int32_t vel_field, float dt, int32_t per_component,
               void* stream);

/* The same step on n AoS records of record_bytes bytes with f32 x[3] at byte x_off and
 * f32 v[3] at byte v_off, one thread per record (Particle<SIZE> of Listing 4).  The
 * buffer, the record size and the offsets must be multiples of 4 bytes. */
int soax_euler_aos(void* rec, int64_t n, int64_t record_bytes, int64_t x_off, int64_t v_off, float dt,
                   void* stream);

/* ---------------------------------------------------------------- adjoint */

/* Defining passages for the adjoint calls: the paper has no derivative of the step; they
 * differentiate soax_step's operation (Eq. 1 generalised, Sec. 2) in reverse mode, the
 * training-system form this library adds on top of it, with the loss of
 * soax_minimage_loss.
 *
 * Workspace bytes for K steps with a checkpoint every ckpt_every steps. */
int soax_adjoint_workspace_bytes(soax_t h, int32_t K, int32_t ckpt_every, size_t* bytes);

/* Forward: K steps in place with soax_step_fused's arithmetic (bit-identical to
 * soax_step_fused(h, fl, K)), saving the state (position as fixed-point turns, velocity)
 * at steps 0, ckpt_every, 2*ckpt_every, ... into ws.  tau_field must be -1. */
int soax_step_checkpointed(soax_t h, const soax_flow* fl, int32_t K, int32_t ckpt_every, void* ws,
                           size_t ws_bytes, void* stream);

/* Reverse: given adjoints xbarK (3 f64 planes) and vbarK (3 f64 planes, or NULL for 0)
 * of the state after the K steps of the last soax_step_checkpointed on this ws,
 * recompute each segment from its checkpoint and write xbar0, vbar0 (3 f64 planes each)
 * and grad[4] = dL/d(A, B, C, tau) (device f64[4], summed over particles in a fixed
 * order: the result is bit-reproducible).  The f32 rounding of v and the periodic wrap
 * are differentiated as the identity.  Pointer arrays are host arrays of 3 device
 * pointers. */
int soax_step_adjoint(soax_t h, const soax_flow* fl, int32_t K, int32_t ckpt_every, void* ws,
                      size_t ws_bytes, const double* const* xbarK, const double* const* vbarK,
                      double* const* xbar0, double* const* vbar0, double* grad, void* stream);

/* L = (1/n) sum_p |d_p|^2 with d the minimum image of x_p - xtgt_p in the periodic box,
 * written to loss (device f64[1]); if xbar is not NULL, xbar = dL/dx = (2/n) d (3 f64
 * planes).  Deterministic.  xtgt: host array of 3 device pointers.  ws: at least
 * 8*ceil(n/256) bytes (an adjoint workspace of the same handle always suffices). */
int soax_minimage_loss(soax_t h, int32_t pos_field, const double* const* xtgt, double* loss,
                       double* const* xbar, void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------- batched */

/* Defining passages for the batched calls: the paper runs one particle set per program
 * (Sec. 2, 3); many independent sets advanced in one launch are this library's addition,
 * with soax_step's arithmetic per particle (Eq. 1 generalised) and the particle-level data
 * parallelism of the GPU SIMT model (Sec. 3.2).
 *
 * Workspace bytes for advancing nens ensembles with soax_step_batched (any tune). */
int soax_batched_workspace_bytes(const soax_t* hs, int32_t nens, const soax_tune* tune,
                                 size_t* bytes);

/* Advance nens (1..4096) independent ensembles (each its own handle and soax_flow; dt
 * must be equal) nsteps steps, every step one persistent launch over all ensembles (or,
 * with tune->fuse_steps, one launch for all steps).  Per particle the arithmetic is
 * bit-identical to soax_step (to soax_step_fused with tune->fuse_steps), whatever the
 * launch shape.  The first call for a given (hs, fls, tune, ws) builds a tile table on
 * the host and copies it into ws, synchronising the stream; later calls with the same
 * arguments only launch, so they can be captured in a CUDA graph.
 * tune == NULL: parts_per_thread 4, block 256, vec_bits 128, no fusion. */
int soax_step_batched(const soax_t* hs, const soax_flow* fls, int32_t nens, int32_t nsteps,
                      const soax_tune* tune, void* ws, size_t ws_bytes, void* stream);

/* Forget the plan soax_step_batched recorded for the workspace at ws (NULL or unknown:
 * no effect): the next call with it uploads its plan again.  The library skips the upload
 * when a workspace address comes back with the same plan, so call this whenever the
 * memory behind a workspace may have been written by anything else -- in particular
 * after allocating a workspace at an address an earlier, freed one had.  A plan the
 * memory no longer holds is not followed: the kernels find its header changed, do
 * nothing and record SOAX_EINVAL for soax_sync. */
int soax_batched_forget(const void* ws);

/* Time every candidate launch shape of one form on nsteps_probe steps of the given
 * ensembles (which it advances: pass scratch copies) and write the fastest to out.  The
 * form is read from out->fuse_steps on entry (0: one launch per step, 1: fused) and kept.
 * Synchronises. */
int soax_autotune(const soax_t* hs, const soax_flow* fls, int32_t nens, int32_t nsteps_probe,
                  void* ws, size_t ws_bytes, soax_tune* out, void* stream);

/* ------------------------------------------------------------------ status */

/* Synchronise stream, then report and clear the device status word of the current
 * device: SOAX_OK, or the code a device-side check stored since the last soax_sync.
 * SOAX_ECUDA if the stream reported an error. */
int soax_sync(void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SOAX_H */
