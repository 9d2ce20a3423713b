// Whole-array operations of the SoAx container (Sec. 4): SetToValue applied to every
// array (apply<F>(), Listing 7), fused linear combinations and general expressions over
// planes such as posArr(0) = velArr(1) - velArr(2) (Listing 5), evaluated in one pass per
// expression (the loop fusion of Sec. 4.2.2) instead of one pass per operator.
#include <cmath>
#include <cstring>
#include <string>

#include "soax_internal.h"

namespace soax {

constexpr int kMaxTerms = 8;

struct FillArgs {
  void* planes[kMaxPlanes];
  int32_t es[kMaxPlanes];
  uint64_t pattern[kMaxPlanes];  // the element's bytes, little-endian, in the low es bytes
  int nplanes;
  int64_t n;
};

__global__ void __launch_bounds__(256) k_fill(const __grid_constant__ FillArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int p = 0; p < a.nplanes; ++p) {
    const int es = a.es[p];
    // 16 bytes of the repeated element (es divides 16).
    uint64_t w = a.pattern[p];
    if (es == 1) w = (w & 0xFF) * 0x0101010101010101ull;
    else if (es == 4) w = (w & 0xFFFFFFFFull) * 0x0000000100000001ull;
    const uint4 v = make_uint4((uint32_t)w, (uint32_t)(w >> 32), (uint32_t)w, (uint32_t)(w >> 32));
    const int64_t bytes = a.n * es, n16 = bytes >> 4;
    uint4* dst = static_cast<uint4*>(a.planes[p]);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) dst[i] = v;
    unsigned char* tail = static_cast<unsigned char*>(a.planes[p]);
    for (int64_t i = (n16 << 4) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < bytes; i += stride)
      tail[i] = (unsigned char)(w >> (8 * (i % 8)));
  }
}

template <typename T>
struct LinArgs {
  T* dst;
  const T* src[kMaxTerms];
  T coef[kMaxTerms];
  T constant;
  int nterms;
  int64_t n;
};

__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T>
__global__ void __launch_bounds__(256) k_lincomb(const __grid_constant__ LinArgs<T> a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    T acc = a.constant;
    for (int k = 0; k < a.nterms; ++k) acc = fma_rn(a.coef[k], a.src[k][i], acc);
    a.dst[i] = acc;
  }
}


// ------------------------------------------------------------- general expressions
// A postfix program over planes of the live set, evaluated element by element in one
// pass (the expression templates of Sec. 4.2 with the loop fusion of Sec. 4.2.2, at run
// time).  Each block takes tiles of ept x blockDim consecutive elements: it first stages
// every loaded source of the tile in shared memory with asynchronous copies (all of the
// tile's loads in flight at once, no registers held), then runs the program over the
// tile's elements with the operand stack in shared memory (each thread owns its slots,
// so no barrier), then stores the result.  The program is the same for every element, so
// the interpreter's branches are uniform.
constexpr int kExprMaxOps = 64;
constexpr int kExprMaxLoads = 16;
constexpr int kExprMaxDepth = 16;
constexpr int kExprBlock = 256;

enum : int8_t { kOpLoad = 0, kOpConst, kOpAdd, kOpSub, kOpMul, kOpDiv, kOpNeg, kOpAbs, kOpSqrt, kOpMin, kOpMax,
                kOpFma };

struct ExprArgs {
  const void* lsrc[kExprMaxLoads];  // the loaded planes, in program order
  double value[kExprMaxOps];        // constants (kOpConst), as given
  int8_t op[kExprMaxOps];
  int8_t ltype[kExprMaxLoads];      // soax_dtype of each loaded plane
  int8_t les[kExprMaxLoads];        // its element size
  int nops, nload, depth, ept;
  void* dst;
  int dst_f32;
  int64_t n;
};

__device__ __forceinline__ void cp_async_4(void* smem, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)), "l"(g)
               : "memory");
}
__device__ __forceinline__ void cp_async_8(void* smem, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)), "l"(g)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

template <typename T>
__device__ __forceinline__ T expr_convert(uint64_t raw, int type);
template <>
__device__ __forceinline__ double expr_convert<double>(uint64_t raw, int type) {
  switch (type) {
    case SOAX_I32: return (double)(int32_t)(uint32_t)raw;
    case SOAX_I64: return __ll2double_rn((long long)raw);
    case SOAX_U8: return (double)(uint8_t)raw;
    case SOAX_F32: return (double)__uint_as_float((uint32_t)raw);
    default: return __longlong_as_double((long long)raw);
  }
}
template <>
__device__ __forceinline__ float expr_convert<float>(uint64_t raw, int type) {
  switch (type) {
    case SOAX_I32: return __int2float_rn((int)(uint32_t)raw);
    case SOAX_I64: return __ll2float_rn((long long)raw);
    case SOAX_U8: return (float)(uint8_t)raw;
    case SOAX_F32: return __uint_as_float((uint32_t)raw);
    default: return __double2float_rn(__longlong_as_double((long long)raw));
  }
}

__device__ __forceinline__ float e_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double e_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float e_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double e_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float e_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double e_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float e_div(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double e_div(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float e_sqrt(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double e_sqrt(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ float e_abs(float a) { return fabsf(a); }
__device__ __forceinline__ double e_abs(double a) { return fabs(a); }
__device__ __forceinline__ float e_const(double v, float*) { return __double2float_rn(v); }
__device__ __forceinline__ double e_const(double v, double*) { return v; }

template <typename T>
__global__ void __launch_bounds__(kExprBlock) k_expr(const __grid_constant__ ExprArgs a) {
  extern __shared__ __align__(16) unsigned char expr_smem[];
  const int tid = threadIdx.x, B = blockDim.x, E = a.ept;
  uint64_t* stage = reinterpret_cast<uint64_t*>(expr_smem);        // [nload][E][B] raw elements
  T* stk = reinterpret_cast<T*>(stage + (size_t)a.nload * E * B);  // [depth][E][B]
  const int64_t tile = (int64_t)E * B;
  for (int64_t t0 = (int64_t)blockIdx.x * tile; t0 < a.n; t0 += (int64_t)gridDim.x * tile) {
    for (int l = 0; l < a.nload; ++l) {
      const unsigned char* src = static_cast<const unsigned char*>(a.lsrc[l]);
      const int es = a.les[l];
      for (int k = 0; k < E; ++k) {
        const int64_t i = t0 + (int64_t)k * B + tid;
        uint64_t* slot = stage + ((size_t)l * E + k) * B + tid;
        if (i < a.n) {
          if (es == 8)
            cp_async_8(slot, src + i * 8);
          else if (es == 4)
            cp_async_4(slot, src + i * 4);
          else
            *slot = src[i];
        }
      }
    }
    cp_async_wait_all();
    int sp = 0, ld = 0;
    for (int j = 0; j < a.nops; ++j) {
      const int op = a.op[j];
      if (op == kOpLoad) {
        const int type = a.ltype[ld];
        for (int k = 0; k < E; ++k)
          stk[((size_t)sp * E + k) * B + tid] = expr_convert<T>(stage[((size_t)ld * E + k) * B + tid], type);
        ++ld;
        ++sp;
      } else if (op == kOpConst) {
        const T c = e_const(a.value[j], (T*)nullptr);
        for (int k = 0; k < E; ++k) stk[((size_t)sp * E + k) * B + tid] = c;
        ++sp;
      } else if (op == kOpNeg || op == kOpAbs || op == kOpSqrt) {
        for (int k = 0; k < E; ++k) {
          T& x = stk[((size_t)(sp - 1) * E + k) * B + tid];
          x = op == kOpNeg ? -x : (op == kOpAbs ? e_abs(x) : e_sqrt(x));
        }
      } else if (op == kOpFma) {
        for (int k = 0; k < E; ++k) {
          T& x = stk[((size_t)(sp - 3) * E + k) * B + tid];
          const T y = stk[((size_t)(sp - 2) * E + k) * B + tid], z = stk[((size_t)(sp - 1) * E + k) * B + tid];
          x = fma_rn(x, y, z);
        }
        sp -= 2;
      } else {
        for (int k = 0; k < E; ++k) {
          T& x = stk[((size_t)(sp - 2) * E + k) * B + tid];
          const T y = stk[((size_t)(sp - 1) * E + k) * B + tid];
          switch (op) {
            case kOpAdd: x = e_add(x, y); break;
            case kOpSub: x = e_sub(x, y); break;
            case kOpMul: x = e_mul(x, y); break;
            case kOpDiv: x = e_div(x, y); break;
            case kOpMin: x = x < y ? x : y; break;
            default: x = x > y ? x : y; break;
          }
        }
        --sp;
      }
    }
    for (int k = 0; k < E; ++k) {
      const int64_t i = t0 + (int64_t)k * B + tid;
      if (i < a.n) {
        const T r = stk[(size_t)k * B + tid];
        if (a.dst_f32)
          static_cast<float*>(a.dst)[i] = (float)r;
        else
          static_cast<double*>(a.dst)[i] = (double)r;
      }
    }
  }
}

static bool fill_pattern(int dtype, double v, uint64_t* pat) {
  switch (dtype) {
    case SOAX_I32: {
      if (!(v == std::floor(v) && v >= -2147483648.0 && v <= 2147483647.0)) return false;
      int32_t x = (int32_t)v;
      uint32_t u;
      std::memcpy(&u, &x, 4);
      *pat = u;
      return true;
    }
    case SOAX_I64: {
      if (!(v == std::floor(v) && v >= -9223372036854775808.0 && v < 9223372036854775808.0)) return false;
      int64_t x = (int64_t)v;
      std::memcpy(pat, &x, 8);
      return true;
    }
    case SOAX_U8:
      if (!(v == std::floor(v) && v >= 0.0 && v <= 255.0)) return false;
      *pat = (uint64_t)(uint8_t)v;
      return true;
    case SOAX_F32: {
      if (std::isfinite(v) && std::fabs(v) > 3.4028234663852886e38) return false;
      float x = (float)v;
      uint32_t u;
      std::memcpy(&u, &x, 4);
      *pat = u;
      return true;
    }
    case SOAX_F64:
      std::memcpy(pat, &v, 8);
      return true;
  }
  return false;
}

}  // namespace soax

using namespace soax;

extern "C" int soax_fill(soax_t h, int32_t field, double value, void* stream) {
  if (int r = check_handle(h)) return r;
  if (field < -1 || field >= (int)h->fields.size()) return fail(SOAX_EINVAL, "soax_fill: bad field");
  FillArgs a;
  a.nplanes = 0;
  for (size_t f = 0; f < h->fields.size(); ++f) {
    if (field >= 0 && (int)f != field) continue;
    const Field& F = h->fields[f];
    uint64_t pat = 0;
    if (!fill_pattern(F.dtype, value, &pat))
      return fail(SOAX_EINVAL, "soax_fill: value not representable in field '" + F.name + "'");
    for (int c = 0; c < F.ncomp; ++c) {
      void* p = h->planes[h->current][F.first_plane + c];
      if (!p && h->n > 0) return fail(SOAX_EUNBOUND, "soax_fill: plane not bound");
      a.planes[a.nplanes] = p;
      a.es[a.nplanes] = F.esize;
      a.pattern[a.nplanes] = pat;
      ++a.nplanes;
    }
  }
  if (h->n == 0) return SOAX_OK;
  a.n = h->n;
  const int grid = persistent_grid((const void*)k_fill, 256, 0, grid_for((h->n * 8 + 15) / 16, 256));
  k_fill<<<grid, 256, 0, as_stream(stream)>>>(a);
  return check_launch("soax_fill");
}

extern "C" int soax_lincomb(soax_t h, int32_t dst_field, int32_t dst_comp, int32_t nterms, const int32_t* src_fields,
                            const int32_t* src_comps, const double* coefs, double constant, void* stream) {
  if (int r = check_handle(h)) return r;
  if (nterms < 0 || nterms > kMaxTerms) return fail(SOAX_EINVAL, "soax_lincomb: nterms must be in 0..8");
  if (nterms > 0 && (!src_fields || !src_comps || !coefs)) return fail(SOAX_EINVAL, "soax_lincomb: NULL term arrays");
  auto plane_of = [&](int f, int c, void** out) -> int {
    if (f < 0 || f >= (int)h->fields.size() || c < 0 || c >= h->fields[f].ncomp)
      return fail(SOAX_EINVAL, "soax_lincomb: bad field or component");
    *out = h->planes[h->current][h->fields[f].first_plane + c];
    if (!*out && h->n > 0) return fail(SOAX_EUNBOUND, "soax_lincomb: plane not bound");
    return SOAX_OK;
  };
  void* dst = nullptr;
  if (int r = plane_of(dst_field, dst_comp, &dst)) return r;
  const int dt = h->fields[dst_field].dtype;
  if (dt != SOAX_F32 && dt != SOAX_F64) return fail(SOAX_ESCHEMA, "soax_lincomb: planes must be f32 or f64");
  const void* src[kMaxTerms] = {};
  for (int k = 0; k < nterms; ++k) {
    void* p = nullptr;
    if (int r = plane_of(src_fields[k], src_comps[k], &p)) return r;
    if (h->fields[src_fields[k]].dtype != dt) return fail(SOAX_ESCHEMA, "soax_lincomb: all planes must share one type");
    src[k] = p;
  }
  if (h->n == 0) return SOAX_OK;
  cudaStream_t s = as_stream(stream);
  const int64_t wb = grid_for(h->n, 256);
  if (dt == SOAX_F32) {
    LinArgs<float> a;
    a.dst = static_cast<float*>(dst);
    for (int k = 0; k < nterms; ++k) {
      a.src[k] = static_cast<const float*>(src[k]);
      a.coef[k] = (float)coefs[k];
    }
    a.constant = (float)constant;
    a.nterms = nterms;
    a.n = h->n;
    k_lincomb<float><<<persistent_grid((const void*)k_lincomb<float>, 256, 0, wb), 256, 0, s>>>(a);
  } else {
    LinArgs<double> a;
    a.dst = static_cast<double*>(dst);
    for (int k = 0; k < nterms; ++k) {
      a.src[k] = static_cast<const double*>(src[k]);
      a.coef[k] = coefs[k];
    }
    a.constant = constant;
    a.nterms = nterms;
    a.n = h->n;
    k_lincomb<double><<<persistent_grid((const void*)k_lincomb<double>, 256, 0, wb), 256, 0, s>>>(a);
  }
  return check_launch("soax_lincomb");
}

extern "C" int soax_expr(soax_t h, int32_t dst_field, int32_t dst_comp, const soax_expr_op* prog, int32_t nops,
                         int32_t compute_dtype, void* stream) {
  if (int r = check_handle(h)) return r;
  if (!prog || nops < 1 || nops > kExprMaxOps) return fail(SOAX_EINVAL, "soax_expr: nops must be in 1..64");
  if (compute_dtype != SOAX_F32 && compute_dtype != SOAX_F64)
    return fail(SOAX_EINVAL, "soax_expr: compute_dtype must be SOAX_F32 or SOAX_F64");
  auto plane_of = [&](int f, int c, void** out) -> int {
    if (f < 0 || f >= (int)h->fields.size() || c < 0 || c >= h->fields[f].ncomp)
      return fail(SOAX_EINVAL, "soax_expr: bad field or component");
    *out = h->planes[h->current][h->fields[f].first_plane + c];
    if (!*out && h->n > 0) return fail(SOAX_EUNBOUND, "soax_expr: plane not bound");
    return SOAX_OK;
  };
  void* dst = nullptr;
  if (int r = plane_of(dst_field, dst_comp, &dst)) return r;
  const int dt = h->fields[dst_field].dtype;
  if (dt != SOAX_F32 && dt != SOAX_F64) return fail(SOAX_ESCHEMA, "soax_expr: the destination must be f32 or f64");
  ExprArgs a;
  std::memset(&a, 0, sizeof a);
  int sp = 0, depth = 0;
  for (int j = 0; j < nops; ++j) {
    const int op = prog[j].op;
    a.value[j] = prog[j].value;
    a.op[j] = (int8_t)op;
    int pops = 0, pushes = 1;
    switch (op) {
      case SOAX_EXPR_LOAD: {
        if (a.nload == kExprMaxLoads) return fail(SOAX_EINVAL, "soax_expr: at most 16 loads");
        void* p = nullptr;
        if (int r = plane_of(prog[j].field, prog[j].comp, &p)) return r;
        const Field& F = h->fields[prog[j].field];
        a.lsrc[a.nload] = p;
        a.ltype[a.nload] = (int8_t)F.dtype;
        a.les[a.nload] = (int8_t)F.esize;
        ++a.nload;
        break;
      }
      case SOAX_EXPR_CONST: break;
      case SOAX_EXPR_ADD: case SOAX_EXPR_SUB: case SOAX_EXPR_MUL: case SOAX_EXPR_DIV: case SOAX_EXPR_MIN:
      case SOAX_EXPR_MAX: pops = 2; break;
      case SOAX_EXPR_NEG: case SOAX_EXPR_ABS: case SOAX_EXPR_SQRT: pops = 1; break;
      case SOAX_EXPR_FMA: pops = 3; break;
      default: return fail(SOAX_EINVAL, "soax_expr: unknown operation " + std::to_string(op));
    }
    if (sp < pops) return fail(SOAX_EINVAL, "soax_expr: stack underflow at operation " + std::to_string(j));
    sp += pushes - pops;
    if (sp > depth) depth = sp;
    if (depth > kExprMaxDepth) return fail(SOAX_EINVAL, "soax_expr: stack deeper than 16");
  }
  if (sp != 1) return fail(SOAX_EINVAL, "soax_expr: the program must leave exactly one value");
  if (h->n == 0) return SOAX_OK;
  a.nops = nops;
  a.depth = depth;
  a.dst = dst;
  a.dst_f32 = dt == SOAX_F32;
  a.n = h->n;
  // Elements per thread: enough to give each block about 48 KB of staged loads and stack.
  const size_t tsz = compute_dtype == SOAX_F32 ? 4 : 8;
  const size_t per_elem = (size_t)a.nload * 8 + (size_t)depth * tsz;
  int ept = (int)((48u << 10) / (kExprBlock * per_elem));
  ept = ept < 1 ? 1 : (ept > 16 ? 16 : ept);
  a.ept = ept;
  const size_t smem = per_elem * ept * kExprBlock;
  const void* kern = compute_dtype == SOAX_F32 ? (const void*)k_expr<float> : (const void*)k_expr<double>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 << 10);
  if (e != cudaSuccess) return cuda_fail(e, "soax_expr: shared memory attribute");
  const int64_t tiles = (h->n + (int64_t)ept * kExprBlock - 1) / ((int64_t)ept * kExprBlock);
  const int grid = persistent_grid(kern, kExprBlock, smem, tiles);
  if (compute_dtype == SOAX_F32)
    k_expr<float><<<grid, kExprBlock, smem, as_stream(stream)>>>(a);
  else
    k_expr<double><<<grid, kExprBlock, smem, as_stream(stream)>>>(a);
  return check_launch("soax_expr");
}
