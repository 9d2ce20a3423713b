// Cell key of a binary64 position on a G^3 grid, exactly as binary64 arithmetic defines
// it: c = RN(G / 2pi), i_d = min((int)RN(x_d c), G - 1), key = (iz G + iy) G + ix, with
// integer instructions only.  Shared by soax_cell_keys and the fused step's key output,
// so both give the same bits.
#pragma once
#include <cstdint>

namespace soax {

// c = RN(G / 2pi) in the three forms cell_index uses, built on the host (make_cell_key_k).
struct CellKeyK {
  uint64_t cfx;  // c 2^54 rounded to an integer
  uint64_t cm;   // c's 53-bit significand
  int ce;        // c's biased exponent
  int G;
};

// floor(RN(x * c)) for 0 <= x and 0 < c with x * c < 2^31, computed exactly with integer
// instructions (the binary64 product rounded to nearest-even, then truncated), so the
// result equals (int)(x * c) of IEEE binary64 arithmetic without using the FP64 pipe.
// cm: c's 53-bit significand; ce: c's biased exponent.
__device__ __forceinline__ int floor_mul_rn(double x, uint64_t cm, int ce) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0 || (b >> 63)) return 0;  // zero, subnormal or negative: the product truncates to 0
  const uint64_t mx = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  // M = mx * cm, 105 or 106 bits; x c = M 2^(ex + ce - 2150).
  const uint64_t hi = __umul64hi(mx, cm), lo = mx * cm;
  const int d = (hi >> 41) ? 53 : 52;  // bits to drop to keep 53 significant bits
  uint64_t mr = (hi << (64 - d)) | (lo >> d);
  const uint64_t rem = lo & ((1ull << d) - 1), half = 1ull << (d - 1);
  if (rem > half || (rem == half && (mr & 1))) ++mr;  // round to nearest, ties to even
  const int t = 2150 - ex - ce - d;  // RN(x c) = mr 2^-t
  if (t >= 64) return 0;
  if (t <= 0) return 0x7FFFFFFF;  // outside the key range (clamped by the caller)
  return (int)(mr >> t);
}

// Cell index of one coordinate.  Fast path: P = x c 2^51 in fixed point (X = x 2^61
// exact for 2^-8 <= x < 8, times c 2^54 rounded, high 64 bits) is within 3 units of the
// exact product; the binary64 rounding of x c moves it by at most 2^-44 (x c < 2^10),
// i.e. 128 units, so unless P lies within 131 units of an integer boundary its floor
// equals floor(RN(x c)).  Otherwise (probability ~2^-42, or x < 2^-8) the exact path.
__device__ __forceinline__ int cell_index(double x, uint64_t cfx, uint64_t cm, int ce) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int e = (int)(b >> 52);  // sign bit included: negative x takes the exact path
  if (e >= 1015 && e <= 1025) {
    const uint64_t X = ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << (e - 1014);
    const uint64_t P = __umul64hi(X, cfx);
    const uint64_t frac = P & ((1ull << 51) - 1);
    if (frac >= 131 && frac <= (1ull << 51) - 132) return (int)(P >> 51);
  }
  return floor_mul_rn(x, cm, ce);
}

__device__ __forceinline__ uint32_t cell_key(double x, double y, double z, const CellKeyK& k) {
  const int ix = min(cell_index(x, k.cfx, k.cm, k.ce), k.G - 1);
  const int iy = min(cell_index(y, k.cfx, k.cm, k.ce), k.G - 1);
  const int iz = min(cell_index(z, k.cfx, k.cm, k.ce), k.G - 1);
  return (uint32_t)((iz * k.G + iy) * k.G + ix);
}

}  // namespace soax
