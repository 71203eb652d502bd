// 64-bit fixed-point arithmetic for complex128 amplitudes on the integer pipes
// (used by the fused rotation pass, coset_fx.cuh, and the adjoint runs,
// adjoint.cu).  A value a is held as the signed integer A = round(a * 2^S) for
// an exponent S the caller keeps per coset; |A| < 2^61.  Conversions use the
// IEEE-754 binary64 layout (sign, 11-bit biased exponent, 52-bit fraction with
// an implicit leading one) with integer operations only; values below 2^-1022
// in magnitude (subnormals) are read as zero and results below it are written
// as zero.
#pragma once

#include <cstdint>

namespace pr {
namespace {

constexpr double kTwo62 = 4611686018427387904.0;  // 2^62
constexpr int64_t kTMax = (int64_t(1) << 62) - 1;
// growth bound of one rotation in units of 2^-20 bit
constexpr int kGrowthFrac = 20;

__device__ __forceinline__ void fx_limbs(int64_t T, int32_t &th, int32_t &tl) {
  th = (int32_t)(T >> 31);
  tl = (int32_t)(T & 0x7fffffffLL);
}

// B * T / 2^62, truncated, for |B| < 2^61 and T = th * 2^31 + tl, 0 <= tl < 2^31:
// with B = bh * 2^31 + bl (0 <= bl < 2^31),
//   B T / 2^62 = bh th + (bh tl + bl th) / 2^31 + bl tl / 2^62,
// computed as bh th + floor((bh tl + bl th) / 2^31): the last term (in [0, 1))
// is dropped and the shift floors, so the result is below the exact product by
// less than 2 units of 2^-S, by 3/4 of a unit on average.  The callers add that
// mean back once per component at the end of a run (every component receives
// exactly one product per rotation), not per product.  Written as PTX: each
// partial product is one 32 x 32 -> 64-bit multiply (mul.wide.s32) and the sums
// are plain 64-bit adds, the form that measured fastest on GB300 (a rounding
// constant added per product cost 12 % of the multiply-add rate, 64-bit
// multiply-add addends another 19 %).
__device__ __forceinline__ int64_t fx_prod(int64_t b, int32_t th, int32_t tl) {
  int64_t r;
  asm("{\n\t"
      ".reg .b32 bl, bh;\n\t"
      ".reg .b64 m, n;\n\t"
      "mov.b64 {bl, bh}, %1;\n\t"
      "shf.r.clamp.b32 bh, bl, bh, 31;\n\t"
      "and.b32 bl, bl, 0x7fffffff;\n\t"
      "mul.wide.s32 m, bh, %3;\n\t"
      "mul.wide.s32 n, bl, %2;\n\t"
      "add.s64 m, m, n;\n\t"
      "shr.s64 m, m, 31;\n\t"
      "mul.wide.s32 n, bh, %2;\n\t"
      "add.s64 %0, n, m;\n\t"
      "}"
      : "=l"(r)
      : "l"(b), "r"(th), "r"(tl));
  return r;
}

// binary64 -> A = round(a * 2^S), with kbase = 1085 - S; needs 1085 - S - e >= 2
// for every exponent field e of the coset (guaranteed by the choice of S)
__device__ __forceinline__ int64_t fx_in(double a, int kbase) {
  const uint64_t b = (uint64_t)__double_as_longlong(a);
  const int e = (int)((b >> 52) & 0x7ffu);
  const int k = kbase - e;  // >= 2
  const int ks = k < 63 ? k : 63;
  const uint64_t m10 = ((b & 0xfffffffffffffULL) | 0x10000000000000ULL) << 10;  // < 2^63
  uint64_t mag = (m10 + (1ULL << (ks - 1))) >> ks;
  mag = (k < 64 && e != 0) ? mag : 0ULL;
  return (b >> 63) ? -(int64_t)mag : (int64_t)mag;
}

// A * 2^-S -> binary64 (rounded to nearest, ties away from zero), ebase = 1086 - S
__device__ __forceinline__ double fx_out(int64_t a, int ebase) {
  const uint64_t v = a < 0 ? (uint64_t)(-a) : (uint64_t)a;
  const int lz = __clzll((long long)v);
  const uint64_t nm = v << (lz & 63);  // leading one at bit 63
  const uint64_t m53 = (nm >> 11) + ((nm >> 10) & 1ULL);  // in [2^52, 2^53]
  const int eb = ebase - lz;                               // biased exponent
  uint64_t bits = ((uint64_t)(int64_t)(eb - 1) << 52) + m53;
  bits = (v == 0 || eb <= 0) ? 0ULL : bits;
  return __longlong_as_double((long long)(bits | ((uint64_t)a & 0x8000000000000000ULL)));
}

}  // namespace
}  // namespace pr
