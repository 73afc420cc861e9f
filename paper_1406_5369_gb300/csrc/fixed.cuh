// Exact fixed-point arithmetic for the FP64 outer step of defect correction.
//
// The outer step forms r = f - A u for the finest FP64 level. On this GPU
// FP64 instructions issue at 1/64 of the FP32 rate, so five FP64 operations
// per node make that streaming pass several times slower than its memory
// traffic. When every axis of the constant stencil has the same coefficient
// c = 2^k (Poisson on the unit square or cube with n = 2^m + 1 nodes has
// c = 1/h^2 = 4^m), A u = c (2 dim u - sum of the neighbours) is evaluated
// exactly in 64-bit integers on the integer pipes instead:
//
//   A set of FP64 values whose largest biased exponent is M is held as
//   X = trunc(x * 2^(1085 - B)), B = M + kHead. The lowest bit weighs
//   2^(B - 1085); every |x| < 2^(M - 1022) gives |X| < 2^(63 - kHead) = 2^58,
//   so the stencil sum (at most 2 dim + 2 dim = 12 such terms) and the
//   difference F - S stay below 2^62 and never overflow. Values within a
//   factor 2^kHead of the largest one are represented exactly; smaller ones
//   are truncated at an absolute level of 2^(M - 1080), one thirty-second of
//   the FP64 unit in the last place of the largest value: below the rounding
//   error an FP64 evaluation of the same stencil would make.
//
// So the integer residual is the exact residual of the stored FP64 solution
// up to that truncation; it is rounded once, to FP32 (the inner defect) or
// to FP64 (norms accumulated in FP64). Everything here is integer and bit
// manipulation, except the final int64 -> FP32 (or FP64) conversion.
#pragma once

#include <cuda_runtime.h>

namespace mg {
namespace fx {

constexpr int kHead = 5;  // headroom bits above the largest represented value

// Biased IEEE-754 exponent of x (0 for zero and subnormals, 2047 for Inf/NaN).
__device__ __forceinline__ int dexp(double x) {
  return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ffull);
}

// trunc(x * 2^(1085 - Bt)) as a signed integer: Bt = B puts x on the grid
// 2^(B - 1085), Bt = B + k puts x / 2^k there (exactly). The 53-bit
// significand is placed at bits 57..5 and shifted right by Bt - kHead - ex
// (ex the biased exponent of x); subnormals and zero give 0. Every value a
// caller uses has ex <= Bt - kHead, so the result stays below 2^58 in
// magnitude; others (shift count negative) come out as 0 and are not used.
__device__ __forceinline__ long long to_fixed(double x, int Bt) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned ex = (hi >> 20) & 0x7ffu;
  unsigned long long m = ((unsigned long long)((hi & 0xfffffu) | 0x100000u) << 32) | lo;
  m = ex ? m : 0ull;
  const unsigned t = min((unsigned)(Bt - kHead - (int)ex), 63u);
  const long long v = (long long)((m << kHead) >> t);
  const long long sg = (long long)((int)hi >> 31);  // 0 or -1
  return (v ^ sg) - sg;
}

// Powers of two whose product is 2^E for any E in [-252, 254], each a
// normal FP32 number (a row's scale factor; computed once per row).
struct Pow2f {
  float a, b;
};
__device__ __forceinline__ Pow2f pow2f(int E) {
  const int e1 = E / 2, e2 = E - e1;
  Pow2f p;
  p.a = __int_as_float((min(max(e1, -126), 127) + 127) << 23);
  p.b = __int_as_float((min(max(e2, -126), 127) + 127) << 23);
  return p;
}

// R * 2^E0 as FP32 (conversion rounds toward zero; the scaling by powers of
// two is exact inside the normal range). The int64 -> FP32 conversion
// instruction issues on the FP64 pipe; an integer-only conversion measured
// slower here, where the integer pipe is the busier one.
__device__ __forceinline__ float fixed_to_float(long long R, const Pow2f &p) {
  return (__ll2float_rz(R) * p.a) * p.b;
}

// R * 2^E0 as FP64 (conversion rounds toward zero), with s = 2^E0.
__device__ __forceinline__ double fixed_to_double(long long R, double s) { return __ll2double_rz(R) * s; }

// x >> d for a warp-uniform d >= 0 (arithmetic shift, clamped at 63).
__device__ __forceinline__ long long align_down(long long x, int d) { return x >> (d < 63 ? d : 63); }

__device__ __forceinline__ long long shfl_up64(long long v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ long long shfl_dn64(long long v) { return __shfl_down_sync(0xffffffffu, v, 1); }

// Row exponents are combined across the warp with one reduction each; a
// non-finite value marks its row with this sentinel (its residual is NaN).
constexpr int kNonFinite = 1 << 20;

}  // namespace fx
}  // namespace mg
