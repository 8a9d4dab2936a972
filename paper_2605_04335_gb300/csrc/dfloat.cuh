// Double-FP32 outer loop of the mixed-precision solve (precision mode 2).
//
// Iterative refinement needs the fine residual r = b - lambda - A p in a precision well
// above that of the inner FP32 multigrid; the classical three-precision choice is a
// residual precision equal to the square of the inner one (2^-48 for FP32).  GB300 issues
// FP64 at about 1/64 of its FP32 rate, so native FP64 makes the residual the most
// expensive kernel of a refinement step.  This mode keeps the accumulated solution p, the
// right-hand side b and the stencil coefficients as unevaluated sums hi + lo of two floats
// (48 significant bits) and forms the residual with error-free transformations on the
// FP32 pipe:
//   two_sum(a, b)       s + e = a + b exactly                 (Knuth, 6 flops)
//   fast_two_sum(a, b)  s + e = a + b exactly when |a| >= |b|  (Dekker, 3 flops)
//   two_prod(a, b)      p + e = a * b exactly                  (one FMA for e)
// A product of two pairs keeps hi*hi exactly plus the two cross terms (dropping lo*lo,
// 2^-48 relative); the seven stencil products and b - lambda are summed with two_sum on
// the high parts and a plain float sum of all low parts.  The residual then carries an
// error of a few units of 2^-48 times sum |c| |p| over the stencil, the same form as the
// FP64 residual's 2^-53 bound.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace ibm {
namespace dfl {

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  e = b - (s - a);
}

// (acc_h, acc_l) += (a_h, a_l) * (b_h, b_l); acc_l collects every low-order part
__device__ __forceinline__ void acc_prod(float ah, float al, float bh, float bl, float &acc_h, float &acc_l) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  float s, t;
  two_sum(acc_h, p, s, t);
  acc_h = s;
  acc_l += t + e;
}

// exact float -> double widening by bit manipulation (keeps the FP64 pipe free); normal
// floats, zero and inf map exactly, NaN to a NaN; subnormal floats (below 2^-126, far under any
// low part that matters here) become signed zero
__device__ __forceinline__ double widen(float x) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t s = u & 0x80000000u, ex = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  uint32_t hi, lo = m << 29;
  if (ex == 0) hi = s, lo = 0u;
  else if (ex == 0xffu) hi = s | 0x7ff00000u | (m ? 0x80000u : 0u);   // inf, or a quiet NaN
  else hi = s | ((ex + 896u) << 20) | (m >> 3);
  return __hiloint2double((int)hi, (int)lo);
}

// double -> float by truncating the significand (bit manipulation after the IEEE 754
// binary64 / binary32 layouts, so the FP64 pipe stays free): normal results lie within one
// unit in the last place of the float, toward zero; magnitudes below 2^-126 become signed
// zero, above the float range infinity, and a NaN stays a NaN
__device__ __forceinline__ float narrow_trunc(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const uint32_t s = hi & 0x80000000u, ex = (hi >> 20) & 0x7ffu;
  uint32_t bits;
  if (ex <= 896u) bits = s;
  else if (ex >= 1151u) bits = s | 0x7f800000u | ((ex == 0x7ffu && ((hi & 0xfffffu) | lo)) ? 0x400000u : 0u);
  else bits = s | ((ex - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  return __uint_as_float(bits);
}

// hi + lo as a double (one FP64 add)
__device__ __forceinline__ double join(float h, float l) { return widen(h) + widen(l); }

// double -> (hi, lo): hi the nearest float, lo the nearest float to the remainder
__device__ __forceinline__ void split(double x, float &h, float &l) {
  h = __double2float_rn(x);
  l = __double2float_rn(x - widen(h));
}

}  // namespace dfl
}  // namespace ibm
