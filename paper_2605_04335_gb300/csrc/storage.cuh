// Storage types of level arrays and their conversions to the arithmetic type.
//
// The multigrid computes in FP32 (mixed modes) or FP64; the error e and right-hand side r of
// the coarse levels swept by the fused z-march may be stored in BF16 instead (an option of the
// solve): every load widens exactly (a BF16 value is the upper half of the FP32 bit pattern),
// every store rounds to nearest even.  The helpers below are overloaded on the storage type,
// so one kernel body serves FP32, FP64 and BF16 storage.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace ibm {

using bf16 = __nv_bfloat16;

// the arithmetic type of a storage type
template <typename S> struct Arith { using type = S; };
template <> struct Arith<bf16> { using type = float; };

__device__ __forceinline__ float bf16_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t u) { return __uint_as_float(u & 0xffff0000u); }
__device__ __forceinline__ uint32_t bf16_pack(float a, float b) {   // a in the low half
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&v);
}

// one value
__device__ __forceinline__ float ld1(const float *p) { return *p; }
__device__ __forceinline__ double ld1(const double *p) { return *p; }
__device__ __forceinline__ float ld1(const bf16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ void st1(float *p, float v) { *p = v; }
__device__ __forceinline__ void st1(double *p, double v) { *p = v; }
__device__ __forceinline__ void st1(bf16 *p, float v) { *p = __float2bfloat16_rn(v); }

// two consecutive values (8-byte aligned for FP32, 16 for FP64, 4 for BF16)
__device__ __forceinline__ void ld2(const float *p, float v[2]) {
  const float2 a = *reinterpret_cast<const float2 *>(p);
  v[0] = a.x; v[1] = a.y;
}
__device__ __forceinline__ void ld2(const double *p, double v[2]) {
  const double2 a = *reinterpret_cast<const double2 *>(p);
  v[0] = a.x; v[1] = a.y;
}
__device__ __forceinline__ void ld2(const bf16 *p, float v[2]) {
  const uint32_t u = *reinterpret_cast<const uint32_t *>(p);
  v[0] = bf16_lo(u); v[1] = bf16_hi(u);
}

// a value as it reads back after a store of storage type S (identity unless S is narrower)
template <typename S> __device__ __forceinline__ float as_stored(float v) { return v; }
template <> __device__ __forceinline__ float as_stored<bf16>(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
template <typename S> __device__ __forceinline__ double as_stored(double v) { return v; }

}  // namespace ibm
