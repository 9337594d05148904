// Field storage formats. Every kernel computes in float; what changes is how
// the six field arrays are held in HBM:
//   kF32  : float (4 B)
//   kF16  : IEEE half (2 B), stored value = field * scale[comp]
//   kBF16 : bfloat16 (2 B), stored value = field * scale[comp]
// Scales are powers of two, so scaling and unscaling are exact in float
// (barring overflow/underflow); conversion to the 2-byte formats rounds to
// nearest even.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace sophie {

enum StoreFmt : int { kF32 = 0, kF16 = 1, kBF16 = 2 };

template <int F>
struct Store;

template <>
struct Store<kF32> {
  using T = float;
  static constexpr int kAlign = 4;  // TMA x-coordinate granule in elements (16 B)
  static __device__ __forceinline__ float2 ld2(const T* p, float) {
    return *reinterpret_cast<const float2*>(p);
  }
  static __device__ __forceinline__ float ld(const T* p, float) { return *p; }
  static __device__ __forceinline__ void st2(T* p, float a, float b, float) {
    *reinterpret_cast<float2*>(p) = make_float2(a, b);
  }
  static __device__ __forceinline__ void st(T* p, float a, float) { *p = a; }
};

template <>
struct Store<kF16> {
  using T = __half;
  static constexpr int kAlign = 8;
  static __device__ __forceinline__ float2 ld2(const T* p, float inv) {
    const float2 v = __half22float2(*reinterpret_cast<const __half2*>(p));
    return make_float2(v.x * inv, v.y * inv);
  }
  static __device__ __forceinline__ float ld(const T* p, float inv) { return __half2float(*p) * inv; }
  static __device__ __forceinline__ void st2(T* p, float a, float b, float sc) {
    *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a * sc, b * sc);
  }
  static __device__ __forceinline__ void st(T* p, float a, float sc) { *p = __float2half_rn(a * sc); }
};

template <>
struct Store<kBF16> {
  using T = __nv_bfloat16;
  static constexpr int kAlign = 8;
  static __device__ __forceinline__ float2 ld2(const T* p, float inv) {
    const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
    return make_float2(v.x * inv, v.y * inv);
  }
  static __device__ __forceinline__ float ld(const T* p, float inv) { return __bfloat162float(*p) * inv; }
  static __device__ __forceinline__ void st2(T* p, float a, float b, float sc) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a * sc, b * sc);
  }
  static __device__ __forceinline__ void st(T* p, float a, float sc) { *p = __float2bfloat16_rn(a * sc); }
};

}  // namespace sophie
