// Field storage formats. Every kernel computes in float; what changes is how
// the six field arrays are held in HBM:
//   kF32  : float (4 B)
//   kF16  : IEEE half (2 B), stored value = field * scale[comp]
//   kBF16 : bfloat16 (2 B), stored value = field * scale[comp]
//   kF16HL: two IEEE halves (4 B) hi = half(v), lo = half(v - hi) with
//           v = field * scale[comp]; read back as float(hi) + float(lo), which
//           is exact in float (22 significant bits at most), so about 2^-22
//           relative per store instead of half's 2^-11
// Scales are powers of two, so scaling and unscaling are exact in float
// (barring overflow/underflow); conversion to the 2-byte formats rounds to
// nearest even.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace sophie {

enum StoreFmt : int { kF32 = 0, kF16 = 1, kBF16 = 2, kF16HL = 3 };

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

template <>
struct Store<kF16HL> {
  using T = __half2;  // .x = hi, .y = lo
  static constexpr int kAlign = 4;
  static __device__ __forceinline__ float dec(__half2 h, float inv) {
    return __fadd_rn(__low2float(h), __high2float(h)) * inv;
  }
  static __device__ __forceinline__ __half2 enc(float a, float sc) {
    const float v = a * sc;
    const __half hi = __float2half_rn(v);
    const __half lo = __float2half_rn(__fsub_rn(v, __half2float(hi)));
    return __halves2half2(hi, lo);
  }
  static __device__ __forceinline__ float2 ld2(const T* p, float inv) {
    const uint2 raw = *reinterpret_cast<const uint2*>(p);
    return make_float2(dec(*reinterpret_cast<const __half2*>(&raw.x), inv),
                       dec(*reinterpret_cast<const __half2*>(&raw.y), inv));
  }
  static __device__ __forceinline__ float ld(const T* p, float inv) { return dec(*p, inv); }
  static __device__ __forceinline__ void st2(T* p, float a, float b, float sc) {
    const __half2 ha = enc(a, sc), hb = enc(b, sc);
    uint2 raw;
    raw.x = *reinterpret_cast<const unsigned int*>(&ha);
    raw.y = *reinterpret_cast<const unsigned int*>(&hb);
    *reinterpret_cast<uint2*>(p) = raw;
  }
  static __device__ __forceinline__ void st(T* p, float a, float sc) { *p = enc(a, sc); }
};

// Bytes per stored value.
__host__ __device__ constexpr int store_bytes(int fmt) { return fmt == kF16 || fmt == kBF16 ? 2 : 4; }

}  // namespace sophie
