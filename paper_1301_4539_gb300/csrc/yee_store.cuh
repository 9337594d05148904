// Field storage formats. Every kernel computes in float; what changes is how
// the six field arrays are held in HBM:
//   kF32  : float (4 B)
//   kF16  : IEEE half (2 B), stored value = field * scale[comp]
//   kBF16 : bfloat16 (2 B), stored value = field * scale[comp]
//   kF16HL: two IEEE halves (4 B) hi = half(v), lo = half(v - hi) with
//           v = field * scale[comp]; read back as float(hi) + float(lo), which
//           is exact in float (22 significant bits at most), so about 2^-22
//           relative per store instead of half's 2^-11
//   kF24  : the upper 24 bits of the float (3 B: sign, 8 exponent bits, 15
//           mantissa bits; 2^-16 relative per store, the float's full range,
//           no scale). The value is rounded to 16 significant bits by
//           Veltkamp's splitting (Dekker 1971): c = v * (2^8 + 1),
//           hi = c + (v - c), three float operations in round-to-nearest,
//           after which the low 8 bits of hi's pattern are zero (they are
//           dropped for subnormal values, where the split is not exact).
//           Layout: each z slab holds nine 2-byte planes instead of six: the
//           high halves (bits 31..16) of ex, ey, ez, hx, hy, hz, then three
//           planes of byte pairs (bits 15..8) of (ex, ey), (ez, hx), (hy, hz),
//           first component in the low byte. A value is read back as
//           hi << 16 | lo << 8.
// Scales are powers of two, so scaling and unscaling are exact in float
// (barring overflow/underflow); conversion to the 2-byte formats rounds to
// nearest even.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace sophie {

enum StoreFmt : int { kF32 = 0, kF16 = 1, kBF16 = 2, kF16HL = 3, kF24 = 4,
                      // the step kernels' forms of kF16 / kBF16 / kF16HL when all six
                      // scales are equal: the kernel then computes on the scaled
                      // values themselves (the scheme is linear and a power-of-two
                      // scale commutes with round-to-nearest), with no scale
                      // multiplications; sources are scaled and probe samples
                      // unscaled instead (SrcTable::vmul, PrbTable::pmul)
                      kF16U = 5, kBF16U = 6, kF16HLU = 7 };

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

template <>
struct Store<kF24> {
  using T = unsigned short;  // element of a high-half plane or of a byte-pair plane
  static constexpr int kAlign = 8;
  // byte-pair plane of component f relative to its high-half plane, in planes
  static __device__ __forceinline__ int lo_shift(int f) { return 6 + f / 2 - f; }
  // Veltkamp's split of v into 16 significant bits (round to nearest)
  static __device__ __forceinline__ float2 split2(float2 v) {
    const float2 c = __fmul2_rn(v, make_float2(257.f, 257.f));
    // v - c rounded once (c * -1 is exact)
    return __fadd2_rn(c, __ffma2_rn(c, make_float2(-1.f, -1.f), v));
  }
  static __device__ __forceinline__ float split(float v) {
    const float c = __fmul_rn(v, 257.f);
    return __fadd_rn(c, __fsub_rn(v, c));
  }
  // Component f of two adjacent points: p points at the first point's high half,
  // cs = elements between component planes.
  static __device__ __forceinline__ float2 ld2f(const T* p, int f, long long cs) {
    const uint32_t h = *reinterpret_cast<const uint32_t*>(p);
    const uint32_t l = *reinterpret_cast<const uint32_t*>(p + lo_shift(f) * cs);
    // [0, lo(c0), 0, lo(c1)] of this component, then [0, lo, hi.lo, hi.hi] per point
    const uint32_t z = __byte_perm(l, 0u, (f & 1) ? 0x3414u : 0x2404u);
    return make_float2(__uint_as_float(__byte_perm(z, h, 0x5410u)), __uint_as_float(__byte_perm(z, h, 0x7632u)));
  }
  static __device__ __forceinline__ float ldf(const T* p, int f, long long cs) {
    const uint32_t h = p[0];
    const uint32_t l = (p[lo_shift(f) * cs] >> ((f & 1) * 8)) & 0xFFu;
    return __uint_as_float((h << 16) | (l << 8));
  }
};

// The unit-scale forms: the base format's storage with no scale factors.
template <>
struct Store<kF16U> {
  using T = __half;
  static constexpr int kAlign = 8;
  static __device__ __forceinline__ float2 ld2(const T* p, float) {
    return __half22float2(*reinterpret_cast<const __half2*>(p));
  }
  static __device__ __forceinline__ float ld(const T* p, float) { return __half2float(*p); }
  static __device__ __forceinline__ void st2(T* p, float a, float b, float) {
    *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a, b);
  }
  static __device__ __forceinline__ void st(T* p, float a, float) { *p = __float2half_rn(a); }
};

template <>
struct Store<kBF16U> {
  using T = __nv_bfloat16;
  static constexpr int kAlign = 8;
  static __device__ __forceinline__ float2 ld2(const T* p, float) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
  }
  static __device__ __forceinline__ float ld(const T* p, float) { return __bfloat162float(*p); }
  static __device__ __forceinline__ void st2(T* p, float a, float b, float) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
  }
  static __device__ __forceinline__ void st(T* p, float a, float) { *p = __float2bfloat16_rn(a); }
};

template <>
struct Store<kF16HLU> {
  using T = __half2;  // .x = hi, .y = lo
  static constexpr int kAlign = 4;
  static __device__ __forceinline__ float dec(__half2 h) { return __fadd_rn(__low2float(h), __high2float(h)); }
  static __device__ __forceinline__ __half2 enc(float v) {
    const __half hi = __float2half_rn(v);
    const __half lo = __float2half_rn(__fsub_rn(v, __half2float(hi)));
    return __halves2half2(hi, lo);
  }
  static __device__ __forceinline__ float2 ld2(const T* p, float) {
    const uint2 raw = *reinterpret_cast<const uint2*>(p);
    return make_float2(dec(*reinterpret_cast<const __half2*>(&raw.x)), dec(*reinterpret_cast<const __half2*>(&raw.y)));
  }
  static __device__ __forceinline__ float ld(const T* p, float) { return dec(*p); }
  static __device__ __forceinline__ void st2(T* p, float a, float b, float) {
    const __half2 ha = enc(a), hb = enc(b);
    uint2 raw;
    raw.x = *reinterpret_cast<const unsigned int*>(&ha);
    raw.y = *reinterpret_cast<const unsigned int*>(&hb);
    *reinterpret_cast<uint2*>(p) = raw;
  }
  static __device__ __forceinline__ void st(T* p, float a, float) { *p = enc(a); }
};

// Bytes per stored element (a value, or for kF24 one of a value's 2-byte parts).
__host__ __device__ constexpr int store_bytes(int fmt) {
  return fmt == kF16 || fmt == kBF16 || fmt == kF24 || fmt == kF16U || fmt == kBF16U ? 2 : 4;
}
// Planes per z slab: six components, or nine 2-byte planes for kF24.
__host__ __device__ constexpr int store_planes(int fmt) { return fmt == kF24 ? 9 : 6; }

// Format-generic access used by the kernels. p points at component f of a
// point in a plane-major buffer whose component planes are cs elements apart
// (a shared-memory stage or a global field buffer); inv = 1 / scale.
template <int F>
__device__ __forceinline__ float2 ld2c(const typename Store<F>::T* p, float inv, int f, long long cs) {
  if constexpr (F == kF24)
    return Store<kF24>::ld2f(p, f, cs);
  else
    return Store<F>::ld2(p, inv);
}
template <int F>
__device__ __forceinline__ float ldc(const typename Store<F>::T* p, float inv, int f, long long cs) {
  if constexpr (F == kF24)
    return Store<kF24>::ldf(p, f, cs);
  else
    return Store<F>::ld(p, inv);
}
// Store the six components v[f][0..1] of two adjacent points at o (the first
// point's ex), component planes cs elements apart; mask bit 0 / 1 selects the
// first / second point. With both points the first must sit at an even index.
template <int F>
__device__ __forceinline__ void st6(typename Store<F>::T* o, long long cs, const float (&v)[6][2], const float* sc,
                                    int mask) {
  if constexpr (F == kF24) {
    uint32_t r[6][2];
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const float2 q = Store<kF24>::split2(make_float2(v[f][0], v[f][1]));
      r[f][0] = __float_as_uint(q.x);
      r[f][1] = __float_as_uint(q.y);
    }
    unsigned short* u = o;
    if (mask == 3) {
#pragma unroll
      for (int f = 0; f < 6; ++f) *reinterpret_cast<uint32_t*>(u + f * cs) = __byte_perm(r[f][0], r[f][1], 0x7632u);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        // [lo(2q, c0), lo(2q+1, c0), lo(2q, c1), lo(2q+1, c1)]
        const uint32_t a = __byte_perm(r[2 * q][0], r[2 * q + 1][0], 0x0051u);
        const uint32_t b = __byte_perm(r[2 * q][1], r[2 * q + 1][1], 0x5100u);
        *reinterpret_cast<uint32_t*>(u + (6 + q) * cs) = __byte_perm(a, b, 0x7610u);
      }
    } else if (mask) {
      // one point: selects rather than an index, so r stays in registers
      const bool sec = mask == 2;
      unsigned short* w = u + (sec ? 1 : 0);
#pragma unroll
      for (int f = 0; f < 6; ++f) w[f * cs] = (unsigned short)((sec ? r[f][1] : r[f][0]) >> 16);
#pragma unroll
      for (int q = 0; q < 3; ++q)
        w[(6 + q) * cs] = (unsigned short)__byte_perm(sec ? r[2 * q][1] : r[2 * q][0],
                                                      sec ? r[2 * q + 1][1] : r[2 * q + 1][0], 0x0051u);
    }
  } else {
    using S = Store<F>;
    if (mask == 3) {
#pragma unroll
      for (int f = 0; f < 6; ++f) S::st2(o + f * cs, v[f][0], v[f][1], sc[f]);
    } else if (mask == 1) {
#pragma unroll
      for (int f = 0; f < 6; ++f) S::st(o + f * cs, v[f][0], sc[f]);
    } else if (mask == 2) {
#pragma unroll
      for (int f = 0; f < 6; ++f) S::st(o + f * cs + 1, v[f][1], sc[f]);
    }
  }
}

}  // namespace sophie
