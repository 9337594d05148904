// The Yee update expressions, shared by every step kernel so that all of them
// (plain, temporally blocked) produce bitwise identical fields.
//
// Sec. 2.1 (displayed Hx update and its analogues for the other components):
//   br = (a1 - a0) - (b1 - b0) [+ s]
//   h  = fma(S, br, h)
//   e  = fma(Cb, br, Ca*e)
// with every other operation rounded separately, in exactly this order, so
// the float results are fixed by the expression alone (the CPU oracle
// evaluates the same expression with C's fmaf).
//
// Operand roles per component (index offsets on the storage box):
//   hx: a = ey(k+1), ey(k)   b = ez(j+1), ez(j)
//   hy: a = ez(i+1), ez(i)   b = ex(k+1), ex(k)
//   hz: a = ex(j+1), ex(j)   b = ey(i+1), ey(i)
//   ex: a = hz(j), hz(j-1)   b = hy(k), hy(k-1)
//   ey: a = hx(k), hx(k-1)   b = hz(i), hz(i-1)
//   ez: a = hy(i), hy(i-1)   b = hx(j), hx(j-1)
// On a non-uniform mesh the a difference is scaled by the ratio of the axis
// it is taken along (hx: rz(k), ez: rxd(i), ...) and the b difference likewise;
// primary widths for H, dual widths for E.
#pragma once

namespace sophie {

__device__ __forceinline__ float curl_br(float a1, float a0, float b1, float b0) {
  return __fsub_rn(__fsub_rn(a1, a0), __fsub_rn(b1, b0));
}

__device__ __forceinline__ float h_upd(float h, float S, float a1, float a0, float b1, float b0) {
  return __fmaf_rn(S, curl_br(a1, a0, b1, b0), h);
}

// Non-uniform mesh (Sec. 2.2's 1-D geometric coefficients): each difference
// is scaled by the ratio reference step / width it spans,
//   br = fma(ra, a1 - a0, -(rb * (b1 - b0)))
// which with ra = rb = 1 rounds exactly like curl_br.
__device__ __forceinline__ float curl_br_nu(float ra, float a1, float a0, float rb, float b1, float b0) {
  return __fmaf_rn(ra, __fsub_rn(a1, a0), -__fmul_rn(rb, __fsub_rn(b1, b0)));
}

// The bracket of either mesh: NU selects the scaled form (ratios unused otherwise).
template <bool NU>
__device__ __forceinline__ float bracket(float ra, float a1, float a0, float rb, float b1, float b0) {
  if constexpr (NU)
    return curl_br_nu(ra, a1, a0, rb, b1, b0);
  else
    return curl_br(a1, a0, b1, b0);
}

template <bool NU>
__device__ __forceinline__ float h_upd_r(float h, float S, float ra, float a1, float a0, float rb, float b1,
                                         float b0) {
  return __fmaf_rn(S, bracket<NU>(ra, a1, a0, rb, b1, b0), h);
}

__device__ __forceinline__ float e_upd(float e, float2 c, float br) {
  return __fmaf_rn(c.y, br, __fmul_rn(c.x, e));
}

// Two adjacent points at once with Blackwell's packed f32x2 operations: each
// half of a packed operation is rounded exactly like its scalar counterpart
// (no flush to zero), so these give bitwise the results of curl_br and h_upd
// on (.x, .y) with half the float instructions.
__device__ __forceinline__ float2 fsub2_rn(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 pa, pb, pr;\n\t"
      "mov.b64 pa, {%2, %3};\n\t"
      "mov.b64 pb, {%4, %5};\n\t"
      "sub.rn.f32x2 pr, pa, pb;\n\t"
      "mov.b64 {%0, %1}, pr;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}

__device__ __forceinline__ float2 curl_br2(float2 a1, float2 a0, float2 b1, float2 b0) {
  return fsub2_rn(fsub2_rn(a1, a0), fsub2_rn(b1, b0));
}

__device__ __forceinline__ float2 h_upd2(float2 h, float S, float2 a1, float2 a0, float2 b1, float2 b0) {
  return __ffma2_rn(make_float2(S, S), curl_br2(a1, a0, b1, b0), h);
}

// Packed form of curl_br_nu with the b ratio passed negated, nrb = -rb:
// (-rb) * d rounds to exactly -(rb * d), so the bracket is the same value.
__device__ __forceinline__ float2 curl_br2_nu(float2 ra, float2 a1, float2 a0, float2 nrb, float2 b1, float2 b0) {
  return __ffma2_rn(ra, fsub2_rn(a1, a0), __fmul2_rn(nrb, fsub2_rn(b1, b0)));
}

}  // namespace sophie
