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

}  // namespace sophie
