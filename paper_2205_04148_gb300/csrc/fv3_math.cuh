// fv3_math.cuh -- FP64 helpers that save FP64 pipe time on this GPU (2 FP64
// lanes per SM per clock, so every FP64 instruction counts).
#pragma once

namespace fv3 {

// 1 / x.  FP64: the hardware reciprocal approximation of the high word
// (rcp.approx.ftz.f64) refined by two Newton-Raphson steps
// r <- r + r (1 - x r), each of which squares the relative error; within an
// ulp of the quotient for normal x (checked against division by
// fv3_math_check).  The float path divides.
template <typename R>
__device__ __forceinline__ R rcp(R x) { return R(1) / x; }
template <>
__device__ __forceinline__ double rcp<double>(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// ln(pen / pe) for pen = pe + dp, pe > 0, pen > 0.  With u = dp / (pe + pen),
// pen / pe = (1 + u) / (1 - u) and ln(pen / pe) = 2 atanh(u) =
// 2 (u + u^3/3 + u^5/5 + ...), the Taylor series of atanh.  For |u| <= 1/8
// the terms through u^15 leave a truncation error below 2^-52 relative; the
// thin upper layers (larger u) take the library logarithm.
__device__ __forceinline__ double log_ratio(double pen, double pe, double dp) {
  const double u = dp * rcp(pe + pen);
  if (fabs(u) > 0.125) return log(pen / pe);
  const double v = u * u;
  double s = 1.0 / 15.0;
  s = fma(s, v, 1.0 / 13.0);
  s = fma(s, v, 1.0 / 11.0);
  s = fma(s, v, 1.0 / 9.0);
  s = fma(s, v, 1.0 / 7.0);
  s = fma(s, v, 1.0 / 5.0);
  s = fma(s, v, 1.0 / 3.0);
  s = fma(s, v, 1.0);
  return 2.0 * u * s;
}

}  // namespace fv3
