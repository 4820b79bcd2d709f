// fv3_math.cuh -- FP64 helpers that save FP64 pipe time on this GPU (2 FP64
// lanes per SM per clock, so every FP64 instruction counts): order-preserving
// integer keys for compares, the PPM limiter (reading R4) on the integer
// pipe, a Newton-refined reciprocal and a series log pressure ratio.
#pragma once

namespace fv3 {

// FP64 specialisation.  On this GPU the FP64 pipe has 2 lanes per SM and per
// clock, and FP64 compares, min/max and |x| occupy it like arithmetic does.
// They are done here on the integer pipe instead, on the IEEE bit patterns:
// x -> b ^ ((b >> 63) & 0x7fff...f) is an order-preserving signed integer
// key, the magnitude bits of non-negative doubles order like the values, and
// 2|x| is |x| with the exponent raised by one (twice the bits below the
// normal range).  Results are the same as the generic version except for the
// sign of zero in ties of the clamp, and except when bl*br underflows to zero
// (opposite-signed slopes below 1e-162), neither of which changes a value.
__device__ __forceinline__ long long okey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ long long twice_mag(long long m) {
  return m < (1LL << 52) ? (m << 1) : m + (1LL << 52);
}

// monotone limiter on the cell's deviations (generic, then FP64 on the
// integer pipe -- see okey / twice_mag above)
template <typename R>
__device__ __forceinline__ void ppm_limit(R& bl, R& br) {
  if (bl * br >= R(0)) {
    bl = R(0);
    br = R(0);
  } else if (fabs(bl) > R(2) * fabs(br)) {
    bl = R(-2) * br;
  } else if (fabs(br) > R(2) * fabs(bl)) {
    br = R(-2) * bl;
  }
}
template <>
__device__ __forceinline__ void ppm_limit<double>(double& bl, double& br) {
  const long long sb = __double_as_longlong(bl), sr = __double_as_longlong(br);
  const long long MAG = 0x7fffffffffffffffLL;
  const long long mb = sb & MAG, mr = sr & MAG;
  if ((sb ^ sr) >= 0 || mb == 0 || mr == 0) {
    bl = 0.0;
    br = 0.0;
  } else if (mb > twice_mag(mr)) {
    bl = __longlong_as_double(twice_mag(mr) | (~sr & ~MAG));
  } else if (mr > twice_mag(mb)) {
    br = __longlong_as_double(twice_mag(mb) | (~sb & ~MAG));
  }
}

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
