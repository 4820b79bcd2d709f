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
// integer pipe -- see okey / twice_mag above).  The cases are: a local
// extremum (bl br >= 0: both zero), |bl| > 2|br| (bl = -2 br) and |br| > 2|bl|
// (br = -2 bl); the last two cannot both hold, so each deviation is one
// select of its own (no branch: the warp's lanes take different cases)
template <typename R>
__device__ __forceinline__ void ppm_limit(R& bl, R& br) {
  const bool ext = bl * br >= R(0);
  const R abl = fabs(bl), abr = fabs(br);
  const R nl = abl > R(2) * abr ? R(-2) * br : bl;
  const R nr = abr > R(2) * abl ? R(-2) * bl : br;
  bl = ext ? R(0) : nl;
  br = ext ? R(0) : nr;
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
// fv3_math_check).  FP32: the hardware approximation (rcp.approx.ftz.f32,
// within an ulp) and one Newton-Raphson step, three instructions where the
// IEEE division takes a range check, a branch and several more (the FP32
// stencils are bound by instruction issue); normal x only.
template <typename R>
__device__ __forceinline__ R rcp(R x);
template <>
__device__ __forceinline__ float rcp<float>(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return fmaf(r, fmaf(-x, r, 1.0f), r);
}
template <>
__device__ __forceinline__ double rcp<double>(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// ln(pen / pe) for pen = pe + dp, pe > 0, pen > 0 (kept for the accuracy
// check of fv3_math_check; the column solve uses layer_mean_pressure below).
// With u = dp / (pe + pen),
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

// x as a double.  A float is widened on the integer pipe (the conversion
// instruction runs on the FP64 pipe, which the column solve keeps busy): the
// exponent rebiased from 127 to 1023 and the fraction moved to the top of the
// 52-bit field; subnormal floats normalised with a leading-zero count;
// zeros and infinities keep their sign, a NaN its payload, made quiet.
// Exact, as the conversion is.
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) {
  const unsigned b = __float_as_uint(x), a = b & 0x7fffffffu;
  unsigned hi, lo;
  if (a >= 0x7f800000u) {  // infinity, NaN (quiet)
    hi = 0x7ff00000u | ((a & 0x007fffffu) >> 3) | (a > 0x7f800000u ? 0x00080000u : 0u);
    lo = a << 29;
  } else if (a >= 0x00800000u) {  // normal
    hi = (a >> 3) + (896u << 20);
    lo = a << 29;
  } else if (a == 0u) {
    hi = 0u;
    lo = 0u;
  } else {  // subnormal: a x 2^-149, the leading one moved to bit 23
    const int sh = __clz((int)a) - 8;
    const unsigned f = (a << sh) & 0x007fffffu;
    hi = ((unsigned)(897 - sh) << 20) | (f >> 3);
    lo = f << 29;
  }
  return __hiloint2double((int)(hi | (b & 0x80000000u)), (int)lo);
}

// 1 / a and 1 / b from one reciprocal: r = 1 / (a b), then 1 / a = r b and
// 1 / b = r a (two products instead of a second Newton-refined reciprocal;
// within two ulps for a b in the normal range)
__device__ __forceinline__ void rcp_pair(double a, double b, double& ra, double& rb) {
  const double r = rcp(a * b);
  ra = r * b;
  rb = r * a;
}

// dp / ln(pen / pe) for pen = pe + dp, pe > 0, pen > 0: the pressure that
// splits the gas-law pressure of a layer from its hydrostatic part in the
// column solve.  With u = dp / (pe + pen), ln(pen / pe) = 2 atanh(u), so
// dp / ln(pen / pe) = (pe + pen) / 2 * u / atanh(u), and u / atanh(u) is the
// reciprocal of the series sum_k v^k / (2k + 1) in v = u^2:
//   1 - v/3 - 4v^2/45 - 44v^3/945 - 428v^4/14175 - 10196v^5/467775
//     - 10719068v^6/638512875 - 25865068v^7/1915538625
//     - 5472607916v^8/488462349375 - ...
// (the coefficients of the series division, exact rationals; below they are
// halved, which carries the factor 1/2 through the polynomial without a
// rounding).  For |u| <= 1/8 the terms through v^8 leave a truncation below
// 1e-18 relative, for |u| <= 1/32 (most layers below the top ones) the terms
// through v^4 one below 2e-17 (the next term is 0.022 v^5): one reciprocal
// and a polynomial instead of the logarithm's series and a second
// reciprocal.  The thin upper layers (larger u) divide by the library log.
// The tiers are chosen on the integer bits of |u|.  sum = pe + pen, rsum its
// reciprocal.
__device__ __forceinline__ double layer_mean_pressure(double sum, double rsum, double pen, double pe, double dp) {
  const double u = dp * rsum;
  const long long mag = __double_as_longlong(u) & 0x7fffffffffffffffLL;
  if (mag > 0x3fc0000000000000LL) return dp / log(pen / pe);  // |u| > 1/8
  const double v = u * u;
  double r;
  if (mag <= 0x3fa0000000000000LL) {  // |u| <= 1/32
    r = -214.0 / 14175.0;
  } else {
    r = -2736303958.0 / 488462349375.0;
    r = fma(r, v, -12932534.0 / 1915538625.0);
    r = fma(r, v, -5359534.0 / 638512875.0);
    r = fma(r, v, -5098.0 / 467775.0);
    r = fma(r, v, -214.0 / 14175.0);
  }
  r = fma(r, v, -22.0 / 945.0);
  r = fma(r, v, -2.0 / 45.0);
  r = fma(r, v, -1.0 / 6.0);
  r = fma(r, v, 0.5);
  return sum * r;
}
__device__ __forceinline__ double layer_mean_pressure(double pen, double pe, double dp) {
  const double sum = pe + pen;
  return layer_mean_pressure(sum, rcp(sum), pen, pe, dp);
}

}  // namespace fv3
