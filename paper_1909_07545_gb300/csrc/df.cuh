// df.cuh -- float-float arithmetic for the kernels whose FP32 rounding the
// warping would amplify: the trajectory field, the calibration field, the
// pre-rotation and the image pyramid.  They run once per pose or once per
// frame, so their cost does not matter; what matters is that each stored
// result is its exact value rounded once to float.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2
// (about 48 significant bits).  Every step is FP32 arithmetic:
//   two_sum       Knuth's error-free sum (TAOCP vol. 2, 4.2.2)
//   fast_two_sum  Dekker's error-free sum for |a| >= |b| (Dekker 1971)
//   two_prod      Dekker's error-free product, in its FMA form
//   dd_add, dd_mul, dd_div, dd_sqrt
//                 the double-word algorithms of Hida, Li and Bailey
//                 ("Algorithms for quad-double precision floating point
//                 arithmetic", 2001), restated for float words
//   dd_sincos     the Taylor series of sin and cos, Horner in x^2 with
//                 coefficients 1/n! that the compiler evaluates in double
//   dd_atan2      atan2f, then one Newton correction by the tangent of the
//                 residual angle from dd_sincos
// The rounding-explicit intrinsics keep the compiler from contracting or
// reordering the error-free steps.
#pragma once

#include <cuda_runtime.h>

namespace fs {

struct df {
  float hi, lo;
};

// Host: the float-float nearest to a double (the constants of a kernel).
inline df df_from_double(double v) {
  const float hi = (float)v;
  return df{hi, (float)(v - (double)hi)};
}

__device__ __forceinline__ df df_f(float a) { return df{a, 0.f}; }

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df{s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return df{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df dd_neg(df a) { return df{-a.hi, -a.lo}; }

__device__ __forceinline__ df dd_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  const df t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df dd_sub(df a, df b) { return dd_add(a, dd_neg(b)); }

__device__ __forceinline__ df dd_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ df dd_mul_f(df a, float b) {
  df p = two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

// a / b: three quotient words from the residuals a - q b.
__device__ __forceinline__ df dd_div(df a, df b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  df r = dd_sub(a, dd_mul_f(b, q1));
  const float q2 = __fdiv_rn(r.hi, b.hi);
  r = dd_sub(r, dd_mul_f(b, q2));
  const float q3 = __fdiv_rn(r.hi, b.hi);
  return dd_add(fast_two_sum(q1, q2), df_f(q3));
}

__device__ __forceinline__ df dd_div_f(df a, float b) { return dd_div(a, df_f(b)); }

// sqrt(a) for a >= 0 (0 for a <= 0): the float root corrected by one
// Newton step x + (a - x^2) / (2 x).
__device__ __forceinline__ df dd_sqrt(df a) {
  if (!(a.hi > 0.f)) return df{0.f, 0.f};
  const float x = __fsqrt_rn(a.hi);
  const df r = dd_sub(a, two_prod(x, x));
  return fast_two_sum(x, __fdiv_rn(r.hi, __fmul_rn(2.f, x)));
}

// ------------------------------------------------------------ sin, cos

constexpr int kTaylorTerms = 17;   // k = 0..16: remainder below 1e-19 for |x| <= pi

// (-1)^k / (2k + first)! as float-float words, evaluated by the compiler.
struct DfSeries {
  float hi[kTaylorTerms], lo[kTaylorTerms];
};

constexpr DfSeries taylor_series(int first) {
  DfSeries c{};
  double f = 1.0;                                   // 1 / first!
  for (int n = 2; n <= first; ++n) f /= n;
  for (int k = 0; k < kTaylorTerms; ++k) {
    const double v = (k % 2 == 0) ? f : -f;
    c.hi[k] = (float)v;
    c.lo[k] = (float)(v - (double)c.hi[k]);
    const int n = 2 * k + first;                    // next: 1 / (n + 2)!
    f = f / ((double)(n + 1) * (double)(n + 2));
  }
  return c;
}

static __constant__ const DfSeries kCosSeries = taylor_series(0);
static __constant__ const DfSeries kSinSeries = taylor_series(1);

// sin and cos of x, |x| <= pi.  Terms k < n: for |x| <= 1.8 (every angle of
// a lens up to 206 degrees) the first omitted term is below 2e-18 at n = 12,
// so 12 are taken there and all 17 beyond.
__device__ __forceinline__ void dd_sincos(df x, df& s, df& c) {
  const df y = dd_mul(x, x);
  const int n = fabsf(x.hi) <= 1.8f ? 12 : kTaylorTerms;
  df ps = df{kSinSeries.hi[n - 1], kSinSeries.lo[n - 1]};
  df pc = df{kCosSeries.hi[n - 1], kCosSeries.lo[n - 1]};
#pragma unroll 1
  for (int k = n - 2; k >= 0; --k) {
    ps = dd_add(dd_mul(ps, y), df{kSinSeries.hi[k], kSinSeries.lo[k]});
    pc = dd_add(dd_mul(pc, y), df{kCosSeries.hi[k], kCosSeries.lo[k]});
  }
  s = dd_mul(ps, x);
  c = pc;
}

// atan2(y, x) for y >= 0 (angles in [0, pi]).  With t0 = atan2f, the
// residual angle d = theta - t0 has tan d = (y cos t0 - x sin t0) /
// (x cos t0 + y sin t0); |d| is a few float ulps, so d = tan d up to d^3/3.
__device__ __forceinline__ df dd_atan2(df y, df x) {
  const float t0 = atan2f(y.hi, x.hi);
  df s, c;
  dd_sincos(df_f(t0), s, c);
  const df num = dd_sub(dd_mul(y, c), dd_mul(x, s));
  const df den = dd_add(dd_mul(x, c), dd_mul(y, s));
  if (!(den.hi > 0.f)) return df_f(t0);
  return dd_add(df_f(t0), dd_div(num, den));
}

// Floor and fraction of a float-float position: d = fl + frac, fl an
// integer-valued float, frac in [0, 1).
__device__ __forceinline__ void dd_floor_frac(df d, float& fl, df& frac) {
  fl = floorf(d.hi);
  frac = two_sum(__fsub_rn(d.hi, fl), d.lo);        // d.hi - fl is exact
  if (frac.hi < 0.f) {
    fl = __fsub_rn(fl, 1.f);
    frac = dd_add(frac, df_f(1.f));
  } else if (frac.hi >= 1.f) {
    fl = __fadd_rn(fl, 1.f);
    frac = dd_sub(frac, df_f(1.f));
  }
}

}  // namespace fs
