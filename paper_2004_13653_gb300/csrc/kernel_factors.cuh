// One factor k(s) of each Table 1 product kernel, without its constant, for
// the FP32 paths; and an error-free running sum.
#pragma once
#include "kde_internal.cuh"

namespace kde {

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// cos(pi/2 * s) from its Taylor series in s^2 (terms through s^14; the
// remainder on |s| <= 1 is below 7e-11).
constexpr double kHalfPi = 1.57079632679489661923;
constexpr double cos_coef(int k) {
  double c = 1.0;
  for (int i = 1; i <= 2 * k; ++i) c = c * kHalfPi / (double)i;
  return (k & 1) ? -c : c;
}
__device__ __forceinline__ float cos_half_pi(float s) {
  const float x = s * s;
  float r = (float)cos_coef(7);
  r = fmaf(r, x, (float)cos_coef(6));
  r = fmaf(r, x, (float)cos_coef(5));
  r = fmaf(r, x, (float)cos_coef(4));
  r = fmaf(r, x, (float)cos_coef(3));
  r = fmaf(r, x, (float)cos_coef(2));
  r = fmaf(r, x, (float)cos_coef(1));
  r = fmaf(r, x, (float)cos_coef(0));
  return r;
}

// One kernel factor without its constant.  d is the offset in units of 1/sigma:
// bandwidths for the compact kernels, h sqrt(2 ln 2) for the Gaussian.
template <int KID>
__device__ __forceinline__ float kfactor(float d) {
  if constexpr (KID == KDE_GAUSSIAN) {
    return ex2_approx(-d * d);
  } else if constexpr (KID == KDE_UNIFORM) {
    return fabsf(d) <= 1.0f ? 1.0f : 0.0f;
  } else if constexpr (KID == KDE_TRIANGULAR) {
    return fmaxf(1.0f - fabsf(d), 0.0f);
  } else if constexpr (KID == KDE_EPANECHNIKOV) {
    return fmaxf(fmaf(-d, d, 1.0f), 0.0f);
  } else if constexpr (KID == KDE_QUARTIC) {
    const float t = fmaxf(fmaf(-d, d, 1.0f), 0.0f);
    return t * t;
  } else if constexpr (KID == KDE_TRIWEIGHT) {
    const float t = fmaxf(fmaf(-d, d, 1.0f), 0.0f);
    return t * t * t;
  } else if constexpr (KID == KDE_TRICUBE) {
    const float a = fabsf(d);
    const float t = fmaxf(fmaf(-(a * a), a, 1.0f), 0.0f);
    return t * t * t;
  } else {  // KDE_COSINE
    return fabsf(d) <= 1.0f ? fmaxf(cos_half_pi(d), 0.0f) : 0.0f;
  }
}

// The radial variant of a Table 1 kernel (kernel id 8 + KID) as a function of
// q = |u|^2 (offsets in bandwidths), without its constant: the Table 1 profile
// of r = sqrt(q) on the unit disk.
template <int KID>
__device__ __forceinline__ float kradial(float q) {
  if constexpr (KID == KDE_UNIFORM) {
    return q <= 1.0f ? 1.0f : 0.0f;
  } else if constexpr (KID == KDE_TRIANGULAR) {
    return fmaxf(1.0f - sqrtf(q), 0.0f);
  } else if constexpr (KID == KDE_EPANECHNIKOV) {
    return fmaxf(1.0f - q, 0.0f);
  } else if constexpr (KID == KDE_QUARTIC) {
    const float t = fmaxf(1.0f - q, 0.0f);
    return t * t;
  } else if constexpr (KID == KDE_TRIWEIGHT) {
    const float t = fmaxf(1.0f - q, 0.0f);
    return t * t * t;
  } else if constexpr (KID == KDE_TRICUBE) {
    const float t = fmaxf(fmaf(-q, sqrtf(q), 1.0f), 0.0f);
    return t * t * t;
  } else {  // KDE_COSINE: cos(pi/2 r), Taylor series in r^2 = q
    return q <= 1.0f ? fmaxf(cos_half_pi(sqrtf(q)), 0.0f) : 0.0f;
  }
}

__device__ __forceinline__ void two_sum_acc(float2& run, float v) {
  const float s = run.x + v;
  const float bb = s - run.x;
  const float e = (run.x - (s - bb)) + (v - bb);
  run.x = s;
  run.y += e;
}

}  // namespace kde
