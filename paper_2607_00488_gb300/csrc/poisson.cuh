// Per-bin Poisson deviance terms of -2 ln L (eq. logL).
//
// With C = 2 sum_j [n_j - n_j ln n_j + lnGamma(n_j + 1)] (theta independent,
// computed once per data set in FP64),
//   -2 ln L = C + 2 sum_j t_j,   t_j = mu_j - n_j + n_j ln(n_j / mu_j)
// which is eq. logL term by term (0 ln 0 = 0).  t_j >= 0 and is small where
// the model fits, so summing t instead of mu - n ln mu avoids the large
// cancelling magnitudes of the direct form.
#pragma once

#include <cuda_runtime.h>

namespace srw {

// FP64 term (single-point path).  mu < 0, or mu == 0 with n > 0, gives +inf.
__device__ __forceinline__ double poisson_term_f64(double mu, double n) {
  if (mu < 0.0) return __longlong_as_double(0x7ff0000000000000LL);
  if (n == 0.0) return mu;
  if (mu == 0.0) return __longlong_as_double(0x7ff0000000000000LL);
  return mu - n + n * log(n / mu);
}

// FP32 term of the tensor-core epilogue, branch-free and without per-element
// special cases.  With v = (n - mu)/(n + mu), ln(n/mu) = 2 atanh(v), hence
//   t = (n - mu) v + 2 n (v^3/3 + v^5/5 + v^7/7 + v^9/9 + ...)
// which has no cancellation; for |v| < 0.1 the truncation after v^9 is below
// 1e-10 relative.  Larger |v| uses the direct form, whose cancellation is
// then at most a factor ~10.  Both forms are evaluated and selected, so lanes
// holding different parameter points never diverge; the quotients use the
// fast division (at most 2 ulp).  The bin constants carry n = 0 for masked
// bins (their term is then finite and the caller multiplies it by the 0/1
// mask).  The log argument is floored at 1e-30: for n = 0 the term is
// 0 * ln(1e-30) = 0, so t = mu (mu = 0 included, where n / mu is NaN and the
// floor applies); mu = 0 with n > 0 gives +inf through ln(inf).  mu < 0 is
// left to the caller (it tracks the smallest mu of the active bins).
__device__ __forceinline__ float poisson_term_f32_tc(float mu, float n) {
  const float d = n - mu, s = n + mu;
  const float v = __fdividef(d, s);
  const float v2 = v * v;
  float p = fmaf(v2, 1.f / 9.f, 1.f / 7.f);
  p = fmaf(v2, p, 1.f / 5.f);
  p = fmaf(v2, p, 1.f / 3.f);
  const float ts = fmaf(d, v, 2.f * n * v * v2 * p);
  const float tl = fmaf(n, logf(fmaxf(__fdividef(n, mu), 1e-30f)), -d);  // mu - n = -d exactly
  return fabsf(v) < 0.1f ? ts : tl;
}

// The same term from dm = mu - n (and n), for callers that form mu - n
// directly: an FP32 mu of 1e5 counts carries an absolute rounding error of
// ~6e-3, while mu - n near the data is a few hundred, so its FP32 value is
// ~1e3 times more precise and the series branch then loses nothing to it.
// The log branch (far from the data) takes mu - n of the same rounded mu that
// enters the logarithm: then mu's rounding error e enters t only as
// (1 - n/mu) e, as in the exact expression (dt/dmu = 1 - n/mu); with the
// unrounded dm it would enter as -(n/mu) e, about e itself.
// Same branches, floor and special cases as poisson_term_f32_tc.
__device__ __forceinline__ float poisson_term_f32_dm(float dm, float n) {
  const float mu = n + dm, s = n + mu;
  const float v = __fdividef(-dm, s);
  const float v2 = v * v;
  float p = fmaf(v2, 1.f / 9.f, 1.f / 7.f);
  p = fmaf(v2, p, 1.f / 5.f);
  p = fmaf(v2, p, 1.f / 3.f);
  const float ts = fmaf(-dm, v, 2.f * n * v * v2 * p);
  const float tl = fmaf(n, logf(fmaxf(__fdividef(n, mu), 1e-30f)), mu - n);
  return fabsf(v) < 0.1f ? ts : tl;
}

}  // namespace srw
