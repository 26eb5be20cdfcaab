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

// FP32 term for the batched epilogues, accurate to a few ulp of t.
// With v = (n - mu)/(n + mu), ln(n/mu) = 2 atanh(v), hence
//   t = (n - mu) v + 2 n (v^3/3 + v^5/5 + v^7/7 + v^9/9 + ...)
// which has no cancellation; for |v| < 0.1 the truncation after v^9 is
// below 1e-10 relative.  Larger |v| uses the direct form, whose
// cancellation is then at most a factor ~10.
__device__ __forceinline__ float poisson_term_f32(float mu, float n) {
  if (mu < 0.f) return __int_as_float(0x7f800000);
  if (n == 0.f) return mu;
  if (mu == 0.f) return __int_as_float(0x7f800000);
  const float d = n - mu, s = n + mu;
  const float v = d / s;
  if (fabsf(v) < 0.1f) {
    const float v2 = v * v;
    float p = fmaf(v2, 1.f / 9.f, 1.f / 7.f);
    p = fmaf(v2, p, 1.f / 5.f);
    p = fmaf(v2, p, 1.f / 3.f);
    return fmaf(d, v, 2.f * n * v * v2 * p);
  }
  return (mu - n) + n * logf(n / mu);
}

// Branch-free variant for the tensor-core epilogue, where neighbouring lanes
// hold different parameter points: both forms are evaluated and selected, so
// lanes never diverge.  The quotients use the fast division (at most 2 ulp),
// which keeps the relative error of t at a few ulp in the series range and
// ~1e-7 relative in the log range.
__device__ __forceinline__ float poisson_term_f32_sel(float mu, float n) {
  const float d = n - mu, s = n + mu;
  const float v = __fdividef(d, s);
  const float v2 = v * v;
  float p = fmaf(v2, 1.f / 9.f, 1.f / 7.f);
  p = fmaf(v2, p, 1.f / 5.f);
  p = fmaf(v2, p, 1.f / 3.f);
  const float ts = fmaf(d, v, 2.f * n * v * v2 * p);
  const float tl = (mu - n) + n * logf(__fdividef(n, mu));
  float t = fabsf(v) < 0.1f ? ts : tl;
  t = n == 0.f ? mu : t;
  return (mu < 0.f || (mu == 0.f && n > 0.f)) ? __int_as_float(0x7f800000) : t;
}

// The tensor-core epilogue's term, branch-free and without per-element special
// cases.  The bin constants carry n = 0 for masked bins (their term is then
// finite and the caller multiplies it by the 0/1 mask).  The log argument is
// floored at 1e-30: for n = 0 the term is 0 * ln(1e-30) = 0, so t = mu
// (mu = 0 included, where n / mu is NaN and the floor applies); mu = 0 with
// n > 0 gives +inf through ln(inf).  mu < 0 is left to the caller (it tracks
// the smallest mu of the active bins).  Elsewhere identical to
// poisson_term_f32_sel.
__device__ __forceinline__ float poisson_term_f32_tc(float mu, float n) {
  const float d = n - mu, s = n + mu;
  const float v = __fdividef(d, s);
  const float v2 = v * v;
  float p = fmaf(v2, 1.f / 9.f, 1.f / 7.f);
  p = fmaf(v2, p, 1.f / 5.f);
  p = fmaf(v2, p, 1.f / 3.f);
  const float ts = fmaf(d, v, 2.f * n * v * v2 * p);
  const float tl = (mu - n) + n * logf(fmaxf(__fdividef(n, mu), 1e-30f));
  return fabsf(v) < 0.1f ? ts : tl;
}

}  // namespace srw
