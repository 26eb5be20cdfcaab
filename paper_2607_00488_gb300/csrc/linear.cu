// Exact rank-8 evaluation of the likelihood (srw_loglik_linear in srw.h).
//
// The recoil spectrum is a polynomial in the shifted couplings and mu_hat^2
// (Sec. II: eqs. sm_cross_section, g_tilde, xs_mm, xs_total), so the weighted
// true spectrum is W(theta) = sum_b c_b(theta) shat_b with eight fixed
// coefficient spectra, and the fold of eq. matrix_reweight is linear in them:
//
//   mu(theta) = R W_ref + b + M (c(theta) - c_ref),   M = R shat^T  [n_rec][8]
//
// M is computed once in FP64 (per rec bin, eight dot products of length n_t).
// Per point the kernel forms the eight coefficients, then per rec bin
// Delta = sum_b M_jb (c_b - c_ref,b) (8 FMAs), mu = mu_ref + b + Delta, and the
// Poisson deviance of eq. logL from d = n - mu and s = n + mu (the same series
// / log forms as the batched epilogues), accumulated in double-float.  The
// same linearity gives the gradient:
//   d(-2 ln L)/d theta_k = 2 sum_b (d c_b / d theta_k) sum_j M_jb (1 - n_j/mu_j).
// Four lanes per point, each on every fourth rec bin; the per-bin constants
// (M row, n - mu_ref - b, n + mu_ref + b, n) are staged through shared memory
// in chunks.

#include "dfloat.cuh"
#include "srw_internal.h"

namespace srw {
namespace {

constexpr int kLinThreads = 256;  // 64 points x 4 lanes
constexpr int kLinChunk = 1024;  // rec bins per shared-memory chunk (48 KB)

// M_jb = sum_i R_ji shat_b,i with shat_b,i = B_b,i E_SM,i / S_SM,i (FP64); one
// block per rec bin.
__global__ void linear_m_kernel(const float* __restrict__ R, int ld, int n_t, const double* __restrict__ basis,
                                const double* __restrict__ ssm, const double* __restrict__ esm, double* __restrict__ M) {
  __shared__ double red[kNB][32];
  const int j = blockIdx.x;
  double acc[kNB];
#pragma unroll
  for (int b = 0; b < kNB; ++b) acc[b] = 0.0;
  for (int i = threadIdx.x; i < n_t; i += blockDim.x) {
    const double r = (double)R[(size_t)j * ld + i];
    if (r == 0.0) continue;
    const double sm = ssm[i], e = esm[i];
#pragma unroll
    for (int b = 0; b < kNB; ++b) {
      const double sh = sm != 0.0 ? basis[(size_t)b * n_t + i] * (e / sm) : (b == 6 ? e : 0.0);
      acc[b] += r * sh;
    }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int b = 0; b < kNB; ++b) {
    double v = acc[b];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[b][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < kNB) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[threadIdx.x][k];
    M[(size_t)j * kNB + threadIdx.x] = t;
  }
}

// Per-bin constants: {M_j0..3}, {M_j4..7}, {n - mu_ref - b, n + mu_ref + b, n (or -1: masked), 0},
// and for the profiled evaluation {mu_ref, b, n (or -1), 0}.
__global__ void linear_consts_kernel(const double* __restrict__ M, const double* __restrict__ n64,
                                     const double* __restrict__ bref64, const double* __restrict__ muref,
                                     const unsigned char* __restrict__ mask, int n_rec, float4* __restrict__ out,
                                     float4* __restrict__ outp) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_rec) return;
  const double* m = M + (size_t)j * kNB;
  const double n = n64[j], base = bref64[j];
  const bool on = mask == nullptr || mask[j] != 0;
  out[3 * j] = make_float4((float)m[0], (float)m[1], (float)m[2], (float)m[3]);
  out[3 * j + 1] = make_float4((float)m[4], (float)m[5], (float)m[6], (float)m[7]);
  const double nn = on ? n : 0.0;  // masked bins: n = 0 keeps their (multiplied-out) term finite
  out[3 * j + 2] = make_float4((float)(nn - base), (float)(nn + base), (float)nn, on ? 1.f : 0.f);
  outp[j] = make_float4((float)muref[j], (float)(base - muref[j]), on ? (float)n : -1.f, 0.f);
}

struct Couplings {
  float gle, gre, glt, grt, mu;
};

__device__ __forceinline__ void deviations(const float* th, dfloat s, const CoefRef& ref, float* c, Couplings& g) {
  const dfloat gle = df_add(df_add(dfloat{0.5f, 0.f}, s), th[0]), gre = df_add(s, th[1]);
  const dfloat glt = df_add(df_add(dfloat{-0.5f, 0.f}, s), th[2]), grt = df_add(s, th[3]);
  const dfloat x = df_mul(gle, gre), y = df_mul(glt, grt);
  const dfloat v[kNB] = {df_mul(gle, gle), df_mul(gre, gre), {-x.hi, -x.lo}, df_mul(glt, glt),
                         df_mul(grt, grt), {-y.hi, -y.lo}, {1.f, 0.f}, two_prod(th[4], th[4])};
#pragma unroll
  for (int b = 0; b < kNB; ++b) {
    const dfloat d = df_add(v[b], dfloat{-ref.hi[b], -ref.lo[b]});
    c[b] = d.hi + d.lo;
  }
  g = Couplings{gle.hi + gle.lo, gre.hi + gre.lo, glt.hi + glt.lo, grt.hi + grt.lo, th[4]};
}

// Deviance t = mu - n + n ln(n / mu) from d = n - mu, s = n + mu (n >= 0),
// branch-free (neighbouring lanes hold different bins and points): the atanh
// series where |d| < 0.1 s, the direct form otherwise; t = mu where n = 0;
// +inf where mu <= 0 with data.
__device__ __forceinline__ float deviance_ds(float d, float s, float n) {
  const float mu = n - d;
  const float v = __fdividef(d, s);
  const float v2 = v * v;
  float p = fmaf(v2, 1.f / 9.f, 1.f / 7.f);
  p = fmaf(v2, p, 1.f / 5.f);
  p = fmaf(v2, p, 1.f / 3.f);
  const float ts = fmaf(d, v, 2.f * n * v * v2 * p);
  const float tl = -d + n * logf(__fdividef(n, mu));
  float t = fabsf(v) < 0.1f ? ts : tl;
  t = n == 0.f ? mu : t;
  return (mu < 0.f || (mu == 0.f && n > 0.f)) ? __int_as_float(0x7f800000) : t;
}

// The evaluator's term from d = n - mu and s = n + mu, without per-element
// special cases: the log argument is floored at 1e-30, so n = 0 gives t = mu
// (also for mu = 0) and mu = 0 < n gives +inf; mu < 0 is left to the caller.
__device__ __forceinline__ float deviance_fast(float d, float s, float n) {
  const float mu = n - d;
  const float v = __fdividef(d, s);
  const float v2 = v * v;
  float p = fmaf(v2, 1.f / 9.f, 1.f / 7.f);
  p = fmaf(v2, p, 1.f / 5.f);
  p = fmaf(v2, p, 1.f / 3.f);
  const float ts = fmaf(d, v, 2.f * n * v * v2 * p);
  const float tl = -d + n * logf(fmaxf(__fdividef(n, mu), 1e-30f));
  return fabsf(v) < 0.1f ? ts : tl;
}

// Four lanes per point (adjacent lanes), each on every fourth bin; their sums
// are combined with shuffles.
template <bool GRAD>
__global__ void __launch_bounds__(kLinThreads)
linear_loglik_kernel(const float* __restrict__ theta, int P, dfloat sin2w, CoefRef cref,
                     const float4* __restrict__ consts, int n_rec, const double* __restrict__ c_data,
                     double* __restrict__ out, double* __restrict__ grad, unsigned* __restrict__ status) {
  __shared__ float4 sc[3 * kLinChunk];
  const int quarter = threadIdx.x & 3;
  const int p = blockIdx.x * (kLinThreads / 4) + (threadIdx.x >> 2);
  const bool on = p < P;
  float c[kNB] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  Couplings g{0.f, 0.f, 0.f, 0.f, 0.f};
  if (on) deviations(theta + (size_t)p * 5, sin2w, cref, c, g);
  dfloat acc = {0.f, 0.f};
  bool infinite = false;
  float mneg = 0.f;  // smallest mu of the active bins (below 0: outside the domain)
  float gb[kNB] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int j0 = 0; j0 < n_rec; j0 += kLinChunk) {
    const int cnt = min(kLinChunk, n_rec - j0);
    __syncthreads();
    for (int k = threadIdx.x; k < 3 * cnt; k += blockDim.x) sc[k] = consts[3 * (size_t)j0 + k];
    __syncthreads();
    float ts = 0.f;
    int n_acc = 0;
#pragma unroll 4
    for (int j = quarter; j < cnt; j += 4) {
      const float4 m0 = sc[3 * j], m1 = sc[3 * j + 1], q = sc[3 * j + 2];  // q.w: 1, or 0 where masked
      float dl = m0.x * c[0];
      dl = fmaf(m0.y, c[1], dl);
      dl = fmaf(m0.z, c[2], dl);
      dl = fmaf(m0.w, c[3], dl);
      dl = fmaf(m1.x, c[4], dl);
      dl = fmaf(m1.y, c[5], dl);
      dl = fmaf(m1.z, c[6], dl);
      dl = fmaf(m1.w, c[7], dl);
      const float d = q.x - dl, s = q.y + dl;
      ts = fmaf(deviance_fast(d, s, q.z), q.w, ts);
      mneg = fminf(mneg, (q.z - d) * q.w);
      if (GRAD) {
        const float r = q.w > 0.f ? 1.f - __fdividef(q.z, q.z - d) : 0.f;  // 1 - n / mu
        gb[0] = fmaf(m0.x, r, gb[0]);
        gb[1] = fmaf(m0.y, r, gb[1]);
        gb[2] = fmaf(m0.z, r, gb[2]);
        gb[3] = fmaf(m0.w, r, gb[3]);
        gb[4] = fmaf(m1.x, r, gb[4]);
        gb[5] = fmaf(m1.y, r, gb[5]);
        gb[7] = fmaf(m1.w, r, gb[7]);
      }
      if (++n_acc == 16) {
        if (isinf(ts)) infinite = true;
        else acc = df_add(acc, ts);
        ts = 0.f;
        n_acc = 0;
      }
    }
    if (isinf(ts)) infinite = true;
    else acc = df_add(acc, ts);
  }
  if (mneg < 0.f) infinite = true;
  // combine the four lanes of each point
#pragma unroll
  for (int o = 1; o <= 2; o <<= 1) {
    acc = df_add(acc, df_shfl_xor(acc, o));
    infinite = __shfl_xor_sync(0xffffffffu, (int)infinite, o) || infinite;
    if (GRAD)
#pragma unroll
      for (int b = 0; b < kNB; ++b) gb[b] += __shfl_xor_sync(0xffffffffu, gb[b], o);
  }
  if (!on || quarter != 0) return;
  const double v = infinite ? __longlong_as_double(0x7ff0000000000000LL)
                            : 2.0 * ((double)acc.hi + (double)acc.lo) + *c_data;
  if (infinite) atomicOr(status, kStatusDomain);
  out[p] = v;
  if (GRAD) {
    double* gp = grad + (size_t)p * 5;
    gp[0] = 2.0 * (2.0 * (double)g.gle * gb[0] - (double)g.gre * gb[2]);
    gp[1] = 2.0 * (2.0 * (double)g.gre * gb[1] - (double)g.gle * gb[2]);
    gp[2] = 2.0 * (2.0 * (double)g.glt * gb[3] - (double)g.grt * gb[5]);
    gp[3] = 2.0 * (2.0 * (double)g.grt * gb[4] - (double)g.glt * gb[5]);
    gp[4] = 2.0 * (2.0 * (double)g.mu * gb[7]);
  }
}

constexpr int kNewton = 8;  // Newton steps for the normalisation (quadratic convergence from alpha = 1)

// Profiled evaluation: min over alpha >= 0 of -2 ln L(alpha mu_sig + b) plus
// ((alpha - 1)/sigma)^2 when sigma > 0, with mu_sig = mu_ref + M (c - c_ref).
// Newton on the convex objective, g = 2 sum s (1 - n/mu) + 2 (alpha - 1)/sigma^2,
// h = 2 sum n s^2 / mu^2 + 2 / sigma^2, each step one pass over the bins
// (mu_sig recomputed from the eight coefficients); then the deviance at alpha.
__global__ void __launch_bounds__(kLinThreads)
linear_profiled_kernel(const float* __restrict__ theta, int P, dfloat sin2w, CoefRef cref,
                       const float4* __restrict__ consts, const float4* __restrict__ constp, int n_rec,
                       float inv_var, const double* __restrict__ c_data, double* __restrict__ out,
                       double* __restrict__ alpha_out, unsigned* __restrict__ status) {
  __shared__ float4 sc[3 * kLinChunk];
  const int quarter = threadIdx.x & 3;
  const int p = blockIdx.x * (kLinThreads / 4) + (threadIdx.x >> 2);
  const bool on = p < P;
  float c[kNB] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  Couplings g{0.f, 0.f, 0.f, 0.f, 0.f};
  if (on) deviations(theta + (size_t)p * 5, sin2w, cref, c, g);
  auto stage = [&](int j0, int cnt) {
    __syncthreads();
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
      sc[3 * k] = consts[3 * (size_t)(j0 + k)];
      sc[3 * k + 1] = consts[3 * (size_t)(j0 + k) + 1];
      sc[3 * k + 2] = constp[j0 + k];
    }
    __syncthreads();
  };
  auto signal = [&](int j) {
    const float4 m0 = sc[3 * j], m1 = sc[3 * j + 1];
    float dl = m0.x * c[0];
    dl = fmaf(m0.y, c[1], dl);
    dl = fmaf(m0.z, c[2], dl);
    dl = fmaf(m0.w, c[3], dl);
    dl = fmaf(m1.x, c[4], dl);
    dl = fmaf(m1.y, c[5], dl);
    dl = fmaf(m1.z, c[6], dl);
    dl = fmaf(m1.w, c[7], dl);
    return sc[3 * j + 2].x + dl;
  };
  float alpha = 1.f;
  for (int it = 0; it < kNewton; ++it) {
    float G = 0.f, H = 0.f;
    for (int j0 = 0; j0 < n_rec; j0 += kLinChunk) {
      const int cnt = min(kLinChunk, n_rec - j0);
      stage(j0, cnt);
      for (int j = quarter; j < cnt; j += 4) {
        const float4 q = sc[3 * j + 2];
        const float s = signal(j);
        const float mu = fmaf(alpha, s, q.y);
        const bool live = q.z >= 0.f && mu > 0.f;
        const float r = live ? __fdividef(q.z, mu) : 0.f;  // n / mu
        G += q.z >= 0.f ? s * (1.f - r) : 0.f;
        H += live ? r * s * s / mu : 0.f;
      }
    }
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
      G += __shfl_xor_sync(0xffffffffu, G, o);
      H += __shfl_xor_sync(0xffffffffu, H, o);
    }
    const float gg = 2.f * G + 2.f * (alpha - 1.f) * inv_var, hh = 2.f * H + 2.f * inv_var;
    float next = hh > 0.f ? alpha - gg / hh : (gg > 0.f ? 0.f : alpha);
    alpha = fmaxf(next, 0.f);
  }
  dfloat acc = {0.f, 0.f};
  bool infinite = false;
  for (int j0 = 0; j0 < n_rec; j0 += kLinChunk) {
    const int cnt = min(kLinChunk, n_rec - j0);
    stage(j0, cnt);
    float ts = 0.f;
    int n_acc = 0;
    for (int j = quarter; j < cnt; j += 4) {
      const float4 q = sc[3 * j + 2];
      const float mu = fmaf(alpha, signal(j), q.y);
      const float t = deviance_ds(q.z - mu, q.z + mu, q.z);
      ts += q.z >= 0.f ? t : 0.f;
      if (++n_acc == 16) {
        if (isinf(ts)) infinite = true;
        else acc = df_add(acc, ts);
        ts = 0.f;
        n_acc = 0;
      }
    }
    if (isinf(ts)) infinite = true;
    else acc = df_add(acc, ts);
  }
#pragma unroll
  for (int o = 1; o <= 2; o <<= 1) {
    acc = df_add(acc, df_shfl_xor(acc, o));
    infinite = __shfl_xor_sync(0xffffffffu, (int)infinite, o) || infinite;
  }
  if (!on || quarter != 0) return;
  const double pull = (double)inv_var * ((double)alpha - 1.0) * ((double)alpha - 1.0);
  const double v = infinite ? __longlong_as_double(0x7ff0000000000000LL)
                            : 2.0 * ((double)acc.hi + (double)acc.lo) + *c_data + pull;
  if (infinite) atomicOr(status, kStatusDomain);
  out[p] = v;
  if (alpha_out) alpha_out[p] = alpha;
}

}  // namespace

cudaError_t launch_linear_profiled(const srw_ctx* h, const float* theta, int P, double sigma_alpha, double* out,
                                   double* alpha, cudaStream_t s) {
  const int grid = (P + kLinThreads / 4 - 1) / (kLinThreads / 4);
  const float inv_var = sigma_alpha > 0.0 ? (float)(1.0 / (sigma_alpha * sigma_alpha)) : 0.f;
  linear_profiled_kernel<<<grid, kLinThreads, 0, s>>>(theta, P, df_from_double(h->sin2w), h->cref, h->d_lin,
                                                       h->d_linp, h->n_rec, inv_var, h->d_cdata, out, alpha,
                                                       h->d_status);
  return launch_result();
}

cudaError_t launch_linear_m(srw_ctx* h, cudaStream_t s) {
  linear_m_kernel<<<h->n_rec, 256, 0, s>>>(h->d_R, h->ld_r, h->n_t, h->d_basis, h->d_ssm64, h->d_esm64, h->d_linM);
  return launch_result();
}

cudaError_t launch_linear_consts(srw_ctx* h, cudaStream_t s) {
  linear_consts_kernel<<<(h->n_rec + 255) / 256, 256, 0, s>>>(h->d_linM, h->d_n64, h->d_bref64, h->d_muref64, h->d_mask,
                                                             h->n_rec, h->d_lin, h->d_linp);
  return launch_result();
}

cudaError_t launch_linear_loglik(const srw_ctx* h, const float* theta, int P, double* out, double* grad,
                                 cudaStream_t s) {
  const int grid = (P + kLinThreads / 4 - 1) / (kLinThreads / 4);
  if (grad)
    linear_loglik_kernel<true><<<grid, kLinThreads, 0, s>>>(theta, P, df_from_double(h->sin2w), h->cref, h->d_lin,
                                                            h->n_rec, h->d_cdata, out, grad, h->d_status);
  else
    linear_loglik_kernel<false><<<grid, kLinThreads, 0, s>>>(theta, P, df_from_double(h->sin2w), h->cref, h->d_lin,
                                                             h->n_rec, h->d_cdata, out, nullptr, h->d_status);
  return launch_result();
}

}  // namespace srw
