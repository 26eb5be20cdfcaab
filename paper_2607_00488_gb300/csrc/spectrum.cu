// Recoil-spectrum kernels.
//
// The recoil spectrum of one true-recoil bin i is (Sec. III.A, eq. fT, with
// the cross sections of Sec. II, eqs. sm_cross_section, g_tilde, xs_mm,
// xs_total), in units of sigma0 = 2 G_F^2 m_e / pi:
//
//   S_i = sum_nodes w_n sum_alpha P_alpha(E_n) int_a^b dT [ gL_a^2
//           + gR_a^2 (1 - T/E)^2 - gL_a gR_a m_e T / E^2 ]
//       + kappa mu_hat^2 sum_nodes w_n int_a^b dT (1/T - 1/E)
//
// with a = max(T_lo, t_min), b = min(T_hi, T_max(E_n)) and
// T_max(E) = 2 E^2 / (m_e + 2E).  The integrals are closed forms:
//   int 1            = b - a                       (I0)
//   int T            = (b - a)(a + b) / 2          (I1)
//   int (1 - T/E)^2  = (b - a)(u^2 + u v + v^2)/3, u = 1 - a/E, v = 1 - b/E
//   int (1/T - 1/E)  = log(b/a) - (b - a)/E
// (the (1 - T/E)^2 form avoids the cancellation of expanding the cube).
//
// Nodes are sorted by T_max descending, so the nodes that can reach bin i
// are a prefix [0, bin_count[i]).

#include <cooperative_groups.h>

#include "dfloat.cuh"
#include "srw_internal.h"

namespace cg = cooperative_groups;

namespace srw {
namespace {

constexpr int kBasisThreads = 256;
constexpr int kSpecThreads = 256;
constexpr int kSpecCluster = 4;   // blocks per bin group (thread-block cluster)
constexpr int kBinsPerBlock = 8;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// G0: FP64 coefficient spectra B[8][n_t] (create time, theta independent).
// One block per recoil bin; threads stride over the contributing nodes;
// fixed-order block reduction (deterministic).  FP64 throughout, including
// the near-threshold 1/T magnetic-moment integrals.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBasisThreads)
basis_fp64_kernel(ModelView m, double gl_mu, double gr_mu, double kappa, double* __restrict__ basis) {
  const int i = blockIdx.x;
  const int n_nodes = m.n_nodes;
  const double lo = m.bin64[i], hi = m.bin64[m.n_t + i];
  const double t_min = m.t_min64;
  const int count = m.bin_count[i];
  double acc[kNB];
#pragma unroll
  for (int b = 0; b < kNB; ++b) acc[b] = 0.0;

  for (int n = threadIdx.x; n < count; n += blockDim.x) {
    const double e = m.node64[n];
    const double wpe = m.node64[n_nodes + n], wpm = m.node64[2 * n_nodes + n];
    const double wpt = m.node64[3 * n_nodes + n], w = m.node64[4 * n_nodes + n];
    const double tmax = 2.0 * e * e / (kMe + 2.0 * e);
    double i0, irr, ilr, imm;
    if (m.midpoint) {
      const double tc = 0.5 * (lo + hi);
      if (!(tc >= t_min && tc < tmax)) continue;
      const double dt = hi - lo, y = 1.0 - tc / e;
      i0 = dt;
      irr = dt * y * y;
      ilr = dt * kMe * tc / (e * e);
      imm = dt * (1.0 / tc - 1.0 / e);
    } else {
      const double a = fmax(lo, t_min), b = fmin(hi, tmax);
      if (!(b > a)) continue;
      const double d = b - a, u = 1.0 - a / e, v = 1.0 - b / e;
      i0 = d;
      irr = d * (u * u + u * v + v * v) / 3.0;
      ilr = kMe * d * (a + b) / (2.0 * e * e);
      imm = log1p(d / a) - d / e;
    }
    acc[0] += wpe * i0;
    acc[1] += wpe * irr;
    acc[2] += wpe * ilr;
    acc[3] += wpt * i0;
    acc[4] += wpt * irr;
    acc[5] += wpt * ilr;
    acc[6] += wpm * (gl_mu * gl_mu * i0 + gr_mu * gr_mu * irr - gl_mu * gr_mu * ilr);
    acc[7] += w * kappa * imm;
  }

  __shared__ double red[kBasisThreads / 32][kNB];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int b = 0; b < kNB; ++b) {
    const double v = warp_sum_d(acc[b]);
    if (lane == 0) red[warp][b] = v;
  }
  __syncthreads();
  if (threadIdx.x < kNB) {
    double s = 0.0;
    for (int w = 0; w < kBasisThreads / 32; ++w) s += red[w][threadIdx.x];
    basis[threadIdx.x * m.n_t + i] = s;
  }
}

// Coupling products of the reference point, hi/lo, in the order used by the
// spectrum kernel: gLe^2 gLm^2 gLt^2 gRe^2 gRm^2 gRt^2 gLe.gRe gLm.gRm gLt.gRt kappa mu^2.
struct GRef {
  float v[2][10];
};

// ---------------------------------------------------------------------------
// G1: single-point FP32 spectrum + weights (the per-theta "physics update").
// Each block owns kBinsPerBlock consecutive recoil bins and streams the
// contributing nodes once (coalesced float4 loads), computing the coupling-
// weighted per-node coefficients and the closed-form bin integrals for all
// of its bins.  Outputs (any may be null):
//   S_out[i]   = S_i(theta)
//   W_out[i]   = S_i(theta) / S_SM,i * E_SM,i   (E_SM,i where S_SM,i == 0)
//   ssm_out[i] = S_i(theta)                     (used once at create, theta = 0)
// ---------------------------------------------------------------------------
__global__ void __cluster_dims__(kSpecCluster, 1, 1) __launch_bounds__(kSpecThreads)
spectrum_point_kernel(ModelView m, const float* __restrict__ theta, dfloat sin2w, dfloat kappa, GRef gref,
                      int delta, float* __restrict__ S_out, float* __restrict__ W_out, float* __restrict__ ssm_out) {
  // coupling products as hi + lo float pairs: a single FP32 rounding of a
  // coupling would bias every bin of this theta by the same relative amount
  __shared__ float coef[2][10];
  __shared__ float4 sbin[kBinsPerBlock];
  __shared__ float sbl[kBinsPerBlock];
  __shared__ float red[kSpecThreads / 32][kBinsPerBlock];
  __shared__ float blocksum[kBinsPerBlock];

  // grid: kSpecCluster blocks (one cluster) per group of kBinsPerBlock bins;
  // the blocks of a cluster split the group's node range
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const int first = (blockIdx.x / kSpecCluster) * kBinsPerBlock;
  if (threadIdx.x < 10) {
    // couplings (eq. g_tilde) in double-float arithmetic, one product per
    // thread; nu_mu is unshifted
    const int k = threadIdx.x;
    const dfloat gle = df_add(df_add(dfloat{0.5f, 0.f}, sin2w), theta[0]);
    const dfloat gre = df_add(sin2w, theta[1]);
    const dfloat glt = df_add(df_add(dfloat{-0.5f, 0.f}, sin2w), theta[2]);
    const dfloat grt = df_add(sin2w, theta[3]);
    const dfloat glm = df_add(dfloat{-0.5f, 0.f}, sin2w), grm = sin2w;
    // order: gLe^2 gLm^2 gLt^2 gRe^2 gRm^2 gRt^2 gLe.gRe gLm.gRm gLt.gRt kappa mu^2
    const dfloat x = k == 0 ? gle : k == 1 ? glm : k == 2 ? glt : k == 3 ? gre : k == 4 ? grm : k == 5 ? grt
                   : k == 6 ? gle : k == 7 ? glm : k == 8 ? glt : kappa;
    const dfloat y = k == 0 ? gle : k == 1 ? glm : k == 2 ? glt : k == 3 ? gre : k == 4 ? grm : k == 5 ? grt
                   : k == 6 ? gre : k == 7 ? grm : k == 8 ? grt : two_prod(theta[4], theta[4]);
    const dfloat c = df_mul(x, y);
    // delta mode: monomials of theta minus those of the reference point
    const dfloat d = delta ? df_add(c, dfloat{-gref.v[0][k], -gref.v[1][k]}) : c;
    coef[0][k] = d.hi;
    coef[1][k] = d.lo;
  }
  if (threadIdx.x < kBinsPerBlock) {
    const int i = first + threadIdx.x;
    sbin[threadIdx.x] = i < m.n_t ? m.bin_f[i] : make_float4(1.f, 1.f, 0.f, 0.f);
    sbl[threadIdx.x] = i < m.n_t ? m.bin_l[i] : 0.f;
  }
  __syncthreads();

  float ch[10], cl[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    ch[k] = coef[0][k];
    cl[k] = coef[1][k];
  }
  float acc[kBinsPerBlock];
#pragma unroll
  for (int bb = 0; bb < kBinsPerBlock; ++bb) acc[bb] = 0.f;

  const int count = first < m.n_t ? m.bin_count[first] : 0;
  // software pipeline: the next node's tables load while this node computes
  constexpr int kStride = kSpecThreads * kSpecCluster;
  const int n0 = crank * kSpecThreads + threadIdx.x;
  float4 na_n, nw_n, nl_n;
  if (n0 < count) {
    na_n = m.node_a[n0];
    nw_n = m.node_w[n0];
    nl_n = m.node_wlo[n0];
  }
  for (int n = n0; n < count; n += kStride) {
    const float4 na = na_n;  // E, 1/E, k_n, m_e/E^2
    const float4 nw = nw_n;  // w P_e, w P_mu, w P_tau, w
    const float4 nl = nl_n;
    if (n + kStride < count) {
      na_n = m.node_a[n + kStride];
      nw_n = m.node_w[n + kStride];
      nl_n = m.node_wlo[n + kStride];
    }
    const float inv_e = na.y;
    const int kn = __float_as_int(na.z);
    // per-node coupling-weighted coefficients, hi*hi + (hi*lo + lo*hi): the
    // node weights and couplings enter without a shared FP32 rounding
    const float a0 = fmaf(nw.x, ch[0], fmaf(nw.y, ch[1], nw.z * ch[2])) +
                     (fmaf(nw.x, cl[0], fmaf(nw.y, cl[1], nw.z * cl[2])) +
                      fmaf(nl.x, ch[0], fmaf(nl.y, ch[1], nl.z * ch[2])));
    const float a1 = fmaf(nw.x, ch[3], fmaf(nw.y, ch[4], nw.z * ch[5])) +
                     (fmaf(nw.x, cl[3], fmaf(nw.y, cl[4], nw.z * cl[5])) +
                      fmaf(nl.x, ch[3], fmaf(nl.y, ch[4], nl.z * ch[5])));
    const float a2 = (fmaf(nw.x, ch[6], fmaf(nw.y, ch[7], nw.z * ch[8])) +
                      (fmaf(nw.x, cl[6], fmaf(nw.y, cl[7], nw.z * cl[8])) +
                       fmaf(nl.x, ch[6], fmaf(nl.y, ch[7], nl.z * ch[8])))) * na.w;
    const float a3 = fmaf(nw.w, ch[9], fmaf(nw.w, cl[9], nl.w * ch[9]));
    if (m.midpoint) {
#pragma unroll
      for (int bb = 0; bb < kBinsPerBlock; ++bb) {
        if (first + bb < kn) {
          const float tc = sbin[bb].x, dt = sbin[bb].y;
          const float y = fmaf(-tc, inv_e, 1.f);
          acc[bb] += dt * (a0 + a1 * y * y - a2 * tc + a3 * (1.f / tc - inv_e));
        }
      }
    } else {
      float4 nc = make_float4(0.f, 0.f, 0.f, 0.f);
      if (kn - first < kBinsPerBlock) nc = m.node_c[n];  // this block holds the clipped bin
#pragma unroll
      for (int bb = 0; bb < kBinsPerBlock; ++bb) {
        const int i = first + bb;
        if (i < kn) {  // complete bin [a, b]
          const float4 bf = sbin[bb];  // a, b, I0, I1
          const float u = fmaf(-bf.x, inv_e, 1.f), v = fmaf(-bf.y, inv_e, 1.f);
          const float j = bf.z * fmaf(u, u, fmaf(u, v, v * v)) * (1.f / 3.f);
          acc[bb] += fmaf(a0, bf.z, fmaf(a1, j, fmaf(-a2, bf.w, a3 * fmaf(-bf.z, inv_e, sbl[bb]))));
        } else if (i == kn) {  // bin clipped at T_max(E): integrals precomputed in FP64
          acc[bb] += fmaf(a0, nc.x, fmaf(a1, nc.z, fmaf(-a2, nc.y, a3 * nc.w)));
        }
      }
    }
  }

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int bb = 0; bb < kBinsPerBlock; ++bb) {
    const float v = warp_sum_f(acc[bb]);
    if (lane == 0) red[warp][bb] = v;
  }
  __syncthreads();
  if (threadIdx.x < kBinsPerBlock) {
    float s = 0.f;
    for (int w = 0; w < kSpecThreads / 32; ++w) s += red[w][threadIdx.x];
    blocksum[threadIdx.x] = s;
  }
  // combine the cluster's partial sums in rank order through distributed shared memory
  cluster.sync();
  if (crank == 0 && threadIdx.x < kBinsPerBlock) {
    const int i = first + threadIdx.x;
    float s = 0.f;
    for (int c = 0; c < kSpecCluster; ++c) s += cluster.map_shared_rank(blocksum, c)[threadIdx.x];
    if (i < m.n_t) {
      if (S_out) S_out[i] = s;
      if (ssm_out) ssm_out[i] = s;
      if (W_out) {
        // W = S/S_SM E_SM (E_SM where S_SM = 0); in delta mode S is the
        // deviation from the reference point and so is W (0 where S_SM = 0)
        const float den = m.ssm32[i];
        W_out[i] = den != 0.f ? (s / den) * m.esm32[i] : (delta ? 0.f : m.esm32[i]);
      }
    }
  }
  cluster.sync();  // keep every block's shared memory alive until rank 0 has read it
}

// ---------------------------------------------------------------------------
// Create-time helpers (FP64): S_SM, efficiency, lambda, E_SM and the
// pre-weighted basis shat_b,i = B_b,i E_SM,i / S_SM,i used by the batched
// path, where the weighted true spectrum of point p is
//   W_p,i = sum_b c_b(theta_p) shat_b,i = S_i(theta_p)/S_SM,i * E_SM,i.
// ---------------------------------------------------------------------------
__global__ void ssm_from_basis_kernel(const double* __restrict__ basis, int n_t, double gl_e, double gr_e,
                                      double gl_t, double gr_t, double* __restrict__ ssm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_t) return;
  const double c[kNB] = {gl_e * gl_e, gr_e * gr_e, -gl_e * gr_e, gl_t * gl_t, gr_t * gr_t, -gl_t * gr_t, 1.0, 0.0};
  double s = 0.0;
#pragma unroll
  for (int b = 0; b < kNB; ++b) s += c[b] * basis[b * n_t + i];
  ssm[i] = s;
}

// Column sums eff_i = sum_j R_ji in FP64 (coalesced over i).
__global__ void efficiency_kernel(const float* __restrict__ R, int n_rec, int ld, int n_t, double* __restrict__ eff) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_t) return;
  double s = 0.0;
  for (int j = 0; j < n_rec; ++j) s += (double)R[(size_t)j * ld + i];
  eff[i] = s;
}

// lambda = exposure / sum_i eff_i S_SM,i (single block, fixed order).
__global__ void lambda_kernel(const double* __restrict__ eff, const double* __restrict__ ssm, int n_t,
                              double exposure, double* __restrict__ lambda_out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n_t; i += blockDim.x) s += eff[i] * ssm[i];
  s = warp_sum_d(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *lambda_out = t > 0.0 ? exposure / t : 0.0;
  }
}

__global__ void esm_kernel(const double* __restrict__ ssm, const double* __restrict__ lambda, int n_t,
                           double* __restrict__ esm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_t) esm[i] = *lambda * ssm[i];
}

__global__ void shat_kernel(const double* __restrict__ basis, const double* __restrict__ ssm,
                            const double* __restrict__ esm, int n_t, int k_pad, float* __restrict__ shat,
                            float* __restrict__ shat_lo, float* __restrict__ esm32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k_pad) return;
  if (i >= n_t) {
#pragma unroll
    for (int b = 0; b < kNB; ++b) shat[b * k_pad + i] = shat_lo[b * k_pad + i] = 0.f;
    return;
  }
  const double s = ssm[i], e = esm[i];
  esm32[i] = (float)e;
#pragma unroll
  for (int b = 0; b < kNB; ++b) {
    double v;
    if (s != 0.0) v = basis[b * n_t + i] * (e / s);
    else v = (b == 6) ? e : 0.0;   // w_i = 1 where S_SM,i = 0
    const float hi = (float)v;
    shat[b * k_pad + i] = hi;
    shat_lo[b * k_pad + i] = (float)(v - (double)hi);
  }
}

// Weighted true spectrum of one point from the coefficient spectra (the
// recoil spectrum is a polynomial in the coupling monomials, Sec. II):
//   dW_i = sum_b (c_b(theta) - c_b(theta_ref)) shat_b,i
// with monomials and shat as hi + lo float pairs (delta = 0: the full W).
__global__ void weights_from_basis_kernel(const float* __restrict__ theta, dfloat sin2w, CoefRef cref,
                                          const float* __restrict__ shat, const float* __restrict__ shat_lo,
                                          int k_pad, float* __restrict__ W) {
  // a fold launched as this kernel's programmatic dependent may start now: it
  // streams R and waits for this grid's W before using it
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  __shared__ float ch[kNB], cl[kNB];
  if (threadIdx.x < kNB) {
    const dfloat s = sin2w;
    const dfloat gle = df_add(df_add(dfloat{0.5f, 0.f}, s), theta[0]), gre = df_add(s, theta[1]);
    const dfloat glt = df_add(df_add(dfloat{-0.5f, 0.f}, s), theta[2]), grt = df_add(s, theta[3]);
    const int b = threadIdx.x;
    dfloat c;
    if (b == 0) c = df_mul(gle, gle);
    else if (b == 1) c = df_mul(gre, gre);
    else if (b == 2) { c = df_mul(gle, gre); c = dfloat{-c.hi, -c.lo}; }
    else if (b == 3) c = df_mul(glt, glt);
    else if (b == 4) c = df_mul(grt, grt);
    else if (b == 5) { c = df_mul(glt, grt); c = dfloat{-c.hi, -c.lo}; }
    else if (b == 6) c = dfloat{1.f, 0.f};
    else c = two_prod(theta[4], theta[4]);
    const dfloat d = df_add(c, dfloat{-cref.hi[b], -cref.lo[b]});
    ch[b] = d.hi;
    cl[b] = d.lo;
  }
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k_pad) return;
  float a = 0.f, t = 0.f;
#pragma unroll
  for (int b = 0; b < kNB; ++b) {
    const float sh = shat[(size_t)b * k_pad + i], sl = shat_lo[(size_t)b * k_pad + i];
    a = fmaf(ch[b], sh, a);
    t = fmaf(cl[b], sh, fmaf(ch[b], sl, t));
  }
  W[i] = a + t;
}

// Reference fold (create / set-reference time, FP64):
//   W_ref,i = sum_b c_b(theta_ref) B_b,i E_SM,i / S_SM,i   (E_SM,i where S_SM,i = 0)
//   mu_ref,j = sum_i R_ji W_ref,i
__global__ void wref_kernel(const double* __restrict__ basis, const double* __restrict__ ssm,
                            const double* __restrict__ esm, int n_t, CoefRef c, double* __restrict__ wref) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_t) return;
  const double sm = ssm[i], e = esm[i];
  if (sm == 0.0) {
    wref[i] = e;
    return;
  }
  double v = 0.0;
#pragma unroll
  for (int b = 0; b < kNB; ++b) v += ((double)c.hi[b] + (double)c.lo[b]) * basis[b * n_t + i];
  wref[i] = v * (e / sm);
}

__global__ void muref_kernel(const float* __restrict__ R, int ld, int n_t, const double* __restrict__ wref,
                             double* __restrict__ muref) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < n_t; i += blockDim.x) s += (double)R[(size_t)j * ld + i] * wref[i];
  s = warp_sum_d(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    muref[j] = t;
  }
}

}  // namespace

cudaError_t launch_reference_fold(srw_ctx* h, cudaStream_t s) {
  double* d_w = nullptr;
  cudaError_t e = dev_malloc_async(&d_w, sizeof(double) * h->n_t, s);
  if (e != cudaSuccess) return e;
  wref_kernel<<<(h->n_t + 255) / 256, 256, 0, s>>>(h->d_basis, h->d_ssm64, h->d_esm64, h->n_t, h->cref, d_w);
  muref_kernel<<<h->n_rec, 256, 0, s>>>(h->d_R, h->ld_r, h->n_t, d_w, h->d_muref64);
  if ((e = launch_result()) != cudaSuccess) return e;
  return cudaFreeAsync(d_w, s);
}

cudaError_t launch_weights_from_basis(const srw_ctx* h, const float* theta, float* W, cudaStream_t s) {
  weights_from_basis_kernel<<<(h->k_pad + 255) / 256, 256, 0, s>>>(theta, df_from_double(h->sin2w), h->cref,
                                                                  h->d_shat, h->d_shat_lo, h->k_pad, W);
  return launch_result();
}

cudaError_t launch_basis_fp64(const srw_ctx* h, cudaStream_t s) {
  const ModelView m = model_view(h);
  const double gl_mu = -0.5 + h->sin2w, gr_mu = h->sin2w;
  basis_fp64_kernel<<<h->n_t, kBasisThreads, 0, s>>>(m, gl_mu, gr_mu, h->kappa, h->d_basis);
  return launch_result();
}

cudaError_t launch_spectrum_point(const srw_ctx* h, const float* theta, float* S_out, float* W_out, float* ssm_out,
                                  cudaStream_t s, bool delta) {
  const ModelView m = model_view(h);
  const int grid = (h->n_t + kBinsPerBlock - 1) / kBinsPerBlock * kSpecCluster;
  GRef g;
  for (int k = 0; k < 10; ++k) {
    g.v[0][k] = h->gref[0][k];
    g.v[1][k] = h->gref[1][k];
  }
  delta = delta && h->use_ref;
  spectrum_point_kernel<<<grid, kSpecThreads, 0, s>>>(m, theta, df_from_double(h->sin2w), df_from_double(h->kappa),
                                                        g, delta ? 1 : 0, S_out, W_out, ssm_out);
  return launch_result();
}

// Builds S_SM (FP64), lambda, E_SM and shat.  Requires d_basis.
cudaError_t launch_build_shat(srw_ctx* h, cudaStream_t s) {
  const int n_t = h->n_t, thr = 256;
  const int g_t = (n_t + thr - 1) / thr;
  const double s2 = h->sin2w;
  ssm_from_basis_kernel<<<g_t, thr, 0, s>>>(h->d_basis, n_t, 0.5 + s2, s2, -0.5 + s2, s2, h->d_ssm64);
  cudaError_t e = launch_result();
  if (e != cudaSuccess) return e;
  if (!h->has_esm_input) {
    double* d_eff = nullptr;
    double* d_lam = nullptr;
    if ((e = dev_malloc_async(&d_eff, sizeof(double) * (n_t + 1), s)) != cudaSuccess) return e;
    d_lam = d_eff + n_t;
    efficiency_kernel<<<g_t, thr, 0, s>>>(h->d_R, h->n_rec, h->ld_r, n_t, d_eff);
    lambda_kernel<<<1, 1024, 0, s>>>(d_eff, h->d_ssm64, n_t, h->exposure, d_lam);
    esm_kernel<<<g_t, thr, 0, s>>>(h->d_ssm64, d_lam, n_t, h->d_esm64);
    if ((e = launch_result()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(&h->lambda, d_lam, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaFreeAsync(d_eff, s)) != cudaSuccess) return e;
  }
  const int g_k = (h->k_pad + thr - 1) / thr;
  shat_kernel<<<g_k, thr, 0, s>>>(h->d_basis, h->d_ssm64, h->d_esm64, n_t, h->k_pad, h->d_shat, h->d_shat_lo,
                                    h->d_esm32);
  return launch_result();
}

}  // namespace srw
