// Per-component joint response (Sec. III.B, eq. Rij) on the fold's
// concatenated (component, true bin) axis, and single-point spectra from the
// FP64 coefficient spectra.
//
// Create time, FP64: the live-time-corrected column sums of each component's
// Monte Carlo histogram give its global normalisation and the true bins that
// hold events; the host then fixes the component's factor N_k s^(k) / Z_k and
// the gather writes
//   R_cat[j][col0 + c] = M_j * factor_k * N^(k)_{j, i_c} / M^(k)_j
// (FP64 product, one FP32 rounding).

#include "srw_internal.h"

namespace srw {
namespace {

// One thread per true bin; rows j stream with consecutive threads reading
// consecutive columns of the row-major histogram (coalesced).
__global__ void joint_colsum_kernel(const double* __restrict__ hist, const double* __restrict__ mask,
                                    const double* __restrict__ live, int n_rec, int n_t, double* __restrict__ colZ,
                                    double* __restrict__ colY) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_t) return;
  double z = 0.0, y = 0.0;
  for (int j = 0; j < n_rec; ++j) {
    const double v = hist[(size_t)j * n_t + i] / mask[j];
    z += v;
    y += live[j] * v;
  }
  colZ[i] = z;
  colY[i] = y;
}

__global__ void joint_gather_kernel(const double* __restrict__ hist, const double* __restrict__ mask,
                                    const double* __restrict__ live, int n_rec, int n_t,
                                    const int* __restrict__ cols, int n_cols, double factor, float* __restrict__ R,
                                    int ld, int col0) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cols) return;
  const size_t i = (size_t)cols[c];
  for (int j = blockIdx.y; j < n_rec; j += gridDim.y) {
    const double row = live[j] * factor / mask[j];
    R[(size_t)j * ld + col0 + c] = (float)(row * hist[(size_t)j * n_t + i]);
  }
}

// Coupling monomials c_b(theta) in FP64 (Sec. II, eq. g_tilde): the NSI
// parameters shift the nu_e and nu_tau chiral couplings.
__device__ void monomials64(const float* theta, double s2, double c[kNB]) {
  const double gle = 0.5 + s2 + (double)theta[0], gre = s2 + (double)theta[1];
  const double glt = -0.5 + s2 + (double)theta[2], grt = s2 + (double)theta[3];
  const double mu = (double)theta[4];
  c[0] = gle * gle;
  c[1] = gre * gre;
  c[2] = -gle * gre;
  c[3] = glt * glt;
  c[4] = grt * grt;
  c[5] = -glt * grt;
  c[6] = 1.0;
  c[7] = mu * mu;
}

__global__ void basis_eval_kernel(const float* __restrict__ theta, double s2, const double* __restrict__ basis,
                                  const double* __restrict__ ssm, const double* __restrict__ esm, int n, int mode,
                                  float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double c[kNB];
  monomials64(theta, s2, c);
  double v = 0.0;
#pragma unroll
  for (int b = 0; b < kNB; ++b) v += c[b] * basis[(size_t)b * n + i];
  if (mode == 1) v = ssm[i] != 0.0 ? v / ssm[i] * esm[i] : esm[i];
  out[i] = (float)v;
}

}  // namespace

cudaError_t launch_joint_colsums(const double* hist, const double* mask, const double* live, int n_rec, int n_t,
                                 double* colZ, double* colY, cudaStream_t s) {
  joint_colsum_kernel<<<(n_t + 127) / 128, 128, 0, s>>>(hist, mask, live, n_rec, n_t, colZ, colY);
  return launch_result();
}

cudaError_t launch_joint_gather(const double* hist, const double* mask, const double* live, int n_rec, int n_t,
                                const int* cols, int n_cols, double factor, float* R, int ld, int col0,
                                cudaStream_t s) {
  if (n_cols <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((n_cols + 127) / 128), (unsigned)(n_rec < 1024 ? n_rec : 1024));
  joint_gather_kernel<<<grid, 128, 0, s>>>(hist, mask, live, n_rec, n_t, cols, n_cols, factor, R, ld, col0);
  return launch_result();
}

cudaError_t launch_basis_eval(const srw_ctx* h, const float* theta, int mode, float* out, cudaStream_t s) {
  basis_eval_kernel<<<(h->n_t + 255) / 256, 256, 0, s>>>(theta, h->sin2w, h->d_basis, h->d_ssm64, h->d_esm64, h->n_t,
                                                         mode, out);
  return launch_result();
}

}  // namespace srw
