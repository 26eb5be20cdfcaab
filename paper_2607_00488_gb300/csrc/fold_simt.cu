// Batched fold in FP32 on the SIMT pipes (the FP32 way of the batched scan).
//
// For P parameter points the fold of eq. matrix_reweight becomes the
// contraction  M[p][j] = sum_i W[p][i] R[j][i]  with the reweighted true
// spectra W[p][i] = w_i(theta_p) E_SM,i.  Because the recoil spectrum is a
// polynomial in the couplings, W[p][i] = sum_b c_b(theta_p) shat_b,i with the
// eight pre-weighted coefficient spectra shat (built once in FP64); each
// block produces its W tile on chip from shat and the 8 coefficients of its
// points, so W is never written to memory.  The epilogue adds the summed
// background, applies the mask, evaluates the Poisson terms and reduces over
// its rec bins per point into FP64 partials (one per rec tile).  The fold is
// taken of W(theta) - W_ref; the FP64 reference fold R W_ref enters with the
// background (b64 argument = background + reference fold).
//
// Accumulation: FP32 FMAs over one 16-wide K tile, tiles combined with Kahan
// compensation.  The rounding of an FMA chain is not independent from row to
// row: neighbouring reconstructed bins accumulate nearly the same sequence of
// partial sums, so their errors share a sign, and -2 ln L sums them with the
// weights 1 - n_j/mu_j, which share it too near a shifted spectrum.  The
// error of a chain grows with its length; 64-term chains moved -2 ln L by
// 1.7e-4 at a point 220 units from the data (FP32 emulation and GB300 agree),
// 16-term chains by 2e-5.

#include <algorithm>
#include <vector>

#include "dfloat.cuh"
#include "poisson.cuh"
#include "srw_internal.h"

namespace srw {
namespace {

constexpr int BM = 64;    // points per block
constexpr int BN = 128;   // rec bins per block
constexpr int BK = 16;
constexpr int THR = 256;  // 16 x 16 threads
constexpr int TM = 4;     // points per thread
constexpr int TN = 8;     // rec bins per thread

// Coupling monomials c_b(theta) (see srw_internal.h) in double-float
// arithmetic, returned as hi + lo float pairs so that W carries no per-theta
// rounding bias.
__device__ __forceinline__ void coefficients(const float* th, dfloat s, const CoefRef& ref, float* hi, float* lo) {
  const dfloat gle = df_add(df_add(dfloat{0.5f, 0.f}, s), th[0]), gre = df_add(s, th[1]);
  const dfloat glt = df_add(df_add(dfloat{-0.5f, 0.f}, s), th[2]), grt = df_add(s, th[3]);
  const dfloat x = df_mul(gle, gre), y = df_mul(glt, grt);
  const dfloat c[kNB] = {df_mul(gle, gle), df_mul(gre, gre), {-x.hi, -x.lo}, df_mul(glt, glt),
                         df_mul(grt, grt), {-y.hi, -y.lo}, {1.f, 0.f}, two_prod(th[4], th[4])};
#pragma unroll
  for (int b = 0; b < kNB; ++b) {
    const dfloat d = df_add(c[b], dfloat{-ref.hi[b], -ref.lo[b]});  // deviation from the reference point
    hi[b] = d.hi;
    lo[b] = d.lo;
  }
}

__global__ void __launch_bounds__(THR, 2)
fold_simt_kernel(const float* __restrict__ theta, int P, dfloat sin2w, CoefRef cref, const float* __restrict__ shat,
                 const float* __restrict__ shat_lo, int k_pad, const float* __restrict__ R, int n_rec, int ld,
                 const double* __restrict__ n64, const double* __restrict__ b64,
                 const unsigned char* __restrict__ mask, double* __restrict__ parts,
                 float* __restrict__ musig_out, unsigned* __restrict__ status, const int2* __restrict__ krange) {
  __shared__ float cs[BM][2 * kNB + 1];
  __shared__ __align__(16) float Ws[2][BK][BM];
  __shared__ __align__(16) float Rs[2][BK][BN + 4];

  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.x * BM, j0 = blockIdx.y * BN;

  if (tid < BM) {
    float hi[kNB], lo[kNB];
    const int p = m0 + tid;
    if (p < P) {
      coefficients(theta + (size_t)p * 5, sin2w, cref, hi, lo);
    } else {
#pragma unroll
      for (int b = 0; b < kNB; ++b) hi[b] = lo[b] = 0.f;
    }
#pragma unroll
    for (int b = 0; b < kNB; ++b) {
      cs[tid][b] = hi[b];
      cs[tid][kNB + b] = lo[b];
    }
  }

  float acc[TM][TN], sum[TM][TN], comp[TM][TN];
#pragma unroll
  for (int r = 0; r < TM; ++r)
#pragma unroll
    for (int c = 0; c < TN; ++c) acc[r][c] = sum[r][c] = comp[r][c] = 0.f;

  // K tiles of this rec tile that hold nonzero response; outside them every
  // product is an exact zero
  const int2 kr = krange ? krange[blockIdx.y] : make_int2(0, k_pad / BK);
  // register staging of the next tile's R (two float4 a thread); the shat
  // values are loaded when the tile's W is formed (kept live across the FMA
  // loop they spilled registers at two blocks per SM)
  const int wk = tid & (BK - 1), mg = (tid >> 4) * TM;
  float4 rv[2];
  auto load_tile = [&](int kt) {
    const int k0 = kt * BK;
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
      const int f = tid + rr * THR, row = f >> 2, c4 = f & 3, j = j0 + row;
      SRW_CHECK(status, k0 + c4 * 4 + 4 <= ld);
      rv[rr] = j < n_rec ? __ldg(reinterpret_cast<const float4*>(R + (size_t)j * ld + k0 + c4 * 4))
                         : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  auto store_tile = [&](int buf, int kt) {
    // W^T tile: W[p][k] = sum_b c_b(p) shat_b[k], (c_hi + c_lo)(s_hi + s_lo) without lo*lo
    float sh[kNB], sl[kNB];
#pragma unroll
    for (int b = 0; b < kNB; ++b) {
      sh[b] = __ldg(shat + (size_t)b * k_pad + kt * BK + wk);
      sl[b] = __ldg(shat_lo + (size_t)b * k_pad + kt * BK + wk);
    }
    float v[TM];
#pragma unroll
    for (int r = 0; r < TM; ++r) {
      float s = 0.f, t = 0.f;
#pragma unroll
      for (int b = 0; b < kNB; ++b) {
        s = fmaf(cs[mg + r][b], sh[b], s);
        t = fmaf(cs[mg + r][kNB + b], sh[b], fmaf(cs[mg + r][b], sl[b], t));
      }
      v[r] = s + t;
    }
    *reinterpret_cast<float4*>(&Ws[buf][wk][mg]) = make_float4(v[0], v[1], v[2], v[3]);
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {  // R tile, transposed into Rs[k][j]
      const int f = tid + rr * THR, row = f >> 2, c4 = f & 3;
      Rs[buf][c4 * 4 + 0][row] = rv[rr].x;
      Rs[buf][c4 * 4 + 1][row] = rv[rr].y;
      Rs[buf][c4 * 4 + 2][row] = rv[rr].z;
      Rs[buf][c4 * 4 + 3][row] = rv[rr].w;
    }
  };

  __syncthreads();  // the block's coefficients are in shared memory
  if (kr.x < kr.y) load_tile(kr.x);
  for (int kt = kr.x; kt < kr.y; ++kt) {
    const int buf = (kt - kr.x) & 1;
    // the other buffer was last read before the previous iteration's barrier
    store_tile(buf, kt);
    __syncthreads();
    if (kt + 1 < kr.y) load_tile(kt + 1);  // in flight during the FMAs below
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      const float4 a = *reinterpret_cast<const float4*>(&Ws[buf][k][ty * TM]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Rs[buf][k][tx * TN]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Rs[buf][k][tx * TN + 4]);
      const float av[TM] = {a.x, a.y, a.z, a.w};
      const float bv[TN] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
    }
    // each 16-term chain is added to the running sum with Kahan compensation
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
      for (int c = 0; c < TN; ++c) {
        const float y = acc[r][c] - comp[r][c];
        const float t = sum[r][c] + y;
        comp[r][c] = (t - sum[r][c]) - y;
        sum[r][c] = t;
        acc[r][c] = 0.f;
      }
  }

  if (musig_out != nullptr) {  // batched folded spectra
#pragma unroll
    for (int r = 0; r < TM; ++r) {
      const int p = m0 + ty * TM + r;
      if (p >= P) continue;
#pragma unroll
      for (int c = 0; c < TN; ++c) {
        const int j = j0 + tx * TN + c;
        if (j < n_rec) musig_out[(size_t)p * n_rec + j] = sum[r][c] - comp[r][c];
      }
    }
  }
  if (parts == nullptr) return;
  // Epilogue: Poisson terms (FP64) over this block's rec bins, per point.
  double nj[TN], bj[TN];
  bool on[TN];
#pragma unroll
  for (int c = 0; c < TN; ++c) {
    const int j = j0 + tx * TN + c;
    on[c] = j < n_rec && (mask == nullptr || mask[j] != 0);
    nj[c] = on[c] ? n64[j] : 0.0;
    bj[c] = on[c] ? b64[j] : 0.0;
  }
#pragma unroll
  for (int r = 0; r < TM; ++r) {
    double d = 0.0;
#pragma unroll
    for (int c = 0; c < TN; ++c) {
      if (on[c]) d += poisson_term_f64(((double)sum[r][c] - (double)comp[r][c]) + bj[c], nj[c]);
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    const int p = m0 + ty * TM + r;
    if (tx == 0 && p < P) parts[(size_t)blockIdx.y * P + p] = d;
  }
}

}  // namespace

int fold_simt_parts(int n_rec) { return (n_rec + BN - 1) / BN; }

cudaError_t launch_fold_simt(const srw_ctx* h, const float* theta, int P, double* parts, cudaStream_t s,
                             int* n_parts, float* musig_out) {
  const dim3 grid((P + BM - 1) / BM, (h->n_rec + BN - 1) / BN);
  fold_simt_kernel<<<grid, THR, 0, s>>>(theta, P, df_from_double(h->sin2w), h->cref, h->d_shat, h->d_shat_lo, h->k_pad, h->d_R, h->n_rec,
                                        h->ld_r, h->d_n64, h->d_bref64, h->d_mask, parts, musig_out, h->d_status,
                                        h->d_simt_kr);
  if (n_parts) *n_parts = (int)grid.y;
  return launch_result();
}

// Per rec tile of BN bins the K tiles [first, end) between its first and last
// nonzero column of R (FP32, exact zeros outside; a tile without any nonzero
// element gets an empty range).
cudaError_t simt_prepare(srw_ctx* h, const std::vector<float>& R) {
  const int nt = fold_simt_parts(h->n_rec), n_kt = h->k_pad / BK, cols = std::min(h->ld_r, h->k_pad);
  std::vector<int2> kr(nt);
  for (int t = 0; t < nt; ++t) {
    int first = cols, last = -1;
    for (int j = t * BN; j < std::min(h->n_rec, (t + 1) * BN); ++j) {
      const float* row = R.data() + (size_t)j * h->ld_r;
      for (int k = 0; k < first; ++k)
        if (row[k] != 0.f) {
          first = k;
          break;
        }
      for (int k = cols - 1; k > last; --k)
        if (row[k] != 0.f) {
          last = k;
          break;
        }
    }
    kr[t] = last < 0 ? make_int2(0, 0) : make_int2(first / BK, std::min(n_kt, last / BK + 1));
  }
  cudaError_t e = cudaSuccess;
  if (!h->d_simt_kr && (e = dev_malloc(&h->d_simt_kr, sizeof(int2) * (size_t)nt)) != cudaSuccess) return e;
  h->device_bytes += sizeof(int2) * (size_t)nt;
  return cudaMemcpy(h->d_simt_kr, kr.data(), sizeof(int2) * (size_t)nt, cudaMemcpyHostToDevice);
}

}  // namespace srw
