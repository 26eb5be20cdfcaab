// Learned surrogate of the likelihood: a GELU MLP theta -> log mu (expected
// counts per reconstructed bin), trained on spectra of the exact path and
// used to pre-screen dense parameter scans (srw_surrogate_* in srw.h).
//
//   x  = (theta - centre) / half_width                    5 inputs, zero padded to 128
//   h1 = gelu(W1 x + b1), h2 = gelu(W2 h1 + b2), h3 = gelu(W3 h2 + b3)     (256 each)
//   y  = W4 h3 + b4,   log mu_j = m_j + s_j y_j             (n_rec outputs, padded to 256)
//
// gelu(z) = z Phi(z) (erf form).  Training: mean squared error of y against
// standardized targets, Adam with FP32 master weights and BF16 copies of W and
// W^T for the tensor cores.
//
// Every matrix product is one persistent tcgen05 GEMM, C = A B^T with A
// [M][K] and B [N][K] BF16, both K-major (128-byte swizzle, TMA-fed), FP32
// accumulation in TMEM (double-buffered), and an epilogue fused per use:
//   forward, hidden layer : z = C + b; h = gelu(z) -> H, H^T (BF16), gelu'(z) (FP32)
//   forward, output (fit) : y = C + b; e = y - t -> dY = 2e/count, dY^T (BF16); sum e^2
//   backward, data        : dZ = C * gelu'(z) -> dZ, dZ^T (BF16)
//   backward, weights     : dW = C (FP32)          (C = dZ^T H over the batch)
//   forward, output (scan): mu = exp(m + s (C + b)) -> Poisson deviance summed per point
// Activations are stored both row-major (operand A of the next layer's
// product) and transposed (operand of the weight-gradient product), so every
// product reads K-major operands.  Roles of a CTA: warp 0 TMA producer, warp 1
// MMA issuer / TMEM owner, warps 2-9 epilogue: two per TMEM lane quarter
// (warp w reads lanes 32 (w % 4) ...), each on half the columns.  Every wait
// is bounded; a timeout raises kStatusTimeout.

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "dfloat.cuh"
#include "poisson.cuh"
#include "ptx.cuh"
#include "srw_internal.h"
#include "tc.cuh"

namespace srw {
namespace {

using namespace tc;

constexpr int kBM = 128;
constexpr int kBK = 64;
constexpr int kTmaWarp = 0;
constexpr int kMmaWarp = 1;
constexpr int kEpiWarps = 8;                     // two per TMEM lane quarter, each on half the columns
constexpr int kGemmThreads = (2 + kEpiWarps) * 32;
constexpr int kIn = 5;          // theta components
constexpr int kInPad = 128;     // padded input width (one 128-row operand tile)
constexpr int kHidden = 256;

enum EpiMode { kFwdHidden = 0, kFwdOutFit = 1, kBwdData = 2, kWgrad = 3, kFwdOut = 4, kFwdScan = 5, kFwdHiddenScan = 6 };

struct EpiArgs {
  int M, N;              // output rows, columns (multiples of 128 and of the tile width)
  int rows_valid;        // rows >= rows_valid are padding (no loss, no gradient)
  int cols_valid;        // output columns >= cols_valid are padding
  const float* bias;     // [N]
  __nv_bfloat16* out_bf; // row-major BF16 [M][N]
  __nv_bfloat16* out_t;  // transposed BF16 [N][M]
  float* out_f32;        // FP32 [M][N]: gelu'(z), dW, or y
  const float* aux;      // fit: targets [M][N]; backward data: gelu'(z) [M][N]
  float scale;           // fit: 2 / (rows_valid * cols_valid)
  double* loss;          // fit: += sum of squared errors
  const float4* binc;    // scan: per bin {m_j + s_j b_j, s_j, n_j, n_j ln n_j - n_j} (masked: {0, 0, 0, -1})
  double* parts;         // scan: per (column half-tile, row) partial sums of the deviance
};

template <int BN>
struct GemmShape {
  static constexpr int kAB = kBM * kBK * 2;
  static constexpr int kBB = BN * kBK * 2;
  static constexpr int kStageBytes = kAB + kBB;
  static constexpr int kStages = (200 * 1024 / kStageBytes) < 6 ? (200 * 1024 / kStageBytes) : 6;
  static constexpr int kSmem = kStages * kStageBytes + 1024;
  static constexpr int kTmemCols = 2 * BN;
};

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

__device__ __forceinline__ void store_bf16x16(__nv_bfloat16* dst, const float* v) {
  uint32_t w[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) w[k] = pack_bf16x2(v[2 * k], v[2 * k + 1]);
  uint4* d = reinterpret_cast<uint4*>(dst);
  d[0] = make_uint4(w[0], w[1], w[2], w[3]);
  d[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

__device__ __forceinline__ void store_f32x16(float* dst, const float* v) {
  float4* d = reinterpret_cast<float4*>(dst);
#pragma unroll
  for (int k = 0; k < 4; ++k) d[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
}

template <int BN, int MODE>
__global__ void __launch_bounds__(kGemmThreads, 1)
mlp_gemm_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b, int M, int N,
                int K, const EpiArgs E, unsigned* status) {
  using S = GemmShape<BN>;
  constexpr int ST = S::kStages;
  extern __shared__ unsigned char dsmem_raw[];
  // 1024-byte aligned base for the swizzled tiles, formed by pointer arithmetic on
  // the shared array so that plain loads through it stay shared-memory loads
  // (a round trip through an integer makes them generic loads: slower, and on
  // the long scoreboard)
  unsigned char* smem = dsmem_raw + ((1024u - (ptx::smem_addr(dsmem_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t full[ST], empty[ST], acc_full[2], acc_empty[2], drain;
  __shared__ uint32_t tmem_slot;
  __shared__ unsigned abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_tn = N / BN;
  const int n_tiles = (M / kBM) * n_tn;
  const int n_kb = K / kBK;
  auto a_s = [&](int st) { return smem + (size_t)st * S::kStageBytes; };
  auto b_s = [&](int st) { return smem + (size_t)st * S::kStageBytes + S::kAB; };

  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(&acc_full[b], 1);
      ptx::mbar_init(&acc_empty[b], kEpiWarps);
    }
    ptx::mbar_init(&drain, 1);
    abort_flag = 0u;
    ptx::fence_barrier_init();
  }
  if (warp == kMmaWarp) tmem_alloc(&tmem_slot, S::kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_slot;
  auto give_up = [&]() {
    atomicExch(&abort_flag, 1u);
    atomicOr(status, kStatusTimeout);
  };

  if (warp == kTmaWarp) {
    if (lane == 0) {
      int g = 0, issued = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        if (!ok || aborted(&abort_flag)) break;
        const int m0 = (t / n_tn) * kBM, n0 = (t % n_tn) * BN;
        for (int kb = 0; kb < n_kb; ++kb, ++g) {
          const int st = g % ST;
          if (!ptx::mbar_wait(&empty[st], ((g / ST) & 1) ^ 1, &abort_flag)) {
            give_up();
            ok = false;
            break;
          }
          ptx::mbar_arrive_expect_tx(&full[st], (uint32_t)S::kStageBytes);
          tma_load_2d(a_s(st), &map_a, kb * kBK, m0, &full[st]);
          tma_load_2d(b_s(st), &map_b, kb * kBK, n0, &full[st]);
          issued = g + 1;
        }
      }
      for (int u = max(0, issued - ST); u < issued; ++u)  // never end with copies in flight
        ptx::mbar_wait(&full[u % ST], (u / ST) & 1, nullptr, 100000000ull);
    }
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f16kind(kBM, BN, false);
      int g = 0, tc = -1;
      bool issued_any = false;
      for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        ++tc;
        if (aborted(&abort_flag)) break;
        const int buf = tc & 1;
        if (!ptx::mbar_wait(&acc_empty[buf], ((tc >> 1) & 1) ^ 1, &abort_flag)) {
          give_up();
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(buf * BN);
        bool ok = true;
        for (int kb = 0; kb < n_kb; ++kb, ++g) {
          const int st = g % ST;
          if (!ptx::mbar_wait(&full[st], (g / ST) & 1, &abort_flag)) {
            give_up();
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t as = ptx::smem_addr(a_s(st)), bs = ptx::smem_addr(b_s(st));
#pragma unroll
          for (int ks = 0; ks < kBK / 16; ++ks)
            mma_bf16(d_tmem, smem_desc_sw128(as + ks * 32u), smem_desc_sw128(bs + ks * 32u), idesc, (kb | ks) != 0);
          issued_any = true;
          mma_commit(&empty[st]);
        }
        if (!ok) break;
        mma_commit(&acc_full[buf]);
      }
      if (issued_any) {
        mma_commit(&drain);
        ptx::mbar_wait(&drain, 0, nullptr, 100000000ull);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;                  // TMEM lanes 32 q .. 32 q + 31
    const int half = (warp - 2) >> 2;        // columns [half BN/2, (half + 1) BN/2)
    int tc = -1;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
      ++tc;
      if (__any_sync(0xffffffffu, aborted(&abort_flag))) break;
      const int m0 = (t / n_tn) * kBM, n0 = (t % n_tn) * BN;
      const int buf = tc & 1;
      if (!warp_wait(&acc_full[buf], (tc >> 1) & 1, &abort_flag)) {
        give_up();
        break;
      }
      tc_fence_after();
      const int m = m0 + q * 32 + lane;
      const bool row_on = m < E.rows_valid;
      const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN);
      float sse = 0.f;
      dfloat dev = {0.f, 0.f};
      bool infinite = false;
#pragma unroll 1
      for (int c0 = half * (BN / 2); c0 < (half + 1) * (BN / 2); c0 += 16) {
        const int n = n0 + c0;
        float v[16];
        tmem_ld16(tbase + (uint32_t)c0, v);
        if (MODE == kFwdHidden || MODE == kFwdHiddenScan) {
          float gz[16];
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const float z = v[k] + __ldg(E.bias + n + k);
            v[k] = gelu_f(z);
            if (MODE == kFwdHidden) gz[k] = gelu_grad_f(z);
          }
          store_bf16x16(E.out_bf + (size_t)m * N + n, v);
          if (MODE == kFwdHidden) {
            store_f32x16(E.out_f32 + (size_t)m * N + n, gz);
#pragma unroll
            for (int k = 0; k < 16; ++k) E.out_t[(size_t)(n + k) * M + m] = __float2bfloat16_rn(v[k]);
          }
        } else if (MODE == kFwdOutFit) {
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const float y = v[k] + __ldg(E.bias + n + k);
            const float e = (row_on && n + k < E.cols_valid) ? y - E.aux[(size_t)m * N + n + k] : 0.f;
            sse = fmaf(e, e, sse);
            v[k] = e * E.scale;
          }
          store_bf16x16(E.out_bf + (size_t)m * N + n, v);
#pragma unroll
          for (int k = 0; k < 16; ++k) E.out_t[(size_t)(n + k) * M + m] = __float2bfloat16_rn(v[k]);
        } else if (MODE == kBwdData) {
          const float4* gp = reinterpret_cast<const float4*>(E.aux + (size_t)m * N + n);
#pragma unroll
          for (int k4 = 0; k4 < 4; ++k4) {
            const float4 gz = gp[k4];
            v[4 * k4] *= gz.x;
            v[4 * k4 + 1] *= gz.y;
            v[4 * k4 + 2] *= gz.z;
            v[4 * k4 + 3] *= gz.w;
          }
          store_bf16x16(E.out_bf + (size_t)m * N + n, v);
#pragma unroll
          for (int k = 0; k < 16; ++k) E.out_t[(size_t)(n + k) * M + m] = __float2bfloat16_rn(v[k]);
        } else if (MODE == kWgrad) {
          store_f32x16(E.out_f32 + (size_t)m * N + n, v);
        } else if (MODE == kFwdOut) {
#pragma unroll
          for (int k = 0; k < 16; ++k) v[k] += __ldg(E.bias + n + k);
          store_f32x16(E.out_f32 + (size_t)m * N + n, v);
        } else {  // kFwdScan: deviance of mu = exp(lm), lm = m + s (y + b) = log mu:
                  // t = mu - n + n ln(n / mu) = mu - n lm + (n ln n - n)
          float ts = 0.f;
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const float4 c = __ldg(E.binc + n + k);
            const float lm = fmaf(c.y, v[k], c.x);
            ts += fmaf(-c.z, lm, __expf(lm) + c.w);
          }
          if (isinf(ts)) infinite = true;
          else dev = df_add(dev, ts);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&acc_empty[buf]);
      if (MODE == kFwdOutFit) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sse += __shfl_xor_sync(0xffffffffu, sse, o);
        if (lane == 0) atomicAdd(E.loss, (double)sse);
      }
      if (MODE == kFwdScan && row_on)
        E.parts[((size_t)(n0 / BN) * 2 + half) * E.rows_valid + m] =
            infinite ? __longlong_as_double(0x7ff0000000000000LL) : (double)dev.hi + (double)dev.lo;
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kMmaWarp) tmem_dealloc(tmem_base, S::kTmemCols);
}

// theta [rows][5] -> X0 [M][128] and X0^T [128][M] (BF16), normalised to the
// box.  Only columns 0-7 of X0 and rows 0-4 of X0^T are written: the padding
// is zeroed once when the buffers are made.
__global__ void mlp_input_kernel(const float* __restrict__ theta, int rows, int M, float4 c0, float c4, float4 h0,
                                 float h4, __nv_bfloat16* __restrict__ x, __nv_bfloat16* __restrict__ xt) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  float u[kIn] = {0.f, 0.f, 0.f, 0.f, 0.f};
  if (m < rows) {
    const float* th = theta + (size_t)m * kIn;
    u[0] = (th[0] - c0.x) / h0.x;
    u[1] = (th[1] - c0.y) / h0.y;
    u[2] = (th[2] - c0.z) / h0.z;
    u[3] = (th[3] - c0.w) / h0.w;
    u[4] = (th[4] - c4) / h4;
  }
  *reinterpret_cast<uint4*>(x + (size_t)m * kInPad) =
      make_uint4(pack_bf16x2(u[0], u[1]), pack_bf16x2(u[2], u[3]), pack_bf16x2(u[4], 0.f), 0u);
  if (xt)
#pragma unroll
    for (int k = 0; k < kIn; ++k) xt[(size_t)k * M + m] = __float2bfloat16_rn(u[k]);
}

// Per-bin constants of the scan epilogue (from the standardization, the output
// bias and the data): {m_j + s_j b_j, s_j, n_j, n_j ln n_j - n_j}; masked bins
// and padding columns {0, 0, 0, -1} (exp(0) - 1 = 0).
__global__ void scan_consts_kernel(const float* __restrict__ mean, const float* __restrict__ stdv,
                                   const float* __restrict__ bias, const float2* __restrict__ nb, int n, int n_pad,
                                   float4* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_pad) return;
  float4 c = make_float4(0.f, 0.f, 0.f, -1.f);
  if (j < n && nb[j].x >= 0.f) {
    const float nj = nb[j].x;
    c = make_float4(fmaf(stdv[j], bias[j], mean[j]), stdv[j], nj, nj > 0.f ? nj * logf(nj) - nj : 0.f);
  }
  out[j] = c;
}

// db[r] = sum_m dZ^T[r][m]: one warp per row.
__global__ void rowsum_kernel(const __nv_bfloat16* __restrict__ a, int rows, int cols, float* __restrict__ out) {
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= rows) return;
  const int lane = threadIdx.x & 31;
  float s = 0.f;
  for (int c = lane; c < cols; c += 32) s += __bfloat162float(a[(size_t)r * cols + c]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[r] = s;
}

// One flat parameter block of a layer for the Adam update.
struct AdamLayer {
  float* w;              // master FP32 [out][in] (weights) or [out] (biases)
  const float* g;
  float* m;
  float* v;
  __nv_bfloat16* w_bf;   // BF16 copy [out][in] (nullptr for biases)
  __nv_bfloat16* wt_bf;  // BF16 transposed copy [in][out]
  int out, in;           // in = 1 for biases
  long long first;       // offset of this block in the flat index space
};
struct AdamArgs {
  AdamLayer L[8];
  int n_layers;
  long long total;
  float lr, beta1, beta2, eps, c1, c2;  // c1 = 1 - beta1^t, c2 = 1 - beta2^t
};

__global__ void adam_kernel(const AdamArgs A) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.total) return;
  int l = 0;
  while (l + 1 < A.n_layers && i >= A.L[l + 1].first) ++l;
  const AdamLayer& L = A.L[l];
  const long long k = i - L.first;
  const float g = L.g[k];
  const float m = A.beta1 * L.m[k] + (1.f - A.beta1) * g;
  const float v = A.beta2 * L.v[k] + (1.f - A.beta2) * g * g;
  L.m[k] = m;
  L.v[k] = v;
  const float w = L.w[k] - A.lr * (m / A.c1) / (sqrtf(v / A.c2) + A.eps);
  L.w[k] = w;
  if (L.w_bf) {
    const __nv_bfloat16 b = __float2bfloat16_rn(w);
    L.w_bf[k] = b;
    const int o = (int)(k / L.in), c = (int)(k % L.in);
    L.wt_bf[(size_t)c * L.out + o] = b;
  }
}

// FP32 master -> BF16 copies (after the weights are set from the host).
__global__ void cast_weights_kernel(const float* __restrict__ w, int out, int in, __nv_bfloat16* __restrict__ w_bf,
                                    __nv_bfloat16* __restrict__ wt_bf) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (long long)out * in) return;
  const __nv_bfloat16 b = __float2bfloat16_rn(w[k]);
  w_bf[k] = b;
  const int o = (int)(k / in), c = (int)(k % in);
  wt_bf[(size_t)c * out + o] = b;
}

// Training targets: dst [rows][ld] = log(mu_sig + b) from src [rows][n]
// (columns >= n of dst: 0).
__global__ void log_counts_kernel(const float* __restrict__ src, long long rows, int n, int ld,
                                  const double* __restrict__ b64, float* __restrict__ dst) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * ld) return;
  const long long r = i / ld;
  const int j = (int)(i % ld);
  dst[i] = j < n ? logf(fmaxf(src[r * n + j] + (float)b64[j], 1e-30f)) : 0.f;
}

// Per-column sums and sums of squares (FP64) over rows, for the standardization.
// Column sums and sums of squares of one block of 4096 rows, written to the
// block's own slot (no atomics: the statistics, and so every resumed fit, are
// the same bit for bit whatever the order in which the blocks run).
__global__ void colstats_kernel(const float* __restrict__ t, long long rows, int ld, int n, double* __restrict__ s1,
                                double* __restrict__ s2) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const long long r0 = (long long)blockIdx.y * 4096, r1 = min(rows, r0 + 4096);
  double a = 0.0, b = 0.0;
  for (long long r = r0; r < r1; ++r) {
    const double x = t[r * ld + j];
    a += x;
    b += x * x;
  }
  s1[(size_t)blockIdx.y * n + j] = a;
  s2[(size_t)blockIdx.y * n + j] = b;
}

__global__ void finish_stats_kernel(const double* __restrict__ s1, const double* __restrict__ s2, int n_blocks,
                                    long long rows, int n, float* __restrict__ mean, float* __restrict__ stdv) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double a = 0.0, b = 0.0;
  for (int k = 0; k < n_blocks; ++k) {  // fixed order over the row blocks
    a += s1[(size_t)k * n + j];
    b += s2[(size_t)k * n + j];
  }
  const double m = a / (double)rows;
  const double var = fmax(b / (double)rows - m * m, 0.0);
  const double s = sqrt(var);
  mean[j] = (float)m;
  stdv[j] = s > 1e-12 ? (float)s : 1.f;
}

__global__ void standardize_kernel(float* __restrict__ t, long long rows, int ld, int n, const float* __restrict__ mean,
                                   const float* __restrict__ stdv) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * ld) return;
  const int j = (int)(i % ld);
  if (j < n) t[i] = (t[i] - mean[j]) / stdv[j];
}

// -2 ln L = 2 sum of the per-tile deviance partials + the data constant.
template <class T>
__global__ void scan_reduce_kernel(const double* __restrict__ parts, int n_parts, int rows,
                                   const double* __restrict__ c_data, T* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= rows) return;
  double s = 0.0;
  for (int t = 0; t < n_parts; ++t) s += parts[(size_t)t * rows + p];
  out[p] = (T)(2.0 * s + *c_data);
}

// Sobol points in Gray-code order (Antonov-Saleev): point i is the xor of the
// direction numbers V[d][k] over the set bits k of i xor (i >> 1); mapped to
// the box: theta_d = lo_d + (hi_d - lo_d) x_d.
__global__ void sobol_kernel(const uint32_t* __restrict__ V, long long first, int count, float4 lo0, float lo4,
                             float4 w0, float w4, float* __restrict__ theta) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= count) return;
  const unsigned long long i = (unsigned long long)(first + r);
  unsigned long long gcode = i ^ (i >> 1);
  uint32_t x[kIn] = {0u, 0u, 0u, 0u, 0u};
  for (int k = 0; gcode != 0ull && k < 32; ++k, gcode >>= 1)
    if (gcode & 1ull)
#pragma unroll
      for (int d = 0; d < kIn; ++d) x[d] ^= V[d * 32 + k];
  const float s = 2.3283064365386963e-10f;  // 2^-32
  float* out = theta + (size_t)r * kIn;
  out[0] = lo0.x + w0.x * (__uint2float_rn(x[0]) * s);
  out[1] = lo0.y + w0.y * (__uint2float_rn(x[1]) * s);
  out[2] = lo0.z + w0.z * (__uint2float_rn(x[2]) * s);
  out[3] = lo0.w + w0.w * (__uint2float_rn(x[3]) * s);
  out[4] = lo4 + w4 * (__uint2float_rn(x[4]) * s);
}

// The same points for a list of sequence indices.
__global__ void sobol_gather_kernel(const uint32_t* __restrict__ V, const long long* __restrict__ index, int count,
                                    float4 lo0, float lo4, float4 w0, float w4, float* __restrict__ theta) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= count) return;
  const unsigned long long i = (unsigned long long)index[r];
  unsigned long long gcode = i ^ (i >> 1);
  uint32_t x[kIn] = {0u, 0u, 0u, 0u, 0u};
  for (int k = 0; gcode != 0ull && k < 32; ++k, gcode >>= 1)
    if (gcode & 1ull)
#pragma unroll
      for (int d = 0; d < kIn; ++d) x[d] ^= V[d * 32 + k];
  const float s = 2.3283064365386963e-10f;
  float* out = theta + (size_t)r * kIn;
  out[0] = lo0.x + w0.x * (__uint2float_rn(x[0]) * s);
  out[1] = lo0.y + w0.y * (__uint2float_rn(x[1]) * s);
  out[2] = lo0.z + w0.z * (__uint2float_rn(x[2]) * s);
  out[3] = lo0.w + w0.w * (__uint2float_rn(x[3]) * s);
  out[4] = lo4 + w4 * (__uint2float_rn(x[4]) * s);
}

// Radix selection of the k-th smallest non-negative float (whose bit pattern
// orders like its value): histogram of the high 16 bits, then of the low 16
// bits among the values with a given high half.
__global__ void hist_hi_kernel(const float* __restrict__ v, long long n, unsigned* __restrict__ hist) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    atomicAdd(hist + (__float_as_uint(v[i]) >> 16), 1u);
}

__global__ void hist_lo_kernel(const float* __restrict__ v, long long n, unsigned hi, unsigned* __restrict__ hist) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const unsigned b = __float_as_uint(v[i]);
    if ((b >> 16) == hi) atomicAdd(hist + (b & 0xFFFFu), 1u);
  }
}

__device__ __forceinline__ int cell_of(const float* th, float4 lo0, float lo4, float4 w0, float w4, int cpd) {
  const float u[kIn] = {(th[0] - lo0.x) / w0.x, (th[1] - lo0.y) / w0.y, (th[2] - lo0.z) / w0.z, (th[3] - lo0.w) / w0.w,
                        (th[4] - lo4) / w4};
  int c = 0;
  for (int d = kIn - 1; d >= 0; --d) {
    int k = (int)floorf(u[d] * (float)cpd);
    k = k < 0 ? 0 : (k >= cpd ? cpd - 1 : k);
    c = c * cpd + k;
  }
  return c;
}

// Indices (first + i) of the scan points to re-evaluate exactly: surrogate
// value v <= keep, or v > skip and v - margin[cell] <= bound (margin +inf:
// always, -inf: never).  The cell is computed from the point itself.
__global__ void select_kernel(const float* __restrict__ v, const uint32_t* __restrict__ V, long long first, long long n,
                              float keep, float skip, const float* __restrict__ margin, float bound, int cpd,
                              float4 lo0, float lo4, float4 w0, float w4, long long* __restrict__ out,
                              unsigned long long* __restrict__ count, long long cap) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float vi = v[i];
    bool take = vi <= keep;
    if (!take && vi > skip && margin != nullptr) {
      const unsigned long long idx = (unsigned long long)(first + i);
      unsigned long long gcode = idx ^ (idx >> 1);
      uint32_t x[kIn] = {0u, 0u, 0u, 0u, 0u};
      for (int k = 0; gcode != 0ull && k < 32; ++k, gcode >>= 1)
        if (gcode & 1ull)
          for (int d = 0; d < kIn; ++d) x[d] ^= V[d * 32 + k];
      const float s = 2.3283064365386963e-10f;
      const float th[kIn] = {lo0.x + w0.x * (__uint2float_rn(x[0]) * s), lo0.y + w0.y * (__uint2float_rn(x[1]) * s),
                             lo0.z + w0.z * (__uint2float_rn(x[2]) * s), lo0.w + w0.w * (__uint2float_rn(x[3]) * s),
                             lo4 + w4 * (__uint2float_rn(x[4]) * s)};
      take = vi - margin[cell_of(th, lo0, lo4, w0, w4, cpd)] <= bound;
    }
    if (take) {
      const unsigned long long slot = atomicAdd(count, 1ull);
      if ((long long)slot < cap) out[slot] = first + i;
    }
  }
}

// Minimum of non-negative values (their bit patterns order like the values)
// and the first index that attains it.
template <class T>
__global__ void min_bits_kernel(const T* __restrict__ v, long long n, unsigned long long* __restrict__ best) {
  unsigned long long m = ~0ull;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long b = sizeof(T) == 8 ? (unsigned long long)__double_as_longlong((double)v[i])
                                                : (unsigned long long)__float_as_uint((float)v[i]);
    m = b < m ? b : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long x = __shfl_xor_sync(0xffffffffu, m, o);
    m = x < m ? x : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMin(best, m);
}

template <class T>
__global__ void argmin_kernel(const T* __restrict__ v, long long n, const unsigned long long* __restrict__ best,
                              unsigned long long* __restrict__ index) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long b = sizeof(T) == 8 ? (unsigned long long)__double_as_longlong((double)v[i])
                                                : (unsigned long long)__float_as_uint((float)v[i]);
    if (b == *best) atomicMin(index, (unsigned long long)i);
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
  static EncodeTiledFn fn = nullptr;
  if (fn == nullptr) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess && p &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// Tensor map of a row-major BF16 matrix [rows][cols] read in boxes of 64 cols x box_rows.
cudaError_t make_map(CUtensorMap* map, const __nv_bfloat16* base, long long rows, int cols, int box_rows) {
  EncodeTiledFn enc = encoder();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int BN, int MODE>
cudaError_t gemm_attr() {
  return cudaFuncSetAttribute(mlp_gemm_kernel<BN, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              GemmShape<BN>::kSmem);
}

// One prepared product C[M][N] = A[M][K] B[N][K]^T with its epilogue.
struct Gemm {
  CUtensorMap ma, mb;
  int M = 0, N = 0, K = 0, bn = 256, mode = 0;
  EpiArgs E{};
};

template <int BN, int MODE>
cudaError_t launch_mode(const Gemm& g, int sm_count, unsigned* status, cudaStream_t s) {
  const int tiles = (g.M / kBM) * (g.N / BN);
  const int grid = tiles < sm_count ? tiles : sm_count;
  mlp_gemm_kernel<BN, MODE><<<grid, kGemmThreads, GemmShape<BN>::kSmem, s>>>(g.ma, g.mb, g.M, g.N, g.K, g.E, status);
  return srw::launch_result();
}

cudaError_t run_gemm(const Gemm& g, int sm_count, unsigned* status, cudaStream_t s) {
  if (g.bn == 256) {
    switch (g.mode) {
      case kFwdHidden: return launch_mode<256, kFwdHidden>(g, sm_count, status, s);
      case kFwdOutFit: return launch_mode<256, kFwdOutFit>(g, sm_count, status, s);
      case kBwdData: return launch_mode<256, kBwdData>(g, sm_count, status, s);
      case kWgrad: return launch_mode<256, kWgrad>(g, sm_count, status, s);
      case kFwdOut: return launch_mode<256, kFwdOut>(g, sm_count, status, s);
      case kFwdScan: return launch_mode<256, kFwdScan>(g, sm_count, status, s);
      case kFwdHiddenScan: return launch_mode<256, kFwdHiddenScan>(g, sm_count, status, s);
    }
  } else {
    if (g.mode == kWgrad) return launch_mode<128, kWgrad>(g, sm_count, status, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t gemm_attrs() {
  cudaError_t e = gemm_attr<256, kFwdHidden>();
  if (e == cudaSuccess) e = gemm_attr<256, kFwdOutFit>();
  if (e == cudaSuccess) e = gemm_attr<256, kBwdData>();
  if (e == cudaSuccess) e = gemm_attr<256, kWgrad>();
  if (e == cudaSuccess) e = gemm_attr<256, kFwdOut>();
  if (e == cudaSuccess) e = gemm_attr<256, kFwdScan>();
  if (e == cudaSuccess) e = gemm_attr<256, kFwdHiddenScan>();
  if (e == cudaSuccess) e = gemm_attr<128, kWgrad>();
  return e;
}

}  // namespace
}  // namespace srw

// ======================================================================= host state
using srw::Gemm;

struct SurrogateLayer {
  int out = 0, in = 0;  // padded sizes
  float* w = nullptr;   // FP32 master [out][in]
  float* b = nullptr;   // [out]
  float* mw = nullptr, *vw = nullptr, *mb = nullptr, *vb = nullptr;
  float* gw = nullptr, *gb = nullptr;  // gradients
  __nv_bfloat16* w_bf = nullptr;       // [out][in]
  __nv_bfloat16* wt_bf = nullptr;      // [in][out]
};

// Activations of one batch size (training buffers include transposes).
struct SurrogateBatch {
  int M = 0;
  bool train = false;
  __nv_bfloat16 *x = nullptr, *xt = nullptr;
  __nv_bfloat16 *h[3] = {}, *ht[3] = {};
  float* gz[3] = {};
  __nv_bfloat16 *dy = nullptr, *dyt = nullptr;
  __nv_bfloat16 *dz[3] = {}, *dzt[3] = {};
  float* y = nullptr;       // FP32 network output (forward hook)
  double* parts = nullptr;  // scan partials [n_out_pad / 256][M]
  double* loss = nullptr;
  Gemm fwd[4], fwd_out, fwd_scan, wgrad[4], bwd[3];
};

struct srw_surrogate_ctx {
  srw_handle h = nullptr;
  int device = 0, sm_count = 0;
  int n_out = 0, n_out_pad = 0;
  float centre[5] = {}, half[5] = {};
  SurrogateLayer L[4];
  float* mean = nullptr;  // per-bin standardization of log mu
  float* stdv = nullptr;
  float4* binc = nullptr;  // per-bin constants of the scan epilogue
  int stats_ready = 0;
  long long adam_t = 0;
  long long epochs_done = 0;  // completed epochs of the last (resumable) fit
  unsigned* d_status = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<SurrogateBatch*> batches;
  uint32_t* d_sobol = nullptr;  // direction numbers [5][32]
  std::string err;
};

namespace {

srw_status sfail(srw_surrogate s, srw_status st, const std::string& msg) {
  if (s) s->err = msg;
  return st;
}
srw_status scuda(srw_surrogate s, cudaError_t e, const char* what) {
  return sfail(s, e == cudaErrorMemoryAllocation ? SRW_ENOMEM : SRW_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define S_CUDA(s, call, what)                         \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return scuda(s, e_, what); \
  } while (0)

template <class T>
cudaError_t salloc(T** p, size_t n) {
  return srw::dev_malloc(reinterpret_cast<void**>(p), sizeof(T) * (n ? n : 1));
}
template <class T>
void sfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

// A device buffer owned by one call, released on every return path (through
// the stream's pool when it was allocated stream-ordered).
template <class T>
struct CallBuf {
  T* p = nullptr;
  cudaStream_t stream = nullptr;  // set for stream-ordered allocations
  CallBuf() = default;
  CallBuf(const CallBuf&) = delete;
  CallBuf& operator=(const CallBuf&) = delete;
  ~CallBuf() {
    if (!p) return;
    if (stream) cudaFreeAsync(p, stream);
    else cudaFree(p);
  }
};
template <class T>
cudaError_t salloc(CallBuf<T>* b, size_t n) {
  return salloc(&b->p, n);
}
template <class T>
cudaError_t salloc_async(CallBuf<T>* b, size_t n, cudaStream_t st) {
  b->stream = st;
  return srw::dev_malloc_async(&b->p, sizeof(T) * (n ? n : 1), st);
}

// CUDA events of one call, destroyed on every return path.
template <int N>
struct CallEvents {
  cudaEvent_t e[N] = {};
  CallEvents() {
    for (auto& x : e) cudaEventCreate(&x);
  }
  CallEvents(const CallEvents&) = delete;
  CallEvents& operator=(const CallEvents&) = delete;
  ~CallEvents() {
    for (auto& x : e)
      if (x) cudaEventDestroy(x);
  }
};

int round_up(long long x, int m) { return (int)((x + m - 1) / m * m); }

void free_batch(SurrogateBatch* B) {
  sfree(B->x); sfree(B->xt); sfree(B->dy); sfree(B->dyt); sfree(B->y); sfree(B->parts); sfree(B->loss);
  for (int k = 0; k < 3; ++k) {
    sfree(B->h[k]); sfree(B->ht[k]); sfree(B->gz[k]); sfree(B->dz[k]); sfree(B->dzt[k]);
  }
  delete B;
}

// Joe-Kuo direction numbers of dimensions 1-5 (published table: s, a, m_1..m_s).
void sobol_directions(uint32_t* V) {
  struct Poly { int s, a; int m[3]; };
  const Poly P[4] = {{1, 0, {1, 0, 0}}, {2, 1, {1, 3, 0}}, {3, 1, {1, 3, 1}}, {3, 2, {1, 1, 1}}};
  for (int k = 1; k <= 32; ++k) V[k - 1] = 1u << (32 - k);
  for (int d = 1; d < 5; ++d) {
    const Poly& p = P[d - 1];
    uint32_t m[33] = {0};
    for (int k = 1; k <= p.s; ++k) m[k] = (uint32_t)p.m[k - 1];
    for (int k = p.s + 1; k <= 32; ++k) {
      uint32_t v = m[k - p.s] ^ (m[k - p.s] << p.s);
      for (int i = 1; i < p.s; ++i)
        if ((p.a >> (p.s - 1 - i)) & 1) v ^= m[k - i] << i;
      m[k] = v;
    }
    for (int k = 1; k <= 32; ++k) V[d * 32 + k - 1] = m[k] << (32 - k);
  }
}

srw::EpiArgs epi0(int M, int N, int rows_valid, int cols_valid) {
  srw::EpiArgs E{};
  E.M = M;
  E.N = N;
  E.rows_valid = rows_valid;
  E.cols_valid = cols_valid;
  return E;
}

cudaError_t prep(Gemm& g, const __nv_bfloat16* A, const __nv_bfloat16* B, int M, int N, int K, int mode, int bn,
                 const srw::EpiArgs& E) {
  g.M = M;
  g.N = N;
  g.K = K;
  g.mode = mode;
  g.bn = bn;
  g.E = E;
  cudaError_t e = srw::make_map(&g.ma, A, M, K, srw::kBM);
  if (e == cudaSuccess) e = srw::make_map(&g.mb, B, N, K, bn);
  return e;
}

// Buffers and prepared products for batch size M (multiple of 128).
srw_status get_batch(srw_surrogate s, int M, bool train, SurrogateBatch** out) {
  for (SurrogateBatch* B : s->batches)
    if (B->M == M && (B->train || !train)) {
      *out = B;
      return SRW_OK;
    }
  SurrogateBatch* B = new (std::nothrow) SurrogateBatch();
  if (!B) return sfail(s, SRW_ENOMEM, "host allocation");
  B->M = M;
  B->train = train;
  const int H = srw::kHidden, NO = s->n_out_pad;
  cudaError_t e = salloc(&B->x, (size_t)M * srw::kInPad);
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = salloc(&B->h[k], (size_t)M * H);
  if (e == cudaSuccess) e = salloc(&B->parts, (size_t)(NO / 256) * 2 * M);
  if (e == cudaSuccess) e = cudaMemset(B->x, 0, sizeof(__nv_bfloat16) * (size_t)M * srw::kInPad);
  if (e == cudaSuccess) e = salloc(&B->loss, 1);
  if (train) {
    if (e == cudaSuccess) e = salloc(&B->xt, (size_t)M * srw::kInPad);
    if (e == cudaSuccess) e = cudaMemset(B->xt, 0, sizeof(__nv_bfloat16) * (size_t)M * srw::kInPad);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = salloc(&B->ht[k], (size_t)M * H);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = salloc(&B->gz[k], (size_t)M * H);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = salloc(&B->dz[k], (size_t)M * H);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = salloc(&B->dzt[k], (size_t)M * H);
    if (e == cudaSuccess) e = salloc(&B->dy, (size_t)M * NO);
    if (e == cudaSuccess) e = salloc(&B->dyt, (size_t)M * NO);
  }
  if (e != cudaSuccess) {
    free_batch(B);
    return scuda(s, e, "surrogate batch buffers");
  }
  const __nv_bfloat16* act_in[4] = {B->x, B->h[0], B->h[1], B->h[2]};
  // forward, hidden layers
  for (int l = 0; l < 3 && e == cudaSuccess; ++l) {
    srw::EpiArgs E = epi0(M, H, M, H);
    E.bias = s->L[l].b;
    E.out_bf = B->h[l];
    if (train) {
      E.out_t = B->ht[l];
      E.out_f32 = B->gz[l];
    }
    e = prep(B->fwd[l], act_in[l], s->L[l].w_bf, M, H, s->L[l].in, train ? srw::kFwdHidden : srw::kFwdHiddenScan, 256, E);
  }
  // forward, output: plain y (hook) and the scan's deviance
  if (e == cudaSuccess) {
    srw::EpiArgs E = epi0(M, NO, M, s->n_out);
    E.bias = s->L[3].b;
    E.out_f32 = B->y;
    e = prep(B->fwd_out, B->h[2], s->L[3].w_bf, M, NO, H, srw::kFwdOut, 256, E);
  }
  if (e == cudaSuccess) {
    srw::EpiArgs E = epi0(M, NO, M, s->n_out);
    E.bias = s->L[3].b;
    E.binc = s->binc;
    E.parts = B->parts;
    e = prep(B->fwd_scan, B->h[2], s->L[3].w_bf, M, NO, H, srw::kFwdScan, 256, E);
  }
  if (train) {
    if (e == cudaSuccess) {  // fit output: targets set per call
      srw::EpiArgs E = epi0(M, NO, M, s->n_out);
      E.bias = s->L[3].b;
      E.out_bf = B->dy;
      E.out_t = B->dyt;
      E.loss = B->loss;
      e = prep(B->fwd[3], B->h[2], s->L[3].w_bf, M, NO, H, srw::kFwdOutFit, 256, E);
    }
    // weight gradients dW_l = dZ_l^T A_l over the batch (K = M)
    const __nv_bfloat16* dzt[4] = {B->dzt[0], B->dzt[1], B->dzt[2], B->dyt};
    const __nv_bfloat16* actt[4] = {B->xt, B->ht[0], B->ht[1], B->ht[2]};
    for (int l = 0; l < 4 && e == cudaSuccess; ++l) {
      const int out = s->L[l].out, in = s->L[l].in;
      srw::EpiArgs E = epi0(out, in, out, in);
      E.out_f32 = s->L[l].gw;
      e = prep(B->wgrad[l], dzt[l], actt[l], out, in, M, srw::kWgrad, in >= 256 ? 256 : 128, E);
    }
    // backward data: dZ_{l-1} = (dZ_l W_l) * gelu'(z_{l-1}), l = 3, 2, 1 (W_l^T is the K-major operand)
    const __nv_bfloat16* dz_in[3] = {B->dz[1], B->dz[2], B->dy};
    for (int l = 0; l < 3 && e == cudaSuccess; ++l) {  // produces dz[l] from layer l+1
      const int K = s->L[l + 1].out;
      srw::EpiArgs E = epi0(M, H, M, H);
      E.aux = B->gz[l];
      E.out_bf = B->dz[l];
      E.out_t = B->dzt[l];
      e = prep(B->bwd[l], dz_in[l], s->L[l + 1].wt_bf, M, H, K, srw::kBwdData, 256, E);
    }
  }
  if (e != cudaSuccess) {
    free_batch(B);
    return scuda(s, e, "surrogate tensor maps");
  }
  s->batches.push_back(B);
  *out = B;
  return SRW_OK;
}

cudaError_t launch_input(srw_surrogate s, const float* theta, int rows, SurrogateBatch* B, cudaStream_t st) {
  const float4 c0 = make_float4(s->centre[0], s->centre[1], s->centre[2], s->centre[3]);
  const float4 h0 = make_float4(s->half[0], s->half[1], s->half[2], s->half[3]);
  srw::mlp_input_kernel<<<(B->M + 255) / 256, 256, 0, st>>>(theta, rows, B->M, c0, s->centre[4], h0, s->half[4], B->x,
                                                            B->train ? B->xt : nullptr);
  return srw::launch_result();
}

// Forward through the hidden layers (rows of theta; B->M >= rows).
cudaError_t forward_hidden(srw_surrogate s, const float* theta, int rows, SurrogateBatch* B, bool train, cudaStream_t st) {
  cudaError_t e = launch_input(s, theta, rows, B, st);
  for (int l = 0; l < 3 && e == cudaSuccess; ++l) {
    Gemm g = B->fwd[l];
    if (!train) {  // inference: activations only
      g.mode = srw::kFwdHiddenScan;
      g.E.out_t = nullptr;
      g.E.out_f32 = nullptr;
    }
    g.E.rows_valid = rows;
    e = srw::run_gemm(g, s->sm_count, s->d_status, st);
  }
  return e;
}

// One forward + backward pass over rows points with standardized targets
// t [M][n_out_pad] (FP32, device); gradients land in L[l].gw / gb, the summed
// squared error in B->loss.
cudaError_t fit_pass(srw_surrogate s, const float* theta, const float* targets, int rows, SurrogateBatch* B,
                     cudaStream_t st, bool reset_loss = true) {
  cudaError_t e = reset_loss ? cudaMemsetAsync(B->loss, 0, sizeof(double), st) : cudaSuccess;
  if (e == cudaSuccess) e = forward_hidden(s, theta, rows, B, true, st);
  if (e != cudaSuccess) return e;
  Gemm g = B->fwd[3];
  g.E.aux = targets;
  g.E.rows_valid = rows;
  g.E.scale = 2.0f / ((float)rows * (float)s->n_out);
  if ((e = srw::run_gemm(g, s->sm_count, s->d_status, st)) != cudaSuccess) return e;
  // output layer gradients, then down the hidden layers
  for (int l = 3; l >= 0 && e == cudaSuccess; --l) {
    e = srw::run_gemm(B->wgrad[l], s->sm_count, s->d_status, st);
    const __nv_bfloat16* dzt = l == 3 ? B->dyt : B->dzt[l];
    if (e == cudaSuccess) {
      srw::rowsum_kernel<<<(s->L[l].out + 7) / 8, 256, 0, st>>>(dzt, s->L[l].out, B->M, s->L[l].gb);
      e = srw::launch_result();
    }
    if (l > 0 && e == cudaSuccess) e = srw::run_gemm(B->bwd[l - 1], s->sm_count, s->d_status, st);
  }
  return e;
}

cudaError_t adam_update(srw_surrogate s, float lr, float beta1, float beta2, float eps, cudaStream_t st) {
  ++s->adam_t;
  srw::AdamArgs A{};
  long long off = 0;
  int n = 0;
  for (int l = 0; l < 4; ++l) {
    SurrogateLayer& L = s->L[l];
    A.L[n++] = srw::AdamLayer{L.w, L.gw, L.mw, L.vw, L.w_bf, L.wt_bf, L.out, L.in, off};
    off += (long long)L.out * L.in;
    A.L[n++] = srw::AdamLayer{L.b, L.gb, L.mb, L.vb, nullptr, nullptr, L.out, 1, off};
    off += L.out;
  }
  A.n_layers = n;
  A.total = off;
  A.lr = lr;
  A.beta1 = beta1;
  A.beta2 = beta2;
  A.eps = eps;
  A.c1 = (float)(1.0 - std::pow((double)beta1, (double)s->adam_t));
  A.c2 = (float)(1.0 - std::pow((double)beta2, (double)s->adam_t));
  srw::adam_kernel<<<(unsigned)((off + 255) / 256), 256, 0, st>>>(A);
  return srw::launch_result();
}

constexpr int kScanChunk = 1 << 20;  // points per surrogate launch chain in scans

// Surrogate -2 ln L of P points (device theta), written as T (double or float).
template <class T>
srw_status loglik_device(srw_surrogate s, const float* theta, long long P, T* out, cudaStream_t st) {
  srw::scan_consts_kernel<<<(s->n_out_pad + 255) / 256, 256, 0, st>>>(
      s->mean, s->stdv, s->L[3].b, reinterpret_cast<const float2*>(s->h->d_nb2), s->n_out, s->n_out_pad, s->binc);
  for (long long off = 0; off < P; off += kScanChunk) {
    const int rows = (int)std::min<long long>(kScanChunk, P - off);
    SurrogateBatch* B = nullptr;
    srw_status r = get_batch(s, round_up(rows, srw::kBM) < 65536 ? round_up(rows, srw::kBM) : round_up(rows, 65536), false, &B);
    if (r != SRW_OK) return r;
    cudaError_t e = forward_hidden(s, theta + off * 5, rows, B, false, st);
    if (e == cudaSuccess) {
      Gemm g = B->fwd_scan;
      g.E.rows_valid = rows;
      e = srw::run_gemm(g, s->sm_count, s->d_status, st);
    }
    if (e == cudaSuccess) {
      srw::scan_reduce_kernel<T><<<(rows + 255) / 256, 256, 0, st>>>(B->parts, s->n_out_pad / 256 * 2, rows, s->h->d_cdata,
                                                                   out + off);
      e = srw::launch_result();
    }
    if (e != cudaSuccess) return scuda(s, e, "surrogate likelihood");
  }
  return SRW_OK;
}

void box_of(srw_surrogate s, float4* lo0, float* lo4, float4* w0, float* w4) {
  *lo0 = make_float4(s->centre[0] - s->half[0], s->centre[1] - s->half[1], s->centre[2] - s->half[2],
                     s->centre[3] - s->half[3]);
  *lo4 = s->centre[4] - s->half[4];
  *w0 = make_float4(2.f * s->half[0], 2.f * s->half[1], 2.f * s->half[2], 2.f * s->half[3]);
  *w4 = 2.f * s->half[4];
}

srw_status check_status(srw_surrogate s, cudaStream_t st) {
  unsigned v = 0;
  S_CUDA(s, cudaMemcpyAsync(&v, s->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "status read");
  S_CUDA(s, cudaStreamSynchronize(st), "sync");
  if (v) S_CUDA(s, cudaMemsetAsync(s->d_status, 0, sizeof(unsigned), st), "status reset");
  if (v & srw::kStatusTimeout) return sfail(s, SRW_ETIMEOUT, "a bounded device wait expired; the kernel aborted");
  return SRW_OK;
}

srw_status upload_weights(srw_surrogate s, const float* const* w) {
  const int real_in[4] = {srw::kIn, srw::kHidden, srw::kHidden, srw::kHidden};
  const int real_out[4] = {srw::kHidden, srw::kHidden, srw::kHidden, s->n_out};
  for (int l = 0; l < 4; ++l) {
    SurrogateLayer& L = s->L[l];
    std::vector<float> W((size_t)L.out * L.in, 0.f), b(L.out, 0.f);
    for (int o = 0; o < real_out[l]; ++o) {
      for (int i = 0; i < real_in[l]; ++i) W[(size_t)o * L.in + i] = w[2 * l][(size_t)o * real_in[l] + i];
      b[o] = w[2 * l + 1][o];
    }
    for (float x : W)
      if (!std::isfinite(x)) return sfail(s, SRW_EINVAL, "weights must be finite");
    S_CUDA(s, cudaMemcpy(L.w, W.data(), sizeof(float) * W.size(), cudaMemcpyHostToDevice), "upload weights");
    S_CUDA(s, cudaMemcpy(L.b, b.data(), sizeof(float) * b.size(), cudaMemcpyHostToDevice), "upload biases");
    S_CUDA(s, cudaMemset(L.mw, 0, sizeof(float) * W.size()), "adam state");
    S_CUDA(s, cudaMemset(L.vw, 0, sizeof(float) * W.size()), "adam state");
    S_CUDA(s, cudaMemset(L.mb, 0, sizeof(float) * L.out), "adam state");
    S_CUDA(s, cudaMemset(L.vb, 0, sizeof(float) * L.out), "adam state");
    srw::cast_weights_kernel<<<(unsigned)((W.size() + 255) / 256), 256, 0, s->stream>>>(L.w, L.out, L.in, L.w_bf, L.wt_bf);
    S_CUDA(s, srw::launch_result(), "cast weights");
  }
  s->adam_t = 0;
  S_CUDA(s, cudaStreamSynchronize(s->stream), "sync");
  return SRW_OK;
}

}  // namespace

extern "C" {

srw_status srw_surrogate_create(srw_handle h, const float* centre, const float* half_width, const float* const* weights,
                                srw_surrogate* out) {
  if (!out) return SRW_EINVAL;
  *out = nullptr;
  if (!h || !centre || !half_width || !weights) return SRW_EINVAL;
  for (int k = 0; k < 8; ++k)
    if (!weights[k]) return SRW_EINVAL;
  for (int k = 0; k < 5; ++k)
    if (!std::isfinite(centre[k]) || !(half_width[k] > 0.f)) return SRW_EINVAL;
  if (!h->has_data || !h->tensor_ok) return SRW_EUNSUPPORTED;
  srw_surrogate s = new (std::nothrow) srw_surrogate_ctx();
  if (!s) return SRW_ENOMEM;
  s->h = h;
  s->device = h->device;
  s->sm_count = h->sm_count;
  s->n_out = h->n_rec;
  s->n_out_pad = round_up(h->n_rec, 256);
  for (int k = 0; k < 5; ++k) {
    s->centre[k] = centre[k];
    s->half[k] = half_width[k];
  }
  const int outs[4] = {srw::kHidden, srw::kHidden, srw::kHidden, s->n_out_pad};
  const int ins[4] = {srw::kInPad, srw::kHidden, srw::kHidden, srw::kHidden};
  cudaError_t e = cudaSetDevice(s->device);
  if (e == cudaSuccess) e = srw::gemm_attrs();
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = salloc(&s->d_status, 1);
  if (e == cudaSuccess) e = cudaMemset(s->d_status, 0, sizeof(unsigned));
  for (int l = 0; l < 4 && e == cudaSuccess; ++l) {
    SurrogateLayer& L = s->L[l];
    L.out = outs[l];
    L.in = ins[l];
    const size_t nw = (size_t)L.out * L.in;
    e = salloc(&L.w, nw);
    if (e == cudaSuccess) e = salloc(&L.b, L.out);
    if (e == cudaSuccess) e = salloc(&L.mw, nw);
    if (e == cudaSuccess) e = salloc(&L.vw, nw);
    if (e == cudaSuccess) e = salloc(&L.mb, L.out);
    if (e == cudaSuccess) e = salloc(&L.vb, L.out);
    if (e == cudaSuccess) e = salloc(&L.gw, nw);
    if (e == cudaSuccess) e = salloc(&L.gb, L.out);
    if (e == cudaSuccess) e = salloc(&L.w_bf, nw);
    if (e == cudaSuccess) e = salloc(&L.wt_bf, nw);
  }
  if (e == cudaSuccess) e = salloc(&s->mean, s->n_out_pad);
  if (e == cudaSuccess) e = salloc(&s->stdv, s->n_out_pad);
  if (e == cudaSuccess) e = salloc(&s->binc, s->n_out_pad);
  if (e == cudaSuccess) {  // identity standardization until training sets it
    std::vector<float> z(s->n_out_pad, 0.f), o(s->n_out_pad, 1.f);
    e = cudaMemcpy(s->mean, z.data(), sizeof(float) * z.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->stdv, o.data(), sizeof(float) * o.size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) {
    uint32_t V[5 * 32];
    sobol_directions(V);
    e = salloc(&s->d_sobol, 5 * 32);
    if (e == cudaSuccess) e = cudaMemcpy(s->d_sobol, V, sizeof(V), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    srw_surrogate_destroy(s);
    return e == cudaErrorMemoryAllocation ? SRW_ENOMEM : SRW_ECUDA;
  }
  const srw_status st = upload_weights(s, weights);
  if (st != SRW_OK) {
    srw_surrogate_destroy(s);
    return st;
  }
  *out = s;
  return SRW_OK;
}

srw_status srw_surrogate_set_weights(srw_surrogate s, const float* const* weights) {
  if (!s || !weights) return SRW_EINVAL;
  for (int k = 0; k < 8; ++k)
    if (!weights[k]) return sfail(s, SRW_EINVAL, "NULL weight array");
  return upload_weights(s, weights);
}

srw_status srw_surrogate_get_weights(srw_surrogate s, float* const* weights) {
  if (!s || !weights) return SRW_EINVAL;
  const int real_in[4] = {srw::kIn, srw::kHidden, srw::kHidden, srw::kHidden};
  const int real_out[4] = {srw::kHidden, srw::kHidden, srw::kHidden, s->n_out};
  S_CUDA(s, cudaStreamSynchronize(s->stream), "sync");
  for (int l = 0; l < 4; ++l) {
    const SurrogateLayer& L = s->L[l];
    std::vector<float> W((size_t)L.out * L.in), b(L.out);
    S_CUDA(s, cudaMemcpy(W.data(), L.w, sizeof(float) * W.size(), cudaMemcpyDeviceToHost), "read weights");
    S_CUDA(s, cudaMemcpy(b.data(), L.b, sizeof(float) * b.size(), cudaMemcpyDeviceToHost), "read biases");
    if (!weights[2 * l] || !weights[2 * l + 1]) return sfail(s, SRW_EINVAL, "NULL weight array");
    for (int o = 0; o < real_out[l]; ++o) {
      for (int i = 0; i < real_in[l]; ++i) weights[2 * l][(size_t)o * real_in[l] + i] = W[(size_t)o * L.in + i];
      weights[2 * l + 1][o] = b[o];
    }
  }
  return SRW_OK;
}

srw_status srw_surrogate_forward(srw_surrogate s, const float* theta, int P, float* y) {
  if (!s || !theta || !y || P < 1) return SRW_EINVAL;
  const int M = round_up(P, srw::kBM);
  SurrogateBatch* B = nullptr;
  srw_status st = get_batch(s, M, false, &B);
  if (st != SRW_OK) return st;
  CallBuf<float> th;
  S_CUDA(s, salloc_async(&th, (size_t)5 * P, s->stream), "alloc");
  float* d_th = th.p;
  S_CUDA(s, cudaMemcpyAsync(d_th, theta, sizeof(float) * 5 * (size_t)P, cudaMemcpyHostToDevice, s->stream), "upload");
  cudaError_t e = cudaSuccess;
  if (!B->y) {  // the FP32 output buffer exists only for this hook
    e = salloc(&B->y, (size_t)M * s->n_out_pad);
    B->fwd_out.E.out_f32 = B->y;
  }
  if (e == cudaSuccess) e = forward_hidden(s, d_th, P, B, false, s->stream);
  if (e == cudaSuccess) {
    Gemm g = B->fwd_out;
    g.E.rows_valid = P;
    e = srw::run_gemm(g, s->sm_count, s->d_status, s->stream);
  }
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(y, sizeof(float) * s->n_out, B->y, sizeof(float) * s->n_out_pad, sizeof(float) * s->n_out, P,
                          cudaMemcpyDeviceToHost, s->stream);
  if (e != cudaSuccess) return scuda(s, e, "surrogate forward");
  return check_status(s, s->stream);
}

srw_status srw_surrogate_gradients(srw_surrogate s, const float* theta, const float* targets, int P, float* const* grads,
                                   double* loss) {
  if (!s || !theta || !targets || !grads || P < 1) return SRW_EINVAL;
  const int M = round_up(P, srw::kBM);
  SurrogateBatch* B = nullptr;
  srw_status st = get_batch(s, M, true, &B);
  if (st != SRW_OK) return st;
  CallBuf<float> th, tg;
  S_CUDA(s, salloc_async(&th, (size_t)5 * P, s->stream), "alloc");
  S_CUDA(s, salloc_async(&tg, (size_t)M * s->n_out_pad, s->stream), "alloc");
  float *d_th = th.p, *d_t = tg.p;
  S_CUDA(s, cudaMemsetAsync(d_t, 0, sizeof(float) * (size_t)M * s->n_out_pad, s->stream), "zero");
  S_CUDA(s, cudaMemcpyAsync(d_th, theta, sizeof(float) * 5 * (size_t)P, cudaMemcpyHostToDevice, s->stream), "upload");
  S_CUDA(s, cudaMemcpy2DAsync(d_t, sizeof(float) * s->n_out_pad, targets, sizeof(float) * s->n_out,
                              sizeof(float) * s->n_out, P, cudaMemcpyHostToDevice, s->stream),
         "upload targets");
  cudaError_t e = fit_pass(s, d_th, d_t, P, B, s->stream);
  double sse = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&sse, B->loss, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return scuda(s, e, "surrogate gradients");
  st = check_status(s, s->stream);
  if (st != SRW_OK) return st;
  if (loss) *loss = sse / ((double)P * s->n_out);
  const int real_in[4] = {srw::kIn, srw::kHidden, srw::kHidden, srw::kHidden};
  const int real_out[4] = {srw::kHidden, srw::kHidden, srw::kHidden, s->n_out};
  for (int l = 0; l < 4; ++l) {
    const SurrogateLayer& L = s->L[l];
    std::vector<float> g((size_t)L.out * L.in), gb(L.out);
    S_CUDA(s, cudaMemcpy(g.data(), L.gw, sizeof(float) * g.size(), cudaMemcpyDeviceToHost), "read gradients");
    S_CUDA(s, cudaMemcpy(gb.data(), L.gb, sizeof(float) * gb.size(), cudaMemcpyDeviceToHost), "read gradients");
    if (!grads[2 * l] || !grads[2 * l + 1]) return sfail(s, SRW_EINVAL, "NULL gradient array");
    for (int o = 0; o < real_out[l]; ++o) {
      for (int i = 0; i < real_in[l]; ++i) grads[2 * l][(size_t)o * real_in[l] + i] = g[(size_t)o * L.in + i];
      grads[2 * l + 1][o] = gb[o];
    }
  }
  return SRW_OK;
}

srw_status srw_surrogate_train_step(srw_surrogate s, const float* theta, const float* targets, int P, float lr,
                                    double* loss) {
  if (!s || !theta || !targets || P < 1 || !(lr > 0.f)) return SRW_EINVAL;
  const int M = round_up(P, srw::kBM);
  SurrogateBatch* B = nullptr;
  srw_status st = get_batch(s, M, true, &B);
  if (st != SRW_OK) return st;
  CallBuf<float> th, tg;
  S_CUDA(s, salloc_async(&th, (size_t)5 * P, s->stream), "alloc");
  S_CUDA(s, salloc_async(&tg, (size_t)M * s->n_out_pad, s->stream), "alloc");
  float *d_th = th.p, *d_t = tg.p;
  S_CUDA(s, cudaMemsetAsync(d_t, 0, sizeof(float) * (size_t)M * s->n_out_pad, s->stream), "zero");
  S_CUDA(s, cudaMemcpyAsync(d_th, theta, sizeof(float) * 5 * (size_t)P, cudaMemcpyHostToDevice, s->stream), "upload");
  S_CUDA(s, cudaMemcpy2DAsync(d_t, sizeof(float) * s->n_out_pad, targets, sizeof(float) * s->n_out,
                              sizeof(float) * s->n_out, P, cudaMemcpyHostToDevice, s->stream),
         "upload targets");
  cudaError_t e = fit_pass(s, d_th, d_t, P, B, s->stream);
  if (e == cudaSuccess) e = adam_update(s, lr, 0.9f, 0.999f, 1e-8f, s->stream);
  double sse = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&sse, B->loss, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return scuda(s, e, "surrogate train step");
  if (loss) *loss = sse / ((double)P * s->n_out);
  return check_status(s, s->stream);
}

static srw_status fit_impl(srw_surrogate s, const float* theta, long long n, const srw_fit_opts* o, int first_epoch,
                           int stop_epoch, const char* checkpoint_path, float* epoch_loss) {
  if (!s || !theta || !o || n < 1) return SRW_EINVAL;
  if (stop_epoch <= 0) stop_epoch = o->epochs;
  if (first_epoch < 0 || stop_epoch > o->epochs || first_epoch > stop_epoch)
    return sfail(s, SRW_EINVAL, "need 0 <= first_epoch <= stop_epoch <= epochs");
  if (o->batch < srw::kBM || o->batch % srw::kBM || o->epochs < 0 || !(o->lr > 0.f) || !(o->lr_final >= 0.f))
    return sfail(s, SRW_EINVAL, "batch must be a positive multiple of 128; epochs >= 0; lr > 0");
  if (o->precision < SRW_FP32 || o->precision > SRW_FP16X3) return sfail(s, SRW_EINVAL, "bad precision");
  if (!srw::all_finite(theta, (size_t)(n * 5))) return sfail(s, SRW_EINVAL, "theta must be finite");
  srw_ctx* h = s->h;
  cudaStream_t st = s->stream;
  const int M = o->batch, NO = s->n_out_pad, NR = s->n_out;
  const long long steps = (n + M - 1) / M, n_pad = steps * M;
  constexpr int kGen = 65536;  // training spectra per exact-path launch
  float *d_th = nullptr, *d_t = nullptr, *d_tmp = nullptr;
  double* d_stats = nullptr;
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    sfree(d_th);
    sfree(d_t);
    sfree(d_tmp);
    sfree(d_stats);
  };
  cudaError_t e = salloc(&d_th, (size_t)n_pad * 5);
  if (e == cudaSuccess) e = salloc(&d_t, (size_t)n_pad * NO);
  if (e == cudaSuccess) e = salloc(&d_tmp, (size_t)kGen * NR);
  const int n_sblocks = (int)((n + 4095) / 4096);
  if (e == cudaSuccess) e = salloc(&d_stats, 2 * (size_t)NR * n_sblocks);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_th, 0, sizeof(float) * n_pad * 5, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_t, 0, sizeof(float) * n_pad * NO, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_th, theta, sizeof(float) * n * 5, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    cleanup();
    return scuda(s, e, "training buffers");
  }
  // targets: log of the exact expected counts (signal of the exact path + background)
  for (long long off = 0; off < n; off += kGen) {
    const int cnt = (int)std::min<long long>(kGen, n - off);
    const srw_status r = srw_spectrum_batch(h, d_th + off * 5, cnt, d_tmp, SRW_DEVICE, (srw_precision)o->precision, st);
    if (r != SRW_OK) {
      cleanup();
      return sfail(s, r, std::string("exact spectra: ") + srw_last_error(h));
    }
    srw::log_counts_kernel<<<(unsigned)(((long long)cnt * NO + 255) / 256), 256, 0, st>>>(d_tmp, cnt, NR, NO, h->d_b64,
                                                                                      d_t + off * NO);
  }
  // per-bin standardization over the training set
  srw::colstats_kernel<<<dim3((NR + 255) / 256, (unsigned)n_sblocks), 256, 0, st>>>(
      d_t, n, NO, NR, d_stats, d_stats + (size_t)NR * n_sblocks);
  srw::finish_stats_kernel<<<(NR + 255) / 256, 256, 0, st>>>(d_stats, d_stats + (size_t)NR * n_sblocks, n_sblocks, n,
                                                             NR, s->mean, s->stdv);
  srw::standardize_kernel<<<(unsigned)((n * NO + 255) / 256), 256, 0, st>>>(d_t, n, NO, NR, s->mean, s->stdv);
  if ((e = srw::launch_result()) != cudaSuccess) {
    cleanup();
    return scuda(s, e, "targets");
  }
  SurrogateBatch* B = nullptr;
  srw_status r = get_batch(s, M, true, &B);
  if (r != SRW_OK) {
    cleanup();
    return r;
  }
  const long long total = steps * o->epochs;
  long long t = steps * first_epoch;  // a resumed fit continues the learning-rate schedule
  for (int ep = first_epoch; ep < stop_epoch; ++ep) {
    e = cudaMemsetAsync(B->loss, 0, sizeof(double), st);
    for (long long b = 0; b < steps && e == cudaSuccess; ++b, ++t) {
      const int rows = (int)std::min<long long>(M, n - b * M);
      const double frac = total > 1 ? (double)t / (double)(total - 1) : 0.0;
      const float lr = (float)(o->lr_final + 0.5 * (o->lr - o->lr_final) * (1.0 + std::cos(3.141592653589793 * frac)));
      e = fit_pass(s, d_th + b * M * 5, d_t + b * M * NO, rows, B, st, false);
      if (e == cudaSuccess) e = adam_update(s, lr, 0.9f, 0.999f, 1e-8f, st);
    }
    double sse = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&sse, B->loss, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      cleanup();
      return scuda(s, e, "training");
    }
    // each step's error is already a mean over its own points: average the steps
    if (epoch_loss) epoch_loss[ep] = (float)(sse / ((double)n * NR));
    s->epochs_done = ep + 1;
    s->stats_ready = 1;
    if (checkpoint_path) {
      const srw_status cr = srw_surrogate_save(s, checkpoint_path);
      if (cr != SRW_OK) {
        cleanup();
        return cr;
      }
    }
  }
  cleanup();
  s->stats_ready = 1;
  return check_status(s, st);
}

srw_status srw_surrogate_fit(srw_surrogate s, const float* theta, long long n, const srw_fit_opts* o,
                             float* epoch_loss) {
  if (s) s->epochs_done = 0;
  return fit_impl(s, theta, n, o, 0, 0, nullptr, epoch_loss);
}

srw_status srw_surrogate_fit_resume(srw_surrogate s, const float* theta, long long n, const srw_fit_opts* o,
                                    int first_epoch, int stop_epoch, const char* checkpoint_path, float* epoch_loss) {
  return fit_impl(s, theta, n, o, first_epoch, stop_epoch, checkpoint_path, epoch_loss);
}

srw_status srw_surrogate_loglik(srw_surrogate s, const float* theta, int P, double* out, int where, void* stream) {
  if (!s || !theta || !out || P < 1) return SRW_EINVAL;
  if (where != SRW_HOST && where != SRW_DEVICE) return sfail(s, SRW_EINVAL, "where must be SRW_HOST or SRW_DEVICE");
  cudaStream_t st = stream ? (cudaStream_t)stream : s->stream;
  if (where == SRW_DEVICE) {
    srw_status r = loglik_device<double>(s, theta, P, out, st);
    if (r == SRW_OK && !stream) S_CUDA(s, cudaStreamSynchronize(st), "sync");
    return r;
  }
  if (!srw::all_finite(theta, (size_t)((long long)P * 5))) return sfail(s, SRW_EINVAL, "theta must be finite");
  CallBuf<float> th;
  CallBuf<double> vo;
  S_CUDA(s, salloc_async(&th, (size_t)5 * P, st), "alloc");
  S_CUDA(s, salloc_async(&vo, (size_t)P, st), "alloc");
  float* d_th = th.p;
  double* d_out = vo.p;
  S_CUDA(s, cudaMemcpyAsync(d_th, theta, sizeof(float) * 5 * (size_t)P, cudaMemcpyHostToDevice, st), "upload");
  srw_status r = loglik_device<double>(s, d_th, P, d_out, st);
  if (r == SRW_OK)
    S_CUDA(s, cudaMemcpyAsync(out, d_out, sizeof(double) * (size_t)P, cudaMemcpyDeviceToHost, st), "download");
  if (r != SRW_OK) return r;
  return check_status(s, st);
}

srw_status srw_surrogate_scan_exact(srw_surrogate s, long long first, long long n_points, int precision,
                                    double* best_value, long long* best_index, float* ms) {
  if (!s || n_points < 1 || first < 0) return SRW_EINVAL;
  if (precision != SRW_RANK8 && (precision < SRW_FP32 || precision > SRW_FP16X3)) return SRW_EINVAL;
  cudaStream_t st = s->stream;
  constexpr int kChunk = 65536;
  float4 lo0, w0;
  float lo4, w4;
  box_of(s, &lo0, &lo4, &w0, &w4);
  CallBuf<float> b_th;
  CallBuf<double> b_v, b_o;
  CallBuf<unsigned long long> b_best;
  S_CUDA(s, salloc(&b_th, (size_t)kChunk * 5), "alloc");
  S_CUDA(s, salloc(&b_v, (size_t)n_points), "alloc");
  S_CUDA(s, salloc(&b_o, (size_t)kChunk), "alloc");
  S_CUDA(s, salloc(&b_best, 2), "alloc");
  float* d_th = b_th.p;
  double *d_v = b_v.p, *d_o = b_o.p;
  unsigned long long* d_best = b_best.p;
  CallEvents<2> ev;
  cudaEvent_t e0 = ev.e[0], e1 = ev.e[1];
  cudaEventRecord(e0, st);
  srw_status r = SRW_OK;
  for (long long off = 0; off < n_points && r == SRW_OK; off += kChunk) {
    const int cnt = (int)std::min<long long>(kChunk, n_points - off);
    srw::sobol_kernel<<<(cnt + 255) / 256, 256, 0, st>>>(s->d_sobol, first + off, cnt, lo0, lo4, w0, w4, d_th);
    // fixed input and output buffers: the exact path replays one captured graph per chunk size
    r = precision == SRW_RANK8 ? srw_loglik_linear(s->h, d_th, cnt, d_o, nullptr, SRW_DEVICE, st)
                               : srw_loglik(s->h, d_th, cnt, d_o, SRW_DEVICE, (srw_precision)precision, st);
    if (r == SRW_OK && cudaMemcpyAsync(d_v + off, d_o, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      r = SRW_ECUDA;
  }
  const unsigned long long init[2] = {~0ull, ~0ull};
  cudaMemcpyAsync(d_best, init, sizeof(init), cudaMemcpyHostToDevice, st);
  srw::min_bits_kernel<double><<<1024, 256, 0, st>>>(d_v, n_points, d_best);
  srw::argmin_kernel<double><<<1024, 256, 0, st>>>(d_v, n_points, d_best, d_best + 1);
  cudaEventRecord(e1, st);
  unsigned long long res[2] = {0, 0};
  cudaError_t e = cudaMemcpyAsync(res, d_best, sizeof(res), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  if (r != SRW_OK) return sfail(s, r, std::string("exact scan: ") + srw_last_error(s->h));
  if (e != cudaSuccess) return scuda(s, e, "exact scan");
  double v;
  const long long bits = (long long)res[0];
  std::memcpy(&v, &bits, sizeof(v));
  if (best_value) *best_value = v;
  if (best_index) *best_index = first + (long long)res[1];
  if (ms) *ms = t;
  return check_status(s, st);
}

namespace {

// Exact -2 ln L of the points with the listed Sobol indices; returns the
// minimum and the index of the point that attains it (index -1 if count = 0).
srw_status exact_min_of(srw_surrogate s, const long long* d_idx, long long count, int precision, float4 lo0, float lo4,
                        float4 w0, float w4, float* d_th, double* d_o, double* best_value, long long* best_index) {
  cudaStream_t st = s->stream;
  constexpr int kChunk = 65536;
  *best_value = INFINITY;
  *best_index = -1;
  if (count <= 0) return SRW_OK;
  CallBuf<double> b_ex;
  CallBuf<unsigned long long> b_best;
  S_CUDA(s, salloc(&b_ex, (size_t)count), "alloc");
  S_CUDA(s, salloc(&b_best, 2), "alloc");
  double* d_ex = b_ex.p;
  unsigned long long* d_best = b_best.p;
  srw_status r = SRW_OK;
  for (long long off = 0; off < count && r == SRW_OK; off += kChunk) {
    const int cnt = (int)std::min<long long>(kChunk, count - off);
    srw::sobol_gather_kernel<<<(cnt + 255) / 256, 256, 0, st>>>(s->d_sobol, d_idx + off, cnt, lo0, lo4, w0, w4, d_th);
    r = srw_loglik(s->h, d_th, cnt, d_o, SRW_DEVICE, (srw_precision)precision, st);
    if (r == SRW_OK && cudaMemcpyAsync(d_ex + off, d_o, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      r = SRW_ECUDA;
  }
  unsigned long long best[2] = {~0ull, ~0ull};
  cudaError_t e = cudaSuccess;
  if (r == SRW_OK) {
    e = cudaMemcpyAsync(d_best, best, sizeof(best), cudaMemcpyHostToDevice, st);
    srw::min_bits_kernel<double><<<1024, 256, 0, st>>>(d_ex, count, d_best);
    srw::argmin_kernel<double><<<1024, 256, 0, st>>>(d_ex, count, d_best, d_best + 1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(best, d_best, sizeof(best), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpy(best_index, d_idx + best[1], sizeof(long long), cudaMemcpyDeviceToHost);
  }
  cudaStreamSynchronize(st);
  if (r != SRW_OK) return sfail(s, r, std::string("exact re-evaluation: ") + srw_last_error(s->h));
  if (e != cudaSuccess) return scuda(s, e, "exact re-evaluation");
  const long long bits = (long long)best[0];
  std::memcpy(best_value, &bits, sizeof(double));
  return SRW_OK;
}

}  // namespace

srw_status srw_surrogate_scan(srw_surrogate s, const srw_scan_opts* o, srw_scan_result* res) {
  if (!s || !o || !res) return SRW_EINVAL;
  if (o->n_points < 1 || o->first < 0 || !(o->keep_frac > 0.0 && o->keep_frac <= 1.0) || o->n_check < 0 ||
      (o->n_check > 0 && !o->check_theta) || o->cells_per_dim < 1 || o->cells_per_dim > 16 || !(o->tol >= 0.0) ||
      (o->rule != SRW_SCAN_FLAG_CELLS && o->rule != SRW_SCAN_ERROR_BARS) || !(o->margin_factor >= 1.0))
    return sfail(s, SRW_EINVAL, "bad scan options");
  std::memset(res, 0, sizeof(*res));
  cudaStream_t st = s->stream;
  const int cpd = o->cells_per_dim;
  const int n_cells = cpd * cpd * cpd * cpd * cpd;
  res->n_cells = n_cells;
  float4 lo0, w0;
  float lo4, w4;
  box_of(s, &lo0, &lo4, &w0, &w4);
  CallEvents<5> evs;
  cudaEvent_t* ev = evs.e;
  cudaEventRecord(ev[0], st);
  // ---- held-out check: both paths on the check points; per-cell largest |d|
  std::vector<double> cmax(n_cells, -1.0);  // -1: no check point in the cell
  if (o->n_check > 0) {
    CallBuf<float> b_c;
    CallBuf<double> b_ex, b_su;
    S_CUDA(s, salloc(&b_c, (size_t)o->n_check * 5), "alloc");
    S_CUDA(s, salloc(&b_ex, (size_t)o->n_check), "alloc");
    S_CUDA(s, salloc(&b_su, (size_t)o->n_check), "alloc");
    float* d_c = b_c.p;
    double *d_ex = b_ex.p, *d_su = b_su.p;
    S_CUDA(s, cudaMemcpyAsync(d_c, o->check_theta, sizeof(float) * 5 * o->n_check, cudaMemcpyHostToDevice, st), "upload");
    srw_status r = srw_loglik(s->h, d_c, o->n_check, d_ex, SRW_DEVICE, (srw_precision)o->precision, st);
    if (r == SRW_OK) r = loglik_device<double>(s, d_c, o->n_check, d_su, st);
    std::vector<double> ex(o->n_check), su(o->n_check);
    if (r == SRW_OK) {
      cudaMemcpyAsync(ex.data(), d_ex, sizeof(double) * o->n_check, cudaMemcpyDeviceToHost, st);
      cudaMemcpyAsync(su.data(), d_su, sizeof(double) * o->n_check, cudaMemcpyDeviceToHost, st);
      cudaStreamSynchronize(st);
    }
    if (r != SRW_OK) return r;
    for (int i = 0; i < o->n_check; ++i) {
      const float* th = o->check_theta + (size_t)i * 5;
      const float u[5] = {(th[0] - lo0.x) / w0.x, (th[1] - lo0.y) / w0.y, (th[2] - lo0.z) / w0.z, (th[3] - lo0.w) / w0.w,
                          (th[4] - lo4) / w4};
      int c = 0;
      for (int d = 4; d >= 0; --d) {
        int k = (int)std::floor(u[d] * (float)cpd);
        k = k < 0 ? 0 : (k >= cpd ? cpd - 1 : k);
        c = c * cpd + k;
      }
      const double dd = std::isfinite(ex[i]) && std::isfinite(su[i]) ? std::fabs(su[i] - ex[i]) : INFINITY;
      cmax[c] = std::max(cmax[c], dd);
      res->check_max_abs_d = std::max(res->check_max_abs_d, dd);
    }
  }
  for (int c = 0; c < n_cells; ++c)
    if (o->n_check > 0 && (cmax[c] < 0.0 || cmax[c] > o->tol)) ++res->n_flagged_cells;
  cudaEventRecord(ev[1], st);
  // ---- surrogate values of every scan point
  CallBuf<float> b_vals, b_th;
  CallBuf<double> b_o;
  S_CUDA(s, salloc(&b_vals, (size_t)o->n_points), "alloc scan values");
  S_CUDA(s, salloc(&b_th, (size_t)kScanChunk * 5), "alloc");
  S_CUDA(s, salloc(&b_o, 65536), "alloc");
  float* d_vals = b_vals.p;
  float* d_th = b_th.p;
  double* d_o = b_o.p;
  for (long long off = 0; off < o->n_points; off += kScanChunk) {
    const int cnt = (int)std::min<long long>(kScanChunk, o->n_points - off);
    srw::sobol_kernel<<<(cnt + 255) / 256, 256, 0, st>>>(s->d_sobol, o->first + off, cnt, lo0, lo4, w0, w4, d_th);
    const srw_status r = loglik_device<float>(s, d_th, cnt, d_vals + off, st);
    if (r != SRW_OK) return r;
  }
  cudaEventRecord(ev[2], st);
  // ---- threshold of the lowest keep_frac (exact radix selection on the float bits)
  const long long k = std::max<long long>(1, (long long)std::ceil(o->keep_frac * (double)o->n_points));
  CallBuf<unsigned> b_hist;
  CallBuf<unsigned long long> b_cnt;
  CallBuf<long long> b_idx;
  CallBuf<float> b_margin;
  S_CUDA(s, salloc(&b_hist, 65536), "alloc");
  S_CUDA(s, salloc(&b_cnt, 3), "alloc");
  S_CUDA(s, salloc(&b_idx, (size_t)o->n_points), "alloc index list");
  S_CUDA(s, salloc(&b_margin, (size_t)n_cells), "alloc");
  unsigned* d_hist = b_hist.p;
  unsigned long long* d_cnt = b_cnt.p;
  long long* d_idx = b_idx.p;
  float* d_margin = b_margin.p;
  std::vector<unsigned> hist(65536);
  S_CUDA(s, cudaMemsetAsync(d_hist, 0, sizeof(unsigned) * 65536, st), "zero");
  srw::hist_hi_kernel<<<1024, 256, 0, st>>>(d_vals, o->n_points, d_hist);
  S_CUDA(s, cudaMemcpyAsync(hist.data(), d_hist, sizeof(unsigned) * 65536, cudaMemcpyDeviceToHost, st), "hist");
  S_CUDA(s, cudaStreamSynchronize(st), "sync");
  long long cum = 0;
  unsigned hi = 0;
  for (; hi < 65535; ++hi) {
    if (cum + hist[hi] >= k) break;
    cum += hist[hi];
  }
  S_CUDA(s, cudaMemsetAsync(d_hist, 0, sizeof(unsigned) * 65536, st), "zero");
  srw::hist_lo_kernel<<<1024, 256, 0, st>>>(d_vals, o->n_points, hi, d_hist);
  S_CUDA(s, cudaMemcpyAsync(hist.data(), d_hist, sizeof(unsigned) * 65536, cudaMemcpyDeviceToHost, st), "hist");
  S_CUDA(s, cudaStreamSynchronize(st), "sync");
  unsigned lo = 0;
  for (; lo < 65535; ++lo) {
    if (cum + hist[lo] >= k) break;
    cum += hist[lo];
  }
  const unsigned tbits = (hi << 16) | lo;
  float thresh;
  std::memcpy(&thresh, &tbits, sizeof(thresh));
  res->n_kept = cum + hist[lo];
  // per-cell margins: SRW_SCAN_FLAG_CELLS keeps whole flagged cells (+inf);
  // SRW_SCAN_ERROR_BARS uses margin_factor x max(held-out |d|, tol), +inf where
  // a cell holds no check point
  std::vector<float> margin(n_cells);
  for (int c = 0; c < n_cells; ++c) {
    const bool flagged = cmax[c] < 0.0 || cmax[c] > o->tol;
    if (o->rule == SRW_SCAN_FLAG_CELLS) margin[c] = flagged && o->n_check > 0 ? INFINITY : -INFINITY;
    else margin[c] = cmax[c] < 0.0 ? INFINITY : (float)(o->margin_factor * std::max(cmax[c], o->tol));
  }
  S_CUDA(s, cudaMemcpyAsync(d_margin, margin.data(), sizeof(float) * n_cells, cudaMemcpyHostToDevice, st), "upload");
  // surrogate minimum (for the report)
  const unsigned long long init3[3] = {0ull, ~0ull, ~0ull};
  S_CUDA(s, cudaMemcpyAsync(d_cnt, init3, sizeof(init3), cudaMemcpyHostToDevice, st), "init");
  srw::min_bits_kernel<float><<<1024, 256, 0, st>>>(d_vals, o->n_points, d_cnt + 1);
  // pass 1: the lowest keep_frac (+ whole flagged cells under SRW_SCAN_FLAG_CELLS)
  const bool cells = o->rule == SRW_SCAN_FLAG_CELLS;
  srw::select_kernel<<<2048, 256, 0, st>>>(d_vals, s->d_sobol, o->first, o->n_points, thresh, thresh,
                                           cells ? d_margin : nullptr, 0.f, cpd, lo0, lo4, w0, w4, d_idx, d_cnt,
                                           o->n_points);
  unsigned long long sel[2] = {0, 0};
  S_CUDA(s, cudaMemcpyAsync(sel, d_cnt, sizeof(sel), cudaMemcpyDeviceToHost, st), "count");
  S_CUDA(s, cudaStreamSynchronize(st), "sync");
  {
    const unsigned bsur = (unsigned)sel[1];
    float f;
    std::memcpy(&f, &bsur, sizeof(f));
    res->surrogate_min = f;
  }
  long long n_sel = std::min<long long>((long long)sel[0], o->n_points);
  cudaEventRecord(ev[3], st);
  double best = INFINITY;
  long long best_index = -1;
  srw_status r = exact_min_of(s, d_idx, n_sel, o->precision, lo0, lo4, w0, w4, d_th, d_o, &best, &best_index);
  if (r == SRW_OK && !cells) {
    // pass 2: points outside pass 1 that could still beat the best exact value
    // within their cell's error bar
    S_CUDA(s, cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), st), "zero");
    srw::select_kernel<<<2048, 256, 0, st>>>(d_vals, s->d_sobol, o->first, o->n_points, -1.f, thresh, d_margin,
                                             (float)best, cpd, lo0, lo4, w0, w4, d_idx, d_cnt, o->n_points);
    unsigned long long n2 = 0;
    S_CUDA(s, cudaMemcpyAsync(&n2, d_cnt, sizeof(n2), cudaMemcpyDeviceToHost, st), "count");
    S_CUDA(s, cudaStreamSynchronize(st), "sync");
    res->n_rescued = std::min<long long>((long long)n2, o->n_points);
    double b2 = INFINITY;
    long long i2 = -1;
    r = exact_min_of(s, d_idx, res->n_rescued, o->precision, lo0, lo4, w0, w4, d_th, d_o, &b2, &i2);
    if (b2 < best || (b2 == best && i2 >= 0 && i2 < best_index)) {
      best = b2;
      best_index = i2;
    }
    n_sel += res->n_rescued;
  }
  cudaEventRecord(ev[4], st);
  cudaStreamSynchronize(st);
  float t[4] = {0, 0, 0, 0};
  for (int i = 0; i < 4; ++i) cudaEventElapsedTime(&t[i], ev[i], ev[i + 1]);
  if (r != SRW_OK) return r;
  res->n_selected = n_sel;
  res->ms_check = t[0];
  res->ms_surrogate = t[1];
  res->ms_select = t[2];
  res->ms_exact = t[3];
  res->best_value = best;
  res->best_index = best_index;
  if (best_index >= 0) {  // the point itself, from its sequence index (host, same construction)
    uint32_t V[5 * 32];
    sobol_directions(V);
    unsigned long long gcode = (unsigned long long)best_index ^ ((unsigned long long)best_index >> 1);
    uint32_t x[5] = {0, 0, 0, 0, 0};
    for (int kk = 0; gcode && kk < 32; ++kk, gcode >>= 1)
      if (gcode & 1ull)
        for (int d = 0; d < 5; ++d) x[d] ^= V[d * 32 + kk];
    const float lo5[5] = {lo0.x, lo0.y, lo0.z, lo0.w, lo4}, w5[5] = {w0.x, w0.y, w0.z, w0.w, w4};
    for (int d = 0; d < 5; ++d) res->best_theta[d] = lo5[d] + w5[d] * ((float)x[d] * 2.3283064365386963e-10f);
  }
  return check_status(s, st);
}

srw_status srw_surrogate_sobol(srw_surrogate s, long long first, int count, float* theta) {
  if (!s || !theta || count < 1 || first < 0) return SRW_EINVAL;
  float4 lo0, w0;
  float lo4, w4;
  box_of(s, &lo0, &lo4, &w0, &w4);
  float* d = nullptr;
  S_CUDA(s, salloc(&d, (size_t)count * 5), "alloc");
  srw::sobol_kernel<<<(count + 255) / 256, 256, 0, s->stream>>>(s->d_sobol, first, count, lo0, lo4, w0, w4, d);
  cudaError_t e = cudaMemcpyAsync(theta, d, sizeof(float) * 5 * (size_t)count, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  sfree(d);
  if (e != cudaSuccess) return scuda(s, e, "sobol points");
  return SRW_OK;
}

srw_status srw_surrogate_get_standardization(srw_surrogate s, float* mean, float* stdv) {
  if (!s || !mean || !stdv) return SRW_EINVAL;
  S_CUDA(s, cudaStreamSynchronize(s->stream), "sync");
  S_CUDA(s, cudaMemcpy(mean, s->mean, sizeof(float) * s->n_out, cudaMemcpyDeviceToHost), "read");
  S_CUDA(s, cudaMemcpy(stdv, s->stdv, sizeof(float) * s->n_out, cudaMemcpyDeviceToHost), "read");
  return SRW_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Checkpoints: the whole training state (FP32 master weights and biases, Adam
// first and second moments and step count, the per-bin standardization and
// the completed epochs), written to `path + ".tmp"` and renamed over `path`,
// so that a crash leaves either the previous or the new checkpoint.  Binary,
// little-endian, with a 64-bit FNV-1a checksum of the payload.
// ---------------------------------------------------------------------------
namespace {

struct CkptHeader {
  char magic[8];
  int32_t version, n_out, n_out_pad, stats_ready;
  int64_t adam_t, epochs_done;
  float centre[5], half[5];
  int32_t out[4], in[4];
  uint64_t payload_bytes, checksum;
};
constexpr char kCkptMagic[8] = {'S', 'R', 'W', 'C', 'K', 'P', 'T', '1'};

uint64_t fnv1a(const std::vector<unsigned char>& b) {
  uint64_t h = 1469598103934665603ull;
  for (unsigned char c : b) {
    h ^= c;
    h *= 1099511628211ull;
  }
  return h;
}

// The device arrays of the training state in file order, with their lengths.
std::vector<std::pair<float*, size_t>> state_arrays(srw_surrogate s) {
  std::vector<std::pair<float*, size_t>> a;
  for (SurrogateLayer& L : s->L) {
    const size_t nw = (size_t)L.out * L.in;
    a.push_back({L.w, nw});
    a.push_back({L.b, (size_t)L.out});
    a.push_back({L.mw, nw});
    a.push_back({L.vw, nw});
    a.push_back({L.mb, (size_t)L.out});
    a.push_back({L.vb, (size_t)L.out});
  }
  a.push_back({s->mean, (size_t)s->n_out_pad});
  a.push_back({s->stdv, (size_t)s->n_out_pad});
  return a;
}

}  // namespace

extern "C" {

srw_status srw_surrogate_save(srw_surrogate s, const char* path) {
  if (!s || !path) return SRW_EINVAL;
  S_CUDA(s, cudaStreamSynchronize(s->stream), "sync");
  CkptHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, kCkptMagic, 8);
  hd.version = 1;
  hd.n_out = s->n_out;
  hd.n_out_pad = s->n_out_pad;
  hd.stats_ready = s->stats_ready;
  hd.adam_t = s->adam_t;
  hd.epochs_done = s->epochs_done;
  for (int k = 0; k < 5; ++k) {
    hd.centre[k] = s->centre[k];
    hd.half[k] = s->half[k];
  }
  for (int l = 0; l < 4; ++l) {
    hd.out[l] = s->L[l].out;
    hd.in[l] = s->L[l].in;
  }
  std::vector<unsigned char> payload;
  for (auto& a : state_arrays(s)) {
    const size_t off = payload.size();
    payload.resize(off + a.second * sizeof(float));
    S_CUDA(s, cudaMemcpy(payload.data() + off, a.first, a.second * sizeof(float), cudaMemcpyDeviceToHost), "read state");
  }
  hd.payload_bytes = payload.size();
  hd.checksum = fnv1a(payload);
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return sfail(s, SRW_EINVAL, "cannot write checkpoint " + tmp);
  const bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1 &&
                  std::fwrite(payload.data(), 1, payload.size(), f) == payload.size() && std::fflush(f) == 0;
  if (std::fclose(f) != 0 || !ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return sfail(s, SRW_EINVAL, std::string("cannot write checkpoint ") + path);
  }
  return SRW_OK;
}

srw_status srw_surrogate_load(srw_surrogate s, const char* path, long long* epochs_done) {
  if (!s || !path) return SRW_EINVAL;
  FILE* f = std::fopen(path, "rb");
  if (!f) return sfail(s, SRW_EINVAL, std::string("cannot read checkpoint ") + path);
  CkptHeader hd;
  std::vector<unsigned char> payload;
  bool ok = std::fread(&hd, sizeof(hd), 1, f) == 1 && std::memcmp(hd.magic, kCkptMagic, 8) == 0 && hd.version == 1;
  if (ok && hd.payload_bytes < ((uint64_t)1 << 34)) {
    payload.resize(hd.payload_bytes);
    ok = std::fread(payload.data(), 1, payload.size(), f) == payload.size();
  } else {
    ok = false;
  }
  std::fclose(f);
  if (!ok) return sfail(s, SRW_EINVAL, std::string("not a surrogate checkpoint: ") + path);
  if (fnv1a(payload) != hd.checksum) return sfail(s, SRW_EINVAL, std::string("checkpoint checksum mismatch: ") + path);
  bool same = hd.n_out == s->n_out && hd.n_out_pad == s->n_out_pad;
  for (int l = 0; l < 4; ++l) same = same && hd.out[l] == s->L[l].out && hd.in[l] == s->L[l].in;
  for (int k = 0; k < 5; ++k) same = same && hd.centre[k] == s->centre[k] && hd.half[k] == s->half[k];
  if (!same) return sfail(s, SRW_EINVAL, "checkpoint of a different network or parameter box");
  size_t want = 0;
  for (auto& a : state_arrays(s)) want += a.second * sizeof(float);
  if (want != payload.size()) return sfail(s, SRW_EINVAL, "checkpoint size does not match the network");
  S_CUDA(s, cudaStreamSynchronize(s->stream), "sync");
  size_t off = 0;
  for (auto& a : state_arrays(s)) {
    S_CUDA(s, cudaMemcpy(a.first, payload.data() + off, a.second * sizeof(float), cudaMemcpyHostToDevice), "upload state");
    off += a.second * sizeof(float);
  }
  for (SurrogateLayer& L : s->L)
    srw::cast_weights_kernel<<<(unsigned)(((size_t)L.out * L.in + 255) / 256), 256, 0, s->stream>>>(L.w, L.out, L.in,
                                                                                                  L.w_bf, L.wt_bf);
  S_CUDA(s, srw::launch_result(), "cast weights");
  S_CUDA(s, cudaStreamSynchronize(s->stream), "sync");
  s->adam_t = hd.adam_t;
  s->epochs_done = hd.epochs_done;
  s->stats_ready = hd.stats_ready;
  if (epochs_done) *epochs_done = hd.epochs_done;
  return SRW_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Resumable scans: a scan of n points cut into chunks of chunk_points
// consecutive Sobol indices, each chunk an independent srw_surrogate_scan; a
// state file records every completed chunk's result (rewritten through a
// temporary file and a rename after each chunk), so a scan that stops, for
// any reason, continues from its last completed chunk.
// ---------------------------------------------------------------------------
namespace {

std::string scan_key(const srw_scan_opts* o, long long chunk) {
  std::vector<unsigned char> b((size_t)o->n_check * 5 * sizeof(float));
  if (o->n_check > 0) std::memcpy(b.data(), o->check_theta, b.size());
  char k[512];
  std::snprintf(k, sizeof(k),
                "srw-scan 1 first=%lld n=%lld chunk=%lld keep=%.17g tol=%.17g cells=%d prec=%d rule=%d margin=%.17g "
                "check=%d hash=%016llx",
                o->first, o->n_points, chunk, o->keep_frac, o->tol, o->cells_per_dim, o->precision, o->rule,
                o->margin_factor, o->n_check, (unsigned long long)fnv1a(b));
  return k;
}

struct ChunkRecord {
  long long c;
  srw_scan_result r;
};

// 0: read (or no file); 1: the file belongs to another scan; 2: unreadable
int read_scan_state(const char* path, const std::string& key, std::vector<ChunkRecord>& recs) {
  recs.clear();
  FILE* f = std::fopen(path, "r");
  if (!f) return 0;
  char line[1024];
  int st = 0;
  if (!std::fgets(line, sizeof(line), f) || key != std::string(line).substr(0, std::string(line).find('\n'))) st = 1;
  while (st == 0 && std::fgets(line, sizeof(line), f)) {
    ChunkRecord q;
    std::memset(&q, 0, sizeof(q));
    srw_scan_result& r = q.r;
    const int n = std::sscanf(line, "chunk %lld %lg %lld %g %g %g %g %g %lg %lld %lld %lld %d %d %lg %g %g %g %g", &q.c,
                              &r.best_value, &r.best_index, &r.best_theta[0], &r.best_theta[1], &r.best_theta[2],
                              &r.best_theta[3], &r.best_theta[4], &r.surrogate_min, &r.n_kept, &r.n_selected,
                              &r.n_rescued, &r.n_cells, &r.n_flagged_cells, &r.check_max_abs_d, &r.ms_check,
                              &r.ms_surrogate, &r.ms_select, &r.ms_exact);
    if (n != 19) {
      st = 2;
      break;
    }
    recs.push_back(q);
  }
  std::fclose(f);
  return st;
}

bool write_scan_state(const char* path, const std::string& key, const std::vector<ChunkRecord>& recs) {
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return false;
  bool ok = std::fprintf(f, "%s\n", key.c_str()) > 0;
  for (const ChunkRecord& q : recs) {
    const srw_scan_result& r = q.r;
    ok = ok && std::fprintf(f, "chunk %lld %.17g %lld %.9g %.9g %.9g %.9g %.9g %.17g %lld %lld %lld %d %d %.17g %.9g %.9g "
                               "%.9g %.9g\n",
                            q.c, r.best_value, r.best_index, r.best_theta[0], r.best_theta[1], r.best_theta[2],
                            r.best_theta[3], r.best_theta[4], r.surrogate_min, r.n_kept, r.n_selected, r.n_rescued,
                            r.n_cells, r.n_flagged_cells, r.check_max_abs_d, r.ms_check, r.ms_surrogate, r.ms_select,
                            r.ms_exact) > 0;
  }
  ok = std::fflush(f) == 0 && ok;
  if (std::fclose(f) != 0 || !ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return false;
  }
  return true;
}

// The scan's result from its chunks': the smallest exact minimum (ties: the
// smaller Sobol index), counts and times summed.
void merge_chunks(const std::vector<ChunkRecord>& recs, srw_scan_result* res) {
  std::memset(res, 0, sizeof(*res));
  res->best_value = INFINITY;
  res->best_index = -1;
  res->surrogate_min = INFINITY;
  for (const ChunkRecord& q : recs) {
    const srw_scan_result& r = q.r;
    if (r.best_index >= 0 && (r.best_value < res->best_value ||
                              (r.best_value == res->best_value && r.best_index < res->best_index))) {
      res->best_value = r.best_value;
      res->best_index = r.best_index;
      std::memcpy(res->best_theta, r.best_theta, sizeof(r.best_theta));
    }
    res->surrogate_min = std::min(res->surrogate_min, r.surrogate_min);
    res->n_kept += r.n_kept;
    res->n_selected += r.n_selected;
    res->n_rescued += r.n_rescued;
    res->n_cells = r.n_cells;
    res->n_flagged_cells = r.n_flagged_cells;
    res->check_max_abs_d = std::max(res->check_max_abs_d, r.check_max_abs_d);
    res->ms_check += r.ms_check;
    res->ms_surrogate += r.ms_surrogate;
    res->ms_select += r.ms_select;
    res->ms_exact += r.ms_exact;
  }
}

}  // namespace

extern "C" {

srw_status srw_surrogate_scan_chunked(srw_surrogate s, const srw_scan_opts* o, long long chunk_points,
                                      const char* state_path, int max_new_chunks, srw_scan_result* res,
                                      int* complete) {
  if (!s || !o || !res || !state_path || chunk_points < 1) return SRW_EINVAL;
  if (complete) *complete = 0;
  if (o->n_points < 1 || o->first < 0) return sfail(s, SRW_EINVAL, "bad scan options");
  const std::string key = scan_key(o, chunk_points);
  std::vector<ChunkRecord> recs;
  const int rs = read_scan_state(state_path, key, recs);
  if (rs == 1) return sfail(s, SRW_EINVAL, "the state file belongs to a different scan");
  if (rs == 2) return sfail(s, SRW_EINVAL, "the state file is damaged");
  const long long n_chunks = (o->n_points + chunk_points - 1) / chunk_points;
  std::vector<char> done((size_t)n_chunks, 0);
  for (const ChunkRecord& q : recs)
    if (q.c >= 0 && q.c < n_chunks) done[(size_t)q.c] = 1;
  int fresh = 0;
  for (long long c = 0; c < n_chunks; ++c) {
    if (done[(size_t)c]) continue;
    if (max_new_chunks > 0 && fresh >= max_new_chunks) break;
    srw_scan_opts oc = *o;
    oc.first = o->first + c * chunk_points;
    oc.n_points = std::min(chunk_points, o->n_points - c * chunk_points);
    ChunkRecord q;
    q.c = c;
    const srw_status st = srw_surrogate_scan(s, &oc, &q.r);
    if (st != SRW_OK) return st;
    recs.push_back(q);
    done[(size_t)c] = 1;
    ++fresh;
    if (!write_scan_state(state_path, key, recs)) return sfail(s, SRW_EINVAL, "cannot write the scan state file");
  }
  merge_chunks(recs, res);
  bool all = true;
  for (char d : done) all = all && d;
  if (complete) *complete = all ? 1 : 0;
  return SRW_OK;
}

const char* srw_surrogate_last_error(srw_surrogate s) { return s ? s->err.c_str() : "NULL surrogate"; }

srw_status srw_surrogate_destroy(srw_surrogate s) {
  if (!s) return SRW_OK;
  cudaSetDevice(s->device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (SurrogateBatch* B : s->batches) free_batch(B);
  for (SurrogateLayer& L : s->L) {
    sfree(L.w); sfree(L.b); sfree(L.mw); sfree(L.vw); sfree(L.mb); sfree(L.vb); sfree(L.gw); sfree(L.gb);
    sfree(L.w_bf); sfree(L.wt_bf);
  }
  sfree(s->mean);
  sfree(s->stdv);
  sfree(s->binc);
  sfree(s->d_status);
  sfree(s->d_sobol);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
  return SRW_OK;
}

}  // extern "C"
