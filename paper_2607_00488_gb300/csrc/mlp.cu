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
// MMA issuer / TMEM owner, warps 2-5 epilogue (warp w reads TMEM lanes
// 32 (w % 4) ...).  Every wait is bounded; a timeout raises kStatusTimeout.

#include <algorithm>
#include <cmath>
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
constexpr int kGemmThreads = 6 * 32;
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
  const float* mean;     // scan: per-bin mean / std of log mu
  const float* stdv;
  const float2* nb;      // scan: {n_j, or -1 where masked, unused}
  double* parts;         // scan: per (column tile, row) partial sums of the deviance
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
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dsmem_raw) + 1023) & ~uintptr_t(1023));
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
      ptx::mbar_init(&acc_empty[b], 4);
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
          if (!ptx::mbar_wait(&empty[st], ((g / ST) & 1) ^ 1, &abort_flag, 2000000000ull, 32)) {
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
    const int q = warp & 3;  // TMEM lanes 32 q .. 32 q + 31
    int tc = -1;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
      ++tc;
      if (__any_sync(0xffffffffu, aborted(&abort_flag))) break;
      const int m0 = (t / n_tn) * kBM, n0 = (t % n_tn) * BN;
      const int buf = tc & 1;
      if (!warp_wait(&acc_full[buf], (tc >> 1) & 1, &abort_flag, 128)) {
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
      for (int c0 = 0; c0 < BN; c0 += 16) {
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
        } else {  // kFwdScan: Poisson deviance of mu = exp(m + s y)
          float ts = 0.f;
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int j = n + k;
            float nj = -1.f, mu = 1.f;
            if (j < E.cols_valid) {
              nj = __ldg(&E.nb[j].x);
              mu = expf(__ldg(E.mean + j) + __ldg(E.stdv + j) * (v[k] + __ldg(E.bias + j)));
            }
            const float tj = poisson_term_f32_sel(mu, nj);
            ts += nj >= 0.f ? tj : 0.f;
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
        E.parts[(size_t)(n0 / BN) * E.rows_valid + m] =
            infinite ? __longlong_as_double(0x7ff0000000000000LL) : (double)dev.hi + (double)dev.lo;
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kMmaWarp) tmem_dealloc(tmem_base, S::kTmemCols);
}

// theta [rows][5] -> X0 [M][128] and X0^T [128][M] (BF16), normalised to the box.
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
  __nv_bfloat16* row = x + (size_t)m * kInPad;
  for (int k = 0; k < kInPad; ++k) {
    const __nv_bfloat16 b = __float2bfloat16_rn(k < kIn ? u[k] : 0.f);
    row[k] = b;
    if (xt) xt[(size_t)k * M + m] = b;
  }
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

// Training targets: log(mu_sig + b) in place ([rows][ld], columns < n valid; padding = 0).
__global__ void log_counts_kernel(float* __restrict__ t, long long rows, int n, int ld, const double* __restrict__ b64) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * ld) return;
  const int j = (int)(i % ld);
  t[i] = j < n ? logf(fmaxf(t[i] + (float)b64[j], 1e-30f)) : 0.f;
}

// Per-column sums and sums of squares (FP64) over rows, for the standardization.
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
  atomicAdd(s1 + j, a);
  atomicAdd(s2 + j, b);
}

__global__ void finish_stats_kernel(const double* __restrict__ s1, const double* __restrict__ s2, long long rows,
                                    int n, float* __restrict__ mean, float* __restrict__ stdv) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double m = s1[j] / (double)rows;
  const double var = fmax(s2[j] / (double)rows - m * m, 0.0);
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

__global__ void scan_reduce_kernel(const double* __restrict__ parts, int n_parts, int rows,
                                   const double* __restrict__ c_data, double* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= rows) return;
  double s = 0.0;
  for (int t = 0; t < n_parts; ++t) s += parts[(size_t)t * rows + p];
  out[p] = 2.0 * s + *c_data;
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
  return cudaGetLastError();
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
  int stats_ready = 0;
  long long adam_t = 0;
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
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (n ? n : 1));
}
template <class T>
void sfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

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
  if (e == cudaSuccess) e = salloc(&B->y, (size_t)M * NO);
  if (e == cudaSuccess) e = salloc(&B->parts, (size_t)(NO / 256) * M);
  if (e == cudaSuccess) e = salloc(&B->loss, 1);
  if (train) {
    if (e == cudaSuccess) e = salloc(&B->xt, (size_t)M * srw::kInPad);
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
    E.mean = s->mean;
    E.stdv = s->stdv;
    E.nb = reinterpret_cast<const float2*>(s->h->d_nb2);
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
  return cudaGetLastError();
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
                     cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(B->loss, 0, sizeof(double), st);
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
      e = cudaGetLastError();
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
  return cudaGetLastError();
}

srw_status check_status(srw_surrogate s, cudaStream_t st) {
  unsigned v = 0;
  S_CUDA(s, cudaMemcpyAsync(&v, s->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "status read");
  S_CUDA(s, cudaStreamSynchronize(st), "sync");
  if (v) S_CUDA(s, cudaMemsetAsync(s->d_status, 0, sizeof(unsigned), st), "status reset");
  if (v & srw::kStatusTimeout) return sfail(s, SRW_ETIMEOUT, "a bounded device wait expired; the kernel aborted");
  return SRW_OK;
}

int round_up(long long x, int m) { return (int)((x + m - 1) / m * m); }

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
    S_CUDA(s, cudaGetLastError(), "cast weights");
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
  float* d_th = nullptr;
  S_CUDA(s, cudaMallocAsync(&d_th, sizeof(float) * 5 * (size_t)P, s->stream), "alloc");
  S_CUDA(s, cudaMemcpyAsync(d_th, theta, sizeof(float) * 5 * (size_t)P, cudaMemcpyHostToDevice, s->stream), "upload");
  cudaError_t e = forward_hidden(s, d_th, P, B, false, s->stream);
  if (e == cudaSuccess) {
    Gemm g = B->fwd_out;
    g.E.rows_valid = P;
    e = srw::run_gemm(g, s->sm_count, s->d_status, s->stream);
  }
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(y, sizeof(float) * s->n_out, B->y, sizeof(float) * s->n_out_pad, sizeof(float) * s->n_out, P,
                          cudaMemcpyDeviceToHost, s->stream);
  cudaFreeAsync(d_th, s->stream);
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
  float *d_th = nullptr, *d_t = nullptr;
  S_CUDA(s, cudaMallocAsync(&d_th, sizeof(float) * 5 * (size_t)P, s->stream), "alloc");
  S_CUDA(s, cudaMallocAsync(&d_t, sizeof(float) * (size_t)M * s->n_out_pad, s->stream), "alloc");
  S_CUDA(s, cudaMemsetAsync(d_t, 0, sizeof(float) * (size_t)M * s->n_out_pad, s->stream), "zero");
  S_CUDA(s, cudaMemcpyAsync(d_th, theta, sizeof(float) * 5 * (size_t)P, cudaMemcpyHostToDevice, s->stream), "upload");
  S_CUDA(s, cudaMemcpy2DAsync(d_t, sizeof(float) * s->n_out_pad, targets, sizeof(float) * s->n_out,
                              sizeof(float) * s->n_out, P, cudaMemcpyHostToDevice, s->stream),
         "upload targets");
  cudaError_t e = fit_pass(s, d_th, d_t, P, B, s->stream);
  double sse = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&sse, B->loss, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  cudaFreeAsync(d_th, s->stream);
  cudaFreeAsync(d_t, s->stream);
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
  float *d_th = nullptr, *d_t = nullptr;
  S_CUDA(s, cudaMallocAsync(&d_th, sizeof(float) * 5 * (size_t)P, s->stream), "alloc");
  S_CUDA(s, cudaMallocAsync(&d_t, sizeof(float) * (size_t)M * s->n_out_pad, s->stream), "alloc");
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
  cudaFreeAsync(d_th, s->stream);
  cudaFreeAsync(d_t, s->stream);
  if (e != cudaSuccess) return scuda(s, e, "surrogate train step");
  if (loss) *loss = sse / ((double)P * s->n_out);
  return check_status(s, s->stream);
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
  sfree(s->d_status);
  sfree(s->d_sobol);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
  return SRW_OK;
}

}  // extern "C"
