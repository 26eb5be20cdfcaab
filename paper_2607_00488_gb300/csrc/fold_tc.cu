// Batched fold on the 5th-generation tensor cores (tcgen05) of sm_103a.
//
// For P parameter points the fold of eq. matrix_reweight is the contraction
//   M[p][j] = sum_i W[p][i] R[j][i],   W[p][i] = sum_b c_b(theta_p) shat_b[i]
// (the weighted true spectra are linear in eight coefficient spectra, see
// srw_internal.h), followed by the Poisson terms of eq. logL, reduced per
// point.  Roles of one persistent CTA (one per SM):
//
//   warps 0-7  W producers: each thread owns four points (rows) of the
//              128-row A tile and 8 of the 64 K of the current block (warp w
//              takes K chunk w); it computes W from the coefficients and the
//              block's coefficient spectra (streamed into a shared-memory ring,
//              read as warp-uniform loads), splits W into BF16 hi (+ lo) and
//              writes it in the 128-byte-swizzled K-major layout the tensor
//              core reads.
//   warps 8-11 epilogue: thread = point; reads its accumulator row from
//              tensor memory (TMEM lane = point, column = rec bin), adds the
//              background, applies the mask, evaluates the Poisson terms and
//              accumulates them per point (double-float), one FP64 partial per
//              (rec tile, point).
//   warp 12    TMA producers: lane 0 streams R hi (+ lo) tiles, 64 x BN,
//              128-byte swizzle; lane 1 streams the 2 KB coefficient-spectra
//              slice of each K block, up to kShatSlots blocks ahead.
//   warp 13    MMA issuer (one thread) and TMEM owner.
//
// The fold is taken of W(theta) - W_ref (the reference point's FP64 fold
// R W_ref enters the epilogue with the background), so the BF16 rounding
// errors scale with the distance of theta from the reference.
// Precision: SRW_BF16 issues hi*hi; SRW_BF16X3 issues hi*hi + hi*lo + lo*hi,
// all accumulating in FP32 in TMEM.  The accumulator is double-buffered
// (2 x BN columns) so the epilogue of one tile overlaps the next tile's MMAs.
//
// Every wait is bounded (ptx.cuh); on a timeout the CTA raises
// kStatusTimeout, drains its outstanding copies and MMAs, frees TMEM and ends.

#include <cuda.h>

#include "dfloat.cuh"
#include "poisson.cuh"
#include "ptx.cuh"
#include "srw_internal.h"

namespace srw {
namespace {

constexpr int kBM = 128;   // points per tile (MMA M, TMEM lanes)
constexpr int kBK = 64;    // K per stage: one 128-byte swizzle atom of BF16
constexpr int kWWarps = 8;
constexpr int kEpiWarp0 = 8;
constexpr int kTmaWarp = 12;
constexpr int kMmaWarp = 13;
constexpr int kThreads = 14 * 32;
constexpr int kShatBytes = kBK * kNB * 4;  // coefficient spectra of one K block (k-major)
constexpr int kShatSlots = 4;              // depth of the coefficient-spectra ring

struct TcMaps {
  CUtensorMap hi[2], lo[2];  // index 0: box rows 128, 1: box rows 256
};

// ---------------------------------------------------------------- tcgen05 PTX
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(ptx::smem_addr(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrives once on `bar` when every tcgen05.mma issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   ptx::smem_addr(bar))
               : "memory");
}

// 32 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

// 16 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          ptx::smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(ptx::smem_addr(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (SBO); LBO unused for this layout.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;                  // LBO (unused) = 16 B
  d |= (uint64_t)(1024u >> 4) << 32;        // SBO = 1024 B
  d |= (uint64_t)1u << 46;                  // descriptor version for sm_100 family
  d |= (uint64_t)2u << 61;                  // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: BF16 x BF16 -> FP32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

__device__ __forceinline__ void coefficients(const float* th, dfloat s, const CoefRef& ref, float* c) {
  const dfloat gle = df_add(df_add(dfloat{0.5f, 0.f}, s), th[0]), gre = df_add(s, th[1]);
  const dfloat glt = df_add(df_add(dfloat{-0.5f, 0.f}, s), th[2]), grt = df_add(s, th[3]);
  const dfloat x = df_mul(gle, gre), y = df_mul(glt, grt);
  const dfloat v[kNB] = {df_mul(gle, gle), df_mul(gre, gre), {-x.hi, -x.lo}, df_mul(glt, glt),
                         df_mul(grt, grt), {-y.hi, -y.lo}, {1.f, 0.f}, two_prod(th[4], th[4])};
#pragma unroll
  for (int b = 0; b < kNB; ++b) {
    const dfloat d = df_add(v[b], dfloat{-ref.hi[b], -ref.lo[b]});  // deviation from the reference point
    c[b] = d.hi + d.lo;
  }
}

__device__ __forceinline__ bool aborted(const unsigned* f) { return *(const volatile unsigned*)f != 0u; }

// Bounded wait taken by all 32 lanes of a warp; the warp proceeds only if
// every lane saw the phase complete, so no lane can run ahead into a
// .sync.aligned instruction or a __syncwarp that the others skip.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, unsigned* abort_flag,
                                          unsigned sleep_ns = 0) {
  const bool ok = ptx::mbar_wait(bar, parity, abort_flag, 2000000000ull, sleep_ns);
  return __all_sync(0xffffffffu, ok);
}

template <int BN, bool X3>
struct TcShape {
  static constexpr int kAB = kBM * kBK * 2;             // bytes of one BF16 A tile
  static constexpr int kBB = BN * kBK * 2;              // bytes of one BF16 B tile
  static constexpr int kStageBytes = (X3 ? 2 : 1) * (kAB + kBB);
  static constexpr int kStages = (200 * 1024 - kShatSlots * kShatBytes) / kStageBytes;
  static constexpr int kSmem = kStages * kStageBytes + kShatSlots * kShatBytes + 1024;  // + alignment slack
  static constexpr int kTmemCols = 2 * BN;
};

template <int BN, bool X3>
__global__ void __launch_bounds__(kThreads, 1)
fold_tc_kernel(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
               const float* __restrict__ theta, int P, dfloat sin2w, CoefRef cref,
               const float4* __restrict__ shat_k8, int k_pad,
               int n_rec, const float2* __restrict__ nb2, double* __restrict__ parts,
               float* __restrict__ musig_out, unsigned* __restrict__ status) {
  using S = TcShape<BN, X3>;
  constexpr int ST = S::kStages;
  extern __shared__ unsigned char dsmem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dsmem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t r_full[ST], w_full[ST], empty[ST], acc_full[2], acc_empty[2], drain;
  __shared__ __align__(8) uint64_t s_full[kShatSlots], s_empty[kShatSlots];
  __shared__ uint32_t tmem_slot;
  __shared__ unsigned abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m_tiles = (P + kBM - 1) / kBM;
  const int n_tiles = (n_rec + BN - 1) / BN;
  const int n_work = m_tiles * n_tiles;
  const int n_kb = k_pad / kBK;

  auto a_hi = [&](int st) { return smem + (size_t)st * S::kStageBytes; };
  auto a_lo = [&](int st) { return smem + (size_t)st * S::kStageBytes + S::kAB; };
  auto b_hi = [&](int st) { return smem + (size_t)st * S::kStageBytes + (X3 ? 2 : 1) * S::kAB; };
  auto b_lo = [&](int st) { return smem + (size_t)st * S::kStageBytes + 2 * S::kAB + S::kBB; };
  auto shat_s = [&](int slot) {
    return reinterpret_cast<float4*>(smem + (size_t)ST * S::kStageBytes + (size_t)slot * kShatBytes);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      ptx::mbar_init(&r_full[s], 1);
      ptx::mbar_init(&w_full[s], kWWarps);
      ptx::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(&acc_full[b], 1);
      ptx::mbar_init(&acc_empty[b], 4);
    }
    for (int q = 0; q < kShatSlots; ++q) {
      ptx::mbar_init(&s_full[q], 1);
      ptx::mbar_init(&s_empty[q], kWWarps);
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

  if (warp < kWWarps) {
    // ------------------------------------------------------------ W producers
    // thread: rows rg, rg + 32, rg + 64, rg + 96 of the A tile and the 8 K of
    // chunk `warp`; the coefficient-spectra loads are warp-uniform and each
    // feeds 32 FMAs (shared-memory wavefronts are the scarce resource here).
    const int rg = lane;
    const int ch = warp;  // 16-byte chunk = 8 consecutive k
    int g = 0;            // global K-block counter (stage ring position)
    for (int work = blockIdx.x; work < n_work; work += gridDim.x) {
      if (__any_sync(0xffffffffu, aborted(&abort_flag))) break;
      const int m0 = (work / n_tiles) * kBM;
      float c[4][kNB];
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) {
        const int p = m0 + rg + 32 * rr;
        if (p < P) coefficients(theta + (size_t)p * 5, sin2w, cref, c[rr]);
        else
#pragma unroll
          for (int b = 0; b < kNB; ++b) c[rr][b] = 0.f;
      }
      bool ok = true;
      for (int kb = 0; kb < n_kb; ++kb, ++g) {
        const int st = g % ST, sl = g % kShatSlots;
        // the A buffers of this stage are free once the MMAs of its previous
        // use have completed; the coefficient spectra come through their own ring
        if (!warp_wait(&empty[st], ((g / ST) & 1) ^ 1, &abort_flag, 64) ||
            !warp_wait(&s_full[sl], (g / kShatSlots) & 1, &abort_flag, 64)) {
          give_up();
          ok = false;
          break;
        }
        const float4* sh = shat_s(sl) + ch * 16;  // 8 k x 8 floats
        uint32_t h[4][4], l[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float w[4][2];
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const float4 s0 = sh[(q * 2 + e) * 2], s1 = sh[(q * 2 + e) * 2 + 1];
            const float sv[kNB] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
#pragma unroll
            for (int rr = 0; rr < 4; ++rr) {
              float a = c[rr][0] * sv[0];
#pragma unroll
              for (int bb = 1; bb < kNB; ++bb) a = fmaf(c[rr][bb], sv[bb], a);
              w[rr][e] = a;
            }
          }
#pragma unroll
          for (int rr = 0; rr < 4; ++rr) {
            h[rr][q] = pack_bf16x2(w[rr][0], w[rr][1]);
            if (X3) {
              const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(&h[rr][q]);
              l[rr][q] = pack_bf16x2(w[rr][0] - __low2float(v), w[rr][1] - __high2float(v));
            }
          }
        }
        // the four rows share the swizzle phase (row & 7)
        const uint32_t off = (uint32_t)((ch ^ (rg & 7)) * 16);
        const uint32_t ah = ptx::smem_addr(a_hi(st)), al = ptx::smem_addr(a_lo(st));
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
          const uint32_t ro = (uint32_t)((rg + 32 * rr) * 128) + off;
          st_shared_v4(ah + ro, h[rr][0], h[rr][1], h[rr][2], h[rr][3]);
          if (X3) st_shared_v4(al + ro, l[rr][0], l[rr][1], l[rr][2], l[rr][3]);
        }
        ptx::fence_proxy_async_smem();  // generic-proxy writes -> visible to the tensor core
        __syncwarp();
        if (lane == 0) {
          ptx::mbar_arrive(&w_full[st]);
          ptx::mbar_arrive(&s_empty[sl]);
        }
      }
      if (!ok) break;
    }
  } else if (warp < kEpiWarp0 + 4) {
    // ------------------------------------------------------------ epilogue
    const int q = warp - kEpiWarp0;  // TMEM lane quarter of this warp
    int tc = 0;
    for (int work = blockIdx.x; work < n_work; work += gridDim.x, ++tc) {
      if (__any_sync(0xffffffffu, aborted(&abort_flag))) break;
      const int m0 = (work / n_tiles) * kBM, nt = work % n_tiles, n0 = nt * BN;
      const int buf = tc & 1;
      if (!warp_wait(&acc_full[buf], (tc >> 1) & 1, &abort_flag, 256)) {
        give_up();
        break;
      }
      tc_fence_after();
      const int p = m0 + q * 32 + lane;
      const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN);
      dfloat acc = {0.f, 0.f};
      bool infinite = false;  // a +inf term (mu <= 0 with data) is kept apart: TwoSum would make it NaN
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        // per-column constants first (warp-uniform loads), then the accumulator row
        float2 dj[16];
        if (parts != nullptr) {
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int j = n0 + c0 + k;
            dj[k] = j < n_rec ? __ldg(nb2 + j) : make_float2(-1.f, 1.f);  // n_j (-1: masked), b_j + ref
          }
        }
        float v[16];
        tmem_ld16(tbase + (uint32_t)c0, v);
        if (musig_out != nullptr && p < P) {  // batched folded spectra (row p)
          float* row = musig_out + (size_t)p * n_rec;
#pragma unroll
          for (int k = 0; k < 16; ++k)
            if (n0 + c0 + k < n_rec) row[n0 + c0 + k] = v[k];
        }
        if (parts != nullptr) {
          float ts = 0.f;
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const float t = poisson_term_f32_sel(v[k] + dj[k].y, dj[k].x);
            ts += dj[k].x >= 0.f ? t : 0.f;  // masked and padding columns add nothing
          }
          if (isinf(ts)) infinite = true;
          else acc = df_add(acc, ts);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&acc_empty[buf]);
      if (parts != nullptr && p < P)
        parts[(size_t)nt * P + p] = infinite ? __longlong_as_double(0x7ff0000000000000LL) : (double)acc.hi + (double)acc.lo;
    }
  } else if (warp == kTmaWarp) {
    // ------------------------------------------------------------ TMA producers
    if (lane == 0) {  // R hi (+ lo) tiles into the stage ring
      int g = 0, issued_g = 0;
      const uint32_t bytes = (uint32_t)(X3 ? 2 : 1) * S::kBB;
      for (int work = blockIdx.x; work < n_work && !aborted(&abort_flag); work += gridDim.x) {
        const int n0 = (work % n_tiles) * BN;
        bool ok = true;
        for (int kb = 0; kb < n_kb; ++kb, ++g) {
          const int st = g % ST;
          if (!ptx::mbar_wait(&empty[st], ((g / ST) & 1) ^ 1, &abort_flag, 2000000000ull, 32)) {
            give_up();
            ok = false;
            break;
          }
          ptx::mbar_arrive_expect_tx(&r_full[st], bytes);
          tma_load_2d(b_hi(st), &map_hi, kb * kBK, n0, &r_full[st]);
          if (X3) tma_load_2d(b_lo(st), &map_lo, kb * kBK, n0, &r_full[st]);
          issued_g = g + 1;
        }
        if (!ok) break;
      }
      // never end with copies in flight
      for (int u = max(0, issued_g - ST); u < issued_g; ++u)
        ptx::mbar_wait(&r_full[u % ST], (u / ST) & 1, nullptr, 100000000ull);
    } else if (lane == 1) {  // coefficient-spectra slices, up to kShatSlots blocks ahead
      const int total = ((n_work - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x) * n_kb;
      int issued = 0;
      for (int g = 0; g < total; ++g) {
        const int sl = g % kShatSlots;
        if (!ptx::mbar_wait(&s_empty[sl], ((g / kShatSlots) & 1) ^ 1, &abort_flag, 2000000000ull, 32)) {
          give_up();
          break;
        }
        ptx::mbar_arrive_expect_tx(&s_full[sl], (uint32_t)kShatBytes);
        ptx::bulk_g2s(shat_s(sl), shat_k8 + (size_t)(g % n_kb) * kBK * 2, (uint32_t)kShatBytes, &s_full[sl]);
        issued = g + 1;
      }
      for (int u = max(0, issued - kShatSlots); u < issued; ++u)
        ptx::mbar_wait(&s_full[u % kShatSlots], (u / kShatSlots) & 1, nullptr, 100000000ull);
    }
  } else {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(kBM, BN);
      int g = 0, tc = 0;
      bool issued_any = false;
      for (int work = blockIdx.x; work < n_work && !aborted(&abort_flag); work += gridDim.x, ++tc) {
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
          if (!ptx::mbar_wait(&r_full[st], (g / ST) & 1, &abort_flag) ||
              !ptx::mbar_wait(&w_full[st], (g / ST) & 1, &abort_flag)) {
            give_up();
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t ah = ptx::smem_addr(a_hi(st)), bh = ptx::smem_addr(b_hi(st));
          const uint32_t al = ptx::smem_addr(a_lo(st)), bl = ptx::smem_addr(b_lo(st));
#pragma unroll
          for (int ks = 0; ks < kBK / 16; ++ks) {
            const uint32_t off = (uint32_t)ks * 32u;  // 16 BF16 along K inside the swizzle atom
            mma_bf16(d_tmem, smem_desc_sw128(ah + off), smem_desc_sw128(bh + off), idesc, (kb | ks) != 0);
            if (X3) {
              mma_bf16(d_tmem, smem_desc_sw128(ah + off), smem_desc_sw128(bl + off), idesc, 1u);
              mma_bf16(d_tmem, smem_desc_sw128(al + off), smem_desc_sw128(bh + off), idesc, 1u);
            }
          }
          issued_any = true;
          mma_commit(&empty[st]);  // frees the stage once these MMAs have read it
        }
        if (!ok) break;
        mma_commit(&acc_full[buf]);  // accumulator complete
      }
      // before TMEM is released every issued MMA must have finished
      if (issued_any) {
        mma_commit(&drain);
        ptx::mbar_wait(&drain, 0, nullptr, 100000000ull);
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kMmaWarp) tmem_dealloc(tmem_base, S::kTmemCols);
}

// R (FP32, n_rec x ld) -> BF16 hi + lo (rec_pad x k_pad, zero padding); and
// shat (FP32 [8][k_pad]) -> k-major [k_pad][8] for the W producers.
__global__ void split_r_kernel(const float* __restrict__ R, int n_rec, int ld, int rec_pad, int k_pad,
                               __nv_bfloat16* __restrict__ rhi, __nv_bfloat16* __restrict__ rlo) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)rec_pad * k_pad) return;
  const int j = (int)(idx / k_pad), k = (int)(idx % k_pad);
  const float x = (j < n_rec && k < ld) ? R[(size_t)j * ld + k] : 0.f;
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  rhi[idx] = h;
  rlo[idx] = __float2bfloat16_rn(x - __bfloat162float(h));
}

__global__ void shat_k8_kernel(const float* __restrict__ shat, int k_pad, float* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= k_pad) return;
#pragma unroll
  for (int b = 0; b < kNB; ++b) out[(size_t)k * kNB + b] = shat[(size_t)b * k_pad + k];
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

template <int BN, bool X3>
cudaError_t set_attr() {
  return cudaFuncSetAttribute(fold_tc_kernel<BN, X3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              TcShape<BN, X3>::kSmem);
}

template <int BN, bool X3>
cudaError_t launch_cfg(const srw_ctx* h, const TcMaps* maps, const float* theta, int P, double* parts,
                       float* musig_out, cudaStream_t s) {
  using S = TcShape<BN, X3>;
  const int work = ((P + kBM - 1) / kBM) * ((h->n_rec + BN - 1) / BN);
  const int grid = work < h->sm_count ? work : h->sm_count;
  const int bi = BN == 256 ? 1 : 0;
  fold_tc_kernel<BN, X3><<<grid, kThreads, S::kSmem, s>>>(
      maps->hi[bi], maps->lo[bi], theta, P, df_from_double(h->sin2w), h->cref,
      reinterpret_cast<const float4*>(h->d_shat_k8),
      h->k_pad, h->n_rec, reinterpret_cast<const float2*>(h->d_nb2), parts, musig_out, h->d_status);
  return cudaGetLastError();
}

}  // namespace

bool tc_supported(const srw_ctx* h) { return h->cc_major == 10 && h->cc_minor == 3; }

static const FoldConfig kConfigs[] = {
    {1, 256, 0, kWWarps},
    {1, 128, 0, kWWarps},
};

int tc_num_configs() { return (int)(sizeof(kConfigs) / sizeof(kConfigs[0])); }
FoldConfig tc_config(int i) { return kConfigs[i]; }

cudaError_t launch_split_r(srw_ctx* h, cudaStream_t s) {
  const size_t n = (size_t)h->rec_pad * h->k_pad;
  split_r_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(h->d_R, h->n_rec, h->ld_r, h->rec_pad, h->k_pad,
                                                             h->d_rhi, h->d_rlo);
  shat_k8_kernel<<<(h->k_pad + 255) / 256, 256, 0, s>>>(h->d_shat, h->k_pad, h->d_shat_k8);
  return cudaGetLastError();
}

cudaError_t tc_prepare(srw_ctx* h) {
  cudaError_t ea = set_attr<256, true>();
  if (ea == cudaSuccess) ea = set_attr<256, false>();
  if (ea == cudaSuccess) ea = set_attr<128, true>();
  if (ea == cudaSuccess) ea = set_attr<128, false>();
  if (ea != cudaSuccess) return ea;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q);
  if (e != cudaSuccess || fn == nullptr || q != cudaDriverEntryPointSuccess) return cudaErrorNotSupported;
  EncodeTiledFn encode = reinterpret_cast<EncodeTiledFn>(fn);
  TcMaps* maps = new (std::nothrow) TcMaps();
  if (!maps) return cudaErrorMemoryAllocation;
  const cuuint64_t dims[2] = {(cuuint64_t)h->k_pad, (cuuint64_t)h->rec_pad};
  const cuuint64_t strides[1] = {(cuuint64_t)h->k_pad * 2};
  const cuuint32_t estr[2] = {1, 1};
  for (int bi = 0; bi < 2; ++bi) {
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)(bi ? 256 : 128)};
    for (int lo = 0; lo < 2; ++lo) {
      CUresult r = encode(lo ? &maps->lo[bi] : &maps->hi[bi], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                          lo ? (void*)h->d_rlo : (void*)h->d_rhi, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) {
        delete maps;
        return cudaErrorInvalidValue;
      }
    }
  }
  h->tmap = maps;
  return cudaSuccess;
}

void tc_release(srw_ctx* h) {
  delete static_cast<TcMaps*>(h->tmap);
  h->tmap = nullptr;
}

cudaError_t launch_fold_tc(const srw_ctx* h, const float* theta, int P, int precision, const FoldConfig& cfg,
                           double* parts, cudaStream_t s, int* n_parts, float* musig_out) {
  const TcMaps* maps = static_cast<const TcMaps*>(h->tmap);
  if (!maps) return cudaErrorNotSupported;
  const bool x3 = precision == SRW_BF16X3;
  if (n_parts) *n_parts = (h->n_rec + cfg.bn - 1) / cfg.bn;
  if (cfg.bn == 256) return x3 ? launch_cfg<256, true>(h, maps, theta, P, parts, musig_out, s)
                               : launch_cfg<256, false>(h, maps, theta, P, parts, musig_out, s);
  return x3 ? launch_cfg<128, true>(h, maps, theta, P, parts, musig_out, s)
            : launch_cfg<128, false>(h, maps, theta, P, parts, musig_out, s);
}

}  // namespace srw
