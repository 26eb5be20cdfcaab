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
//              takes K chunk w); it computes W from the coefficients (seven
//              terms: the constant monomial is always in the reference fold)
//              and the block's coefficient spectra (streamed into a
//              shared-memory ring, read as warp-uniform loads), splits W into
//              hi (+ lo) halves and writes it in the 128-byte-swizzled K-major
//              layout the tensor core reads.
//   warps 8-11 epilogue: thread = point; reads its accumulator row from
//              tensor memory (TMEM lane = point, column = rec bin), adds the
//              background and reference fold (one float4 of constants per
//              bin), evaluates the Poisson terms with the mask multiplied out
//              and accumulates them per point (double-float), one FP64 partial
//              per (rec tile, point).
//   warp 12    TMA producer: streams R hi (+ lo) tiles, BK x BN, swizzled.
//   warp 13    MMA issuer (one thread) and TMEM owner.
//   warp 14    TMA producer of the coefficient-spectra slice of each K block
//              (BK x 8 floats), up to kShatSlots blocks ahead.
//
// The fold is taken of W(theta) - W_ref (the reference point's FP64 fold
// R W_ref enters the epilogue with the background), so the BF16 rounding
// errors scale with the distance of theta from the reference.
// Precision: SRW_BF16 issues hi*hi; SRW_BF16X3 issues hi*hi + hi*lo + lo*hi,
// all accumulating in FP32 in TMEM.  SRW_FP16X3 issues the same three
// products on FP16 halves (11 significant bits each instead of 8): every row
// j of R is stored scaled by r_j and every point's W - W_ref by s_p, exact
// powers of two that bring the largest element to [2^13, 2^14) (FP16 keeps
// full precision from 2^-14 up to 65504); the epilogue multiplies the
// accumulator by 1 / (s_p r_j), which is exact.  The accumulator is double-buffered
// (2 x BN columns) so the epilogue of one tile overlaps the next tile's MMAs.
//
// Each rec tile runs only the range of K blocks in which its split response
// has nonzero elements (kbr, from create time); the skipped blocks hold
// zeros in both halves, so their products are exact zeros.
//
// Grouped launches (several detector configurations with their own binning,
// response, data and points in one persistent grid) use the same kernel: each
// work item names its configuration, whose descriptor (tensor maps, spectra,
// per-bin constants, tile width) the roles read per item.  The host builds the
// item lists (see group.cu).
//
// Every wait is bounded (ptx.cuh); on a timeout the CTA raises
// kStatusTimeout, drains its outstanding copies and MMAs, frees TMEM and ends.

#include <cuda.h>

#include <cmath>
#include <vector>

#include "dfloat.cuh"
#include "poisson.cuh"
#include "ptx.cuh"
#include "srw_internal.h"
#include "tc.cuh"

namespace srw {
namespace {

using namespace tc;

constexpr int kBM = 128;   // points per tile (MMA M, TMEM lanes)
constexpr int kBK = 64;    // true bins per block of the zero-block ranges (and the widest stage)
constexpr int kWWarps = 8;
constexpr int kEpiWarp0 = 8;
constexpr int kTmaWarp = 12;
constexpr int kMmaWarp = 13;
constexpr int kShatWarp = 14;
constexpr int kThreads = 15 * 32;

// Pipeline stage of BK true bins (BK = 64: rows of 128 bytes, 128-byte
// swizzle; BK = 32: rows of 64 bytes, 64-byte swizzle, twice the stages in
// the same shared memory, so the R tiles' TMA loads are issued further ahead
// of the MMAs that consume them).  The W producers write 16-byte chunks of 8
// true bins: BK / 8 chunks per row.  With BK = 64 the eight producer warps
// take one chunk each; with BK = 32 they form two groups of four that take
// turns over the stages, so each warp still computes four rows of eight bins
// (the coefficient-spectra loads of a chunk feed four rows).
template <int BK>
struct KStage {
  static constexpr int kShatBytes = BK * kNB * 4;       // coefficient spectra of one stage (k-major)
  static constexpr int kShatSlots = 4 * kBK / BK;       // depth of the coefficient-spectra ring (256 true bins)
  static constexpr int kChunks = BK / 8;                // 16-byte chunks of a tile row
  static constexpr int kGroups = kWWarps / kChunks;     // producer warp groups taking turns over the stages
  static constexpr int kPerBlock = kBK / BK;            // stages per block of the zero-block ranges
};

struct TcMaps {
  // [stage width: 0 = 64, 1 = 32 true bins][box rows: 0 = 128, 1 = 256]
  CUtensorMap hi[2][2], lo[2][2];      // BF16 split
  CUtensorMap hi16[2][2], lo16[2][2];  // FP16 split of the row-scaled R
};

__device__ __forceinline__ uint32_t pack_f16x2(float a, float b) {
  const __half2 v = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// hi / lo halves of two values: hi = round(x), lo = round(x - hi), packed in pairs.
template <bool F16>
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  // the residuals (a, b) - hi are exact in FP32; one packed subtraction forms both
  float2 h2;
  if (F16) {
    hi = pack_f16x2(a, b);
    h2 = __half22float2(*reinterpret_cast<const __half2*>(&hi));
  } else {
    hi = pack_bf16x2(a, b);
    h2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&hi));
  }
  uint64_t r;
  asm("sub.rn.f32x2 %0, %1, %2;"
      : "=l"(r)
      : "l"((uint64_t)__float_as_uint(a) | ((uint64_t)__float_as_uint(b) << 32)),
        "l"((uint64_t)__float_as_uint(h2.x) | ((uint64_t)__float_as_uint(h2.y) << 32)));
  const float ra = __uint_as_float((uint32_t)r), rb = __uint_as_float((uint32_t)(r >> 32));
  lo = F16 ? pack_f16x2(ra, rb) : pack_bf16x2(ra, rb);
}

// Power of two s with s * bound in [2^13, 2^14): the FP16 scale of values
// bounded by `bound` in magnitude (1 if bound is 0).
__device__ __forceinline__ float pow2_scale(float bound) {
  if (!(bound > 0.f)) return 1.f;
  int e;
  frexpf(bound, &e);  // bound = m 2^e, m in [0.5, 1)
  e = e < -100 ? -100 : (e > 100 ? 100 : e);
  return ldexpf(1.f, 14 - e);
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

template <int BN, bool X3, int BK = kBK>
struct TcShape {
  using K = KStage<BK>;
  static constexpr int kAB = kBM * BK * 2;              // bytes of one BF16 A tile
  static constexpr int kBB = BN * BK * 2;               // bytes of one BF16 B tile
  static constexpr int kStageBytes = (X3 ? 2 : 1) * (kAB + kBB);
  static constexpr int kShatRing = K::kShatSlots * K::kShatBytes;
  static constexpr int kStages = (200 * 1024 - kShatRing) / kStageBytes;
  static constexpr int kSmem = kStages * kStageBytes + kShatRing + 1024;  // + alignment slack
  static constexpr int kAccCols = BN;  // TMEM columns of one item's accumulator
  static constexpr int kBufs = 2;      // items in flight in TMEM (the epilogue overlaps the next MMAs)
  static constexpr int kTmemCols = kBufs * kAccCols;
};

// K blocks of a rec tile in the order the fold accumulates them: kr = {first
// block, +count} walks up from `first`, {first, -count} walks down (and the
// 16-wide MMA steps inside a stage then run down too, so that the true bins
// are accumulated in strictly decreasing order whatever the stage width).
// kr counts blocks of kBK = 64 true bins; with BK = 32 each is two stages.
// The direction is chosen per tile at create time (see tc_block_ranges).
template <int BK>
__device__ __forceinline__ int kb_count(int2 kr) {
  return KStage<BK>::kPerBlock * (kr.y >= 0 ? kr.y : -kr.y);
}
template <int BK>
__device__ __forceinline__ int kb_at(int2 kr, int kk) {
  constexpr int R = KStage<BK>::kPerBlock;
  return kr.y >= 0 ? R * kr.x + kk : R * kr.x + (R - 1) - kk;
}

constexpr int kMaxGroups = 4096;  // configurations of one grouped launch
constexpr int kPrefetch = 2;      // R blocks prefetched into L2 this many stages ahead
constexpr double kL2ResidentBytes = 64.0 * 1024 * 1024;  // responses up to this size stay in L2 (129 MB)

// K-block walk of the rec tile at n0.  (Staging the walks, or the epilogue's
// per-bin constants, in shared memory was measured: no gain, and 4.8 % slower
// for the constants.)
template <bool GROUPED, int BN>
__device__ __forceinline__ int2 tile_walk(const TcGroup& G, int n0) {
  return G.kbr[n0 / (GROUPED ? G.bn : BN)];
}

// Kernel parameters.  A single-configuration launch walks the m x n tiles of
// g0 with a grid stride; a grouped launch walks per-CTA item lists.
struct TcLaunch {
  TcGroup g0;                  // single configuration (its maps are kernel parameters of their own)
  const TcGroup* groups;       // grouped: one per configuration (nullptr: single)
  const int4* items;           // grouped: slot k * gridDim.x + b = {group, m0, n0, 0}, CTA b's k-th item
  int n_items;                 // single: m_tiles x n_tiles; grouped: slots
  // per point (a group's points start at p_off) two float4: {c0, c1, c2, c3}
  // and {c4, c5, c7, s}, the seven point-dependent coupling coefficients
  // (the constant monomial c6 is always in the reference fold) times the
  // point's power-of-two scale s, and s itself (1 unless SRW_FP16X3); written
  // by coef_kernel / group_coef_kernel
  const float4* coef;
  double* parts;
  float* musig_out;            // single configuration only: [P][n_rec] folded deviations
  unsigned* status;
  int inject;                  // injected timeout (host-side fault injection): CTA 0's epilogue gives up
  int prefetch;                // 1: prefetch R blocks into L2 ahead of the ring (responses that L2 does not hold)
};

// Item loops: a grid stride written directly in blockIdx / gridDim / a kernel
// parameter, which the compiler can see are warp-uniform.  Loop bounds taken
// from memory (per-CTA list offsets) made the fold 6-8% slower: the loops hold
// .sync.aligned tcgen05 instructions and bounded waits.  A grouped launch
// therefore stores CTA b's k-th item at slot k * gridDim.x + b, and each list
// ends with a stop item (group < 0).
#define FOR_ITEMS(idx) for (int idx = (int)blockIdx.x; idx < L.n_items; idx += (int)gridDim.x)

// Configuration (by value) and tile origin of work item idx (gi < 0: a stop
// item of a grouped launch).  A single-
// configuration launch takes its descriptor from the kernel parameters, so its
// fields stay constant-bank operands (no address of a parameter is taken).
template <bool GROUPED, int BN>
__device__ __forceinline__ TcGroup work_at(const TcLaunch& L, int idx, int& m0, int& n0, int& gi) {
  if (!GROUPED) {
    // rec-tile-major: the grid stride walks every CTA across all rec tiles,
    // whose K-block ranges (and so costs) differ
    const int mt = (L.g0.P + kBM - 1) / kBM;
    m0 = (idx % mt) * kBM;
    n0 = (idx / mt) * BN;
    gi = 0;
    return L.g0;
  }
  const int4 it = L.items[idx];
  m0 = it.y;
  n0 = it.z;
  gi = it.x;
  return L.groups[it.x < 0 ? 0 : it.x];
}

// Orders the host's writes of a tensor map in global memory before its use
// by the TMA unit (tensormap proxy).
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map))
               : "memory");
}

// BN: widest rec tile of the launch; it fixes the shared-memory stages and the
// TMEM accumulators.  In a grouped launch each configuration's tile width
// bn <= BN is a runtime value (TMA box, MMA N, epilogue columns); a single
// configuration uses bn = BN.
template <int BN, int BK, bool X3, bool GROUPED, bool F16>
__global__ void __launch_bounds__(kThreads, 1)
fold_tc_kernel(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo, const TcLaunch L) {
  using S = TcShape<BN, X3, BK>;
  using KS = KStage<BK>;
  constexpr int ST = S::kStages;
  constexpr int NB = S::kBufs;
  constexpr int kShatSlots = KS::kShatSlots;
  constexpr int kShatBytes = KS::kShatBytes;
  extern __shared__ unsigned char dsmem_raw[];
  // 1024-byte aligned base for the swizzled tiles, formed by pointer arithmetic on
  // the shared array so that plain loads through it stay shared-memory loads
  // (a round trip through an integer makes them generic loads: slower, and on
  // the long scoreboard)
  unsigned char* smem = dsmem_raw + ((1024u - (ptx::smem_addr(dsmem_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t r_full[ST], w_full[ST], empty[ST], acc_full[NB], acc_empty[NB], drain;
  __shared__ __align__(8) uint64_t s_full[kShatSlots], s_empty[kShatSlots], never;
  __shared__ uint32_t tmem_slot;
  __shared__ unsigned abort_flag;
  __shared__ uint32_t map_fenced[GROUPED ? kMaxGroups / 32 : 1];  // maps already acquired by the R producer

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned* status = L.status;
  double* const parts = L.parts;
  float* const musig_out = L.musig_out;

  auto a_hi = [&](int st) { return smem + (size_t)st * S::kStageBytes; };
  auto a_lo = [&](int st) { return smem + (size_t)st * S::kStageBytes + S::kAB; };
  auto b_hi = [&](int st) { return smem + (size_t)st * S::kStageBytes + (X3 ? 2 : 1) * S::kAB; };
  auto b_lo = [&](int st) { return smem + (size_t)st * S::kStageBytes + 2 * S::kAB + S::kBB; };
  auto shat_s = [&](int slot) {
    return reinterpret_cast<float4*>(smem + (size_t)ST * S::kStageBytes + (size_t)slot * kShatBytes);
  };

  if (GROUPED)
    for (int i = threadIdx.x; i < kMaxGroups / 32; i += blockDim.x) map_fenced[i] = 0u;
  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      ptx::mbar_init(&r_full[s], 1);
      ptx::mbar_init(&w_full[s], kWWarps / KS::kGroups);
      ptx::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < NB; ++b) {
      ptx::mbar_init(&acc_full[b], 1);
      ptx::mbar_init(&acc_empty[b], 4);
    }
    for (int q = 0; q < kShatSlots; ++q) {
      ptx::mbar_init(&s_full[q], 1);
      ptx::mbar_init(&s_empty[q], kWWarps / KS::kGroups);
    }
    ptx::mbar_init(&drain, 1);
    ptx::mbar_init(&never, 1);  // nothing arrives on it (injected timeout)
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
    // chunk `ch`; the coefficient-spectra loads are warp-uniform and each
    // feeds 32 FMAs (shared-memory wavefronts are the scarce resource here).
    // With BK = 32 warp group `wg` produces the stages g with g % 2 == wg.
    const int rg = lane;
    const int ch = warp % KS::kChunks;  // 16-byte chunk = 8 consecutive k
    const int wg = warp / KS::kChunks;
    int g = 0;            // global K-block counter (stage ring position)
    FOR_ITEMS(idx) {
      if (__any_sync(0xffffffffu, aborted(&abort_flag))) break;
      int m0, n0, gi;
      const TcGroup G = work_at<GROUPED, BN>(L, idx, m0, n0, gi);
      if (GROUPED && gi < 0) break;  // stop item: this CTA's list is done
      // K blocks of this rec tile that hold nonzero response (the rest add exact zeros)
      const int2 kr = tile_walk<GROUPED, BN>(G, n0);
      // the coefficients of this thread's four points, computed once per point
      // by the pre-pass (not once per W warp and item)
      float c[4][kNB - 1];
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) {
        const int p = m0 + rg + 32 * rr;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
        if (p < G.P) {
          a = __ldg(L.coef + 2 * ((size_t)G.p_off + p));
          b = __ldg(L.coef + 2 * ((size_t)G.p_off + p) + 1);
        }
        c[rr][0] = a.x; c[rr][1] = a.y; c[rr][2] = a.z; c[rr][3] = a.w;
        c[rr][4] = b.x; c[rr][5] = b.y; c[rr][6] = b.z;
      }
      bool ok = true;
      for (int kk = 0; kk < kb_count<BK>(kr); ++kk, ++g) {
        if (KS::kGroups > 1 && g % KS::kGroups != wg) continue;  // the other group's stage
        const int st = g % ST, sl = g % kShatSlots;
        // the A buffers of this stage are free once the MMAs of its previous
        // use have completed; the coefficient spectra come through their own ring
        if (!warp_wait(&empty[st], ((g / ST) & 1) ^ 1, &abort_flag) ||
            !warp_wait(&s_full[sl], (g / kShatSlots) & 1, &abort_flag)) {
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
              for (int bb = 1; bb < kNB; ++bb)  // the constant monomial (6) is always in the reference fold
                if (bb != 6) a = fmaf(c[rr][bb < 6 ? bb : 6], sv[bb], a);
              w[rr][e] = a;
            }
          }
#pragma unroll
          for (int rr = 0; rr < 4; ++rr) {
            if (X3) split2<F16>(w[rr][0], w[rr][1], h[rr][q], l[rr][q]);
            else h[rr][q] = pack_bf16x2(w[rr][0], w[rr][1]);
          }
        }
        // the four rows share the swizzle phase (rows 32 apart)
        const uint32_t off = swz_offset<BK>(rg, ch);
        const uint32_t ah = ptx::smem_addr(a_hi(st)), al = ptx::smem_addr(a_lo(st));
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
          const uint32_t ro = (uint32_t)(32 * rr * 2 * BK) + off;
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
    // injected timeout (host-side fault injection): one warp of CTA 0 waits for
    // an arrival that never comes, with a 1 ms limit, and gives up
    if (L.inject && blockIdx.x == 0 && q == 0 &&
        !__all_sync(0xffffffffu, ptx::mbar_wait(&never, 0, &abort_flag, 1000000ull)))
      give_up();
    // once this CTA has given up, every item it has not finished gets a NaN
    // partial, so the affected points read NaN instead of a stale value
    bool dead = false;
    int tc = -1;
    FOR_ITEMS(idx) {
      ++tc;
      int m0, n0, gi;
      const TcGroup G = work_at<GROUPED, BN>(L, idx, m0, n0, gi);
      if (GROUPED && gi < 0) break;  // stop item: this CTA's list is done
      const int bn = GROUPED ? G.bn : BN, nt = n0 / bn, n_rec = G.n_rec, P = G.P;
      const int buf = tc % NB;
      const int p = m0 + q * 32 + lane;
      if (!dead && __any_sync(0xffffffffu, aborted(&abort_flag))) dead = true;
      if (!dead && !warp_wait(&acc_full[buf], (tc / NB) & 1, &abort_flag)) {
        give_up();
        dead = true;
      }
      SRW_CHECK(status, nt >= 0 && nt < G.n_tiles && m0 >= 0 && m0 < P);
      if (dead) {
        if (parts != nullptr && p < P)
          parts[G.parts_off + (long long)nt * P + p] = __longlong_as_double(0x7ff8000000000000LL);
        continue;
      }
      tc_fence_after();
      const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * S::kAccCols);
      float sinv = 1.f;  // 1 / s_p (exact: s_p is a power of two)
      if (F16 && p < P) sinv = 1.f / __ldg(L.coef + 2 * ((size_t)G.p_off + p) + 1).w;
      dfloat acc = {0.f, 0.f};
      bool infinite = false;  // a +inf term (mu <= 0 with data) is kept apart: TwoSum would make it NaN
      float mneg = 0.f;       // smallest mu of the active bins (below 0: outside the domain)
#pragma unroll 1
      for (int c0 = 0; c0 < bn; c0 += 16) {
        // per-column constants first (warp-uniform loads), then the accumulator row
        float4 dj[16];
        if (parts != nullptr) {
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int j = n0 + c0 + k;
            // {n_j (0 where masked), b_j + R W_ref - n_j, mask, 1/r_j}; padding columns add nothing
            dj[k] = j < n_rec ? __ldg(G.nb4 + j) : make_float4(0.f, 1.f, 0.f, 0.f);
          }
        } else {  // folded spectra only (no data needed): just the row scales
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int j = n0 + c0 + k;
            dj[k] = make_float4(0.f, 0.f, 0.f, F16 && j < n_rec ? __ldg(G.rinv + j) : 0.f);
          }
        }
        float v[16];
        tmem_ld16(tbase + (uint32_t)c0, v);
        if (musig_out != nullptr && p < P) {  // batched folded spectra (row p)
          float* row = musig_out + (size_t)(G.p_off + p) * n_rec;
#pragma unroll
          for (int k = 0; k < 16; ++k)
            if (n0 + c0 + k < n_rec) row[n0 + c0 + k] = F16 ? v[k] * (sinv * dj[k].w) : v[k];
        }
        if (parts != nullptr) {
          float ts = 0.f;
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            // mu - n (the power-of-two scales of both operands come out exactly)
            const float dm = F16 ? fmaf(v[k], sinv * dj[k].w, dj[k].y) : v[k] + dj[k].y;
            ts = fmaf(poisson_term_f32_dm(dm, dj[k].x), dj[k].z, ts);
            mneg = fminf(mneg, (dj[k].x + dm) * dj[k].z);
          }
          if (isinf(ts) || isnan(ts)) infinite = true;
          else acc = df_add(acc, ts);
        }
      }
      if (mneg < 0.f) infinite = true;
      tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&acc_empty[buf]);
      if (parts != nullptr && p < P)
        parts[G.parts_off + (long long)nt * P + p] =
            infinite ? __longlong_as_double(0x7ff0000000000000LL) : (double)acc.hi + (double)acc.lo;
    }
  } else if (warp == kTmaWarp) {
    // ------------------------------------------------------------ TMA producers
    if (lane == 0) {  // R hi (+ lo) tiles into the stage ring
      int g = 0, issued_g = 0;
      bool ok = true;
      FOR_ITEMS(idx) {
        if (!ok || aborted(&abort_flag)) break;
        int m0, n0, gi;
        const TcGroup G = work_at<GROUPED, BN>(L, idx, m0, n0, gi);
        if (GROUPED && gi < 0) break;  // stop item: this CTA's list is done
        const int2 kr = tile_walk<GROUPED, BN>(G, n0);
        const uint32_t bytes = (uint32_t)((X3 ? 2 : 1) * (GROUPED ? G.bn : BN) * BK * 2);
        const CUtensorMap* mh = &map_hi;
        const CUtensorMap* ml = &map_lo;
        if (GROUPED) {
          mh = G.map_hi;
          ml = G.map_lo;
          if (!((map_fenced[gi >> 5] >> (gi & 31)) & 1u)) {
            tensormap_acquire(mh);
            if (X3) tensormap_acquire(ml);
            map_fenced[gi >> 5] |= 1u << (gi & 31);
          }
        }
        for (int kk = 0; kk < kb_count<BK>(kr); ++kk, ++g) {
          const int kb = kb_at<BK>(kr, kk);
          const int st = g % ST;
          if (!ptx::mbar_wait(&empty[st], ((g / ST) & 1) ^ 1, &abort_flag)) {
            give_up();
            ok = false;
            break;
          }
          SRW_CHECK(status, kb >= 0 && kb < G.k_pad / BK && n0 >= 0 && n0 < G.n_tiles * (GROUPED ? G.bn : BN));
          ptx::mbar_arrive_expect_tx(&r_full[st], bytes);
          tma_load_2d(b_hi(st), mh, kb * BK, n0, &r_full[st]);
          if (X3) tma_load_2d(b_lo(st), ml, kb * BK, n0, &r_full[st]);
          // warm L2 with the block kPrefetch stages ahead: with a two-stage ring
          // a response that does not stay in L2 (many configurations, or one
          // large one) would otherwise expose the HBM latency at every stage
          if (L.prefetch && kk + kPrefetch < kb_count<BK>(kr)) {
            const int kbp = kb_at<BK>(kr, kk + kPrefetch);
            tma_prefetch_2d(mh, kbp * BK, n0);
            if (X3) tma_prefetch_2d(ml, kbp * BK, n0);
          }
          issued_g = g + 1;
        }
      }
      // never end with copies in flight
      for (int u = max(0, issued_g - ST); u < issued_g; ++u)
        ptx::mbar_wait(&r_full[u % ST], (u / ST) & 1, nullptr, 100000000ull);
    }
  } else if (warp == kShatWarp) {
    // ------------------------------------------------------------ coefficient spectra
    // its own warp: a lane of the R producer's warp would share that warp's
    // (mostly suspended) instruction stream
    if (lane == 0) {  // one 2 KB slice per K block, up to kShatSlots blocks ahead
      int g = 0, issued = 0;
      bool ok = true;
      FOR_ITEMS(idx) {
        if (!ok) break;
        int m0, n0, gi;
        const TcGroup G = work_at<GROUPED, BN>(L, idx, m0, n0, gi);
        if (GROUPED && gi < 0) break;  // stop item: this CTA's list is done
        const int2 kr = tile_walk<GROUPED, BN>(G, n0);
        for (int kk = 0; kk < kb_count<BK>(kr); ++kk, ++g) {
          const int kb = kb_at<BK>(kr, kk);
          const int sl = g % kShatSlots;
          if (!ptx::mbar_wait(&s_empty[sl], ((g / kShatSlots) & 1) ^ 1, &abort_flag)) {
            give_up();
            ok = false;
            break;
          }
          SRW_CHECK(status, kb >= 0 && (kb + 1) * BK <= G.k_pad);
          ptx::mbar_arrive_expect_tx(&s_full[sl], (uint32_t)kShatBytes);
          ptx::bulk_g2s(shat_s(sl), G.shat_k8 + (size_t)kb * BK * 2, (uint32_t)kShatBytes, &s_full[sl]);
          issued = g + 1;
        }
      }
      for (int u = max(0, issued - kShatSlots); u < issued; ++u)
        ptx::mbar_wait(&s_full[u % kShatSlots], (u / kShatSlots) & 1, nullptr, 100000000ull);
    }
  } else {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int g = 0;
      bool issued_any = false;
      int tc = -1;
      FOR_ITEMS(idx) {
        ++tc;
        if (aborted(&abort_flag)) break;
        int m0, n0, gi;
        const TcGroup G = work_at<GROUPED, BN>(L, idx, m0, n0, gi);
        if (GROUPED && gi < 0) break;  // stop item: this CTA's list is done
        const int2 kr = tile_walk<GROUPED, BN>(G, n0);
        const uint32_t idesc = idesc_f16kind(kBM, GROUPED ? G.bn : BN, F16);
        const int buf = tc % NB;
        if (!ptx::mbar_wait(&acc_empty[buf], ((tc / NB) & 1) ^ 1, &abort_flag)) {
          give_up();
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(buf * S::kAccCols);
        const bool down = kr.y < 0;  // descending walk: the MMA steps inside a block run down too
        bool ok = true;
        for (int kk = 0; kk < kb_count<BK>(kr); ++kk, ++g) {
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
          for (int q = 0; q < BK / 16; ++q) {
            const int ks = down ? BK / 16 - 1 - q : q;
            const uint32_t off = (uint32_t)ks * 32u;  // 16 BF16 along K inside the swizzle atom
            const uint32_t acc = (kk != 0) || q != 0;  // the item's first update initialises
            mma_bf16(d_tmem, smem_desc_k<BK>(ah + off), smem_desc_k<BK>(bh + off), idesc, acc);
            if (X3) {
              mma_bf16(d_tmem, smem_desc_k<BK>(ah + off), smem_desc_k<BK>(bl + off), idesc, 1u);
              mma_bf16(d_tmem, smem_desc_k<BK>(al + off), smem_desc_k<BK>(bh + off), idesc, 1u);
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

// R -> FP16 hi + lo of r_j R_j (one block per padded row): r_j is the power of
// two that brings the row's largest element to [2^13, 2^14); rinv = 1 / r_j.
__global__ void split_r16_kernel(const float* __restrict__ R, int n_rec, int ld, int k_pad, __half* __restrict__ rhi,
                                 __half* __restrict__ rlo, float* __restrict__ rinv) {
  __shared__ float red[32];
  const int j = blockIdx.x;
  const float* row = R + (size_t)j * ld;
  float m = 0.f;
  if (j < n_rec)
    for (int k = threadIdx.x; k < ld; k += blockDim.x) m = fmaxf(m, fabsf(row[k]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) red[0] = m;
  }
  __syncthreads();
  const float r = pow2_scale(red[0]);
  if (j < n_rec && threadIdx.x == 0) rinv[j] = 1.f / r;
  for (int k = threadIdx.x; k < k_pad; k += blockDim.x) {
    const float x = (j < n_rec && k < ld) ? row[k] * r : 0.f;
    const __half h = __float2half_rn(x);
    rhi[(size_t)j * k_pad + k] = h;
    rlo[(size_t)j * k_pad + k] = __float2half_rn(x - __half2float(h));
  }
}

// Per-point coefficients of the W producers.  The FP16 scale s_p is the power
// of two of the bound sum_b |c_b - c_b,ref| max_i |shat_b,i| of the weighted-
// spectrum deviations (FP32 products and sums without contraction, so every
// caller gets the same power of two); the BF16 splits use s_p = 1.
__device__ __forceinline__ void point_coef(const float* th, const TcGroup& G, bool f16, float4* out) {
  float c[kNB];
  coefficients(th, dfloat{G.sin2w_hi, G.sin2w_lo}, G.cref, c);
  float sc = 1.f;
  if (f16) {
    float bound = 0.f;
#pragma unroll
    for (int b = 0; b < kNB; ++b) bound = __fadd_rn(bound, __fmul_rn(fabsf(c[b]), G.wmax[b]));
    sc = pow2_scale(bound);
  }
  // exact: sc is a power of two
  out[0] = make_float4(c[0] * sc, c[1] * sc, c[2] * sc, c[3] * sc);
  out[1] = make_float4(c[4] * sc, c[5] * sc, c[7] * sc, sc);
}

__global__ void coef_kernel(const TcGroup g0, const float* __restrict__ theta, int f16, float4* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < g0.P) point_coef(theta + (size_t)p * 5, g0, f16 != 0, out + 2 * (size_t)p);
}

__global__ void group_coef_kernel(const TcGroup* __restrict__ groups, const float* __restrict__ theta, int f16,
                                  float4* __restrict__ out) {
  const TcGroup G = groups[blockIdx.y];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < G.P)
    point_coef(theta + ((size_t)G.p_off + p) * 5, G, f16 != 0, out + 2 * ((size_t)G.p_off + p));
}

__global__ void shat_k8_kernel(const float* __restrict__ shat, int k_pad, float* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= k_pad) return;
#pragma unroll
  for (int b = 0; b < kNB; ++b) out[(size_t)k * kNB + b] = shat[(size_t)b * k_pad + k];
}

// Nonzero flags of the (rec tile, K block) pairs of one split: block (kb, t)
// reads the bn x 64 elements of hi and lo in 16-byte pieces (+-0 counts as
// zero: it adds nothing).  The host turns the flags into each tile's range.
__global__ void kb_flags_kernel(const uint4* __restrict__ hi, const uint4* __restrict__ lo, int n_rec, int k_pad,
                                int bn, unsigned char* __restrict__ flags) {
  const int kb = blockIdx.x, t = blockIdx.y;
  const int pieces = k_pad / 8;  // 16-byte pieces per row
  bool nz = false;
  for (int q = threadIdx.x; q < bn * (kBK / 8); q += blockDim.x) {
    const int r = t * bn + q / (kBK / 8);
    if (r < n_rec) {
      const size_t i = (size_t)r * pieces + (size_t)kb * (kBK / 8) + (q % (kBK / 8));
      const uint4 a = hi[i], b = lo[i];
      nz |= ((a.x | a.y | a.z | a.w | b.x | b.y | b.z | b.w) & 0x7fff7fffu) != 0u;
    }
  }
  nz = __syncthreads_or(nz);
  if (threadIdx.x == 0) flags[(size_t)t * gridDim.x + kb] = nz ? 1 : 0;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

template <int BN, int BK, bool X3, bool F16, bool GROUPED>
cudaError_t set_attr1() {
  return cudaFuncSetAttribute(fold_tc_kernel<BN, BK, X3, GROUPED, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              TcShape<BN, X3, BK>::kSmem);
}

// Every instantiation a launch can select: both stage widths for single
// configurations; grouped launches use 64-wide stages.
template <int BN>
cudaError_t set_attr_all() {
  cudaError_t e = cudaSuccess;
#define SRW_ATTR(...) \
  if (e == cudaSuccess) e = set_attr1<__VA_ARGS__>()
  SRW_ATTR(BN, 64, true, false, false);
  SRW_ATTR(BN, 64, true, true, false);
  SRW_ATTR(BN, 64, false, false, false);
  SRW_ATTR(BN, 32, true, false, false);
  SRW_ATTR(BN, 32, true, true, false);
  SRW_ATTR(BN, 32, false, false, false);
  SRW_ATTR(BN, 64, true, false, true);
  SRW_ATTR(BN, 64, true, true, true);
  SRW_ATTR(BN, 64, false, false, true);
#undef SRW_ATTR
  return e;
}

template <int BN, int BK, bool X3, bool GROUPED, bool F16>
cudaError_t launch_kernel(const CUtensorMap& mh, const CUtensorMap& ml, const TcLaunch& L, int grid, cudaStream_t s) {
  fold_tc_kernel<BN, BK, X3, GROUPED, F16><<<grid, kThreads, TcShape<BN, X3, BK>::kSmem, s>>>(mh, ml, L);
  return launch_result();
}

template <int BN, int BK, bool GROUPED>
cudaError_t launch_prec(int precision, const CUtensorMap& mh, const CUtensorMap& ml, const TcLaunch& L, int grid,
                        cudaStream_t s) {
  if (precision == SRW_FP16X3) return launch_kernel<BN, BK, true, GROUPED, true>(mh, ml, L, grid, s);
  if (precision == SRW_BF16X3) return launch_kernel<BN, BK, true, GROUPED, false>(mh, ml, L, grid, s);
  return launch_kernel<BN, BK, false, GROUPED, false>(mh, ml, L, grid, s);
}

cudaError_t launch_single(int bn, int bk, int precision, const CUtensorMap& mh, const CUtensorMap& ml,
                          const TcLaunch& L, int grid, cudaStream_t s) {
  if (bn == 256) return bk == 32 ? launch_prec<256, 32, false>(precision, mh, ml, L, grid, s)
                                 : launch_prec<256, 64, false>(precision, mh, ml, L, grid, s);
  return bk == 32 ? launch_prec<128, 32, false>(precision, mh, ml, L, grid, s)
                  : launch_prec<128, 64, false>(precision, mh, ml, L, grid, s);
}

cudaError_t launch_grouped(int bn_max, int precision, const CUtensorMap& mh, const CUtensorMap& ml, const TcLaunch& L,
                           int grid, cudaStream_t s) {
  if (bn_max == 256) return launch_prec<256, 64, true>(precision, mh, ml, L, grid, s);
  return launch_prec<128, 64, true>(precision, mh, ml, L, grid, s);
}

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (fn == nullptr) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q);
    if (e == cudaSuccess && p != nullptr && q == cudaDriverEntryPointSuccess) fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

}  // namespace

bool tc_supported(const srw_ctx* h) { return h->cc_major == 10 && h->cc_minor == 3; }

// Tensor-core fold configurations (the autotuner's candidates).  Every
// candidate accumulates each output element from the same updates in the
// same order, so they differ in speed only.
static const FoldConfig kConfigs[] = {
    {1, 256, 64, TcShape<256, true, 64>::kStages, kWWarps},
    {1, 256, 32, TcShape<256, true, 32>::kStages, kWWarps},
    {1, 128, 64, TcShape<128, true, 64>::kStages, kWWarps},
    {1, 128, 32, TcShape<128, true, 32>::kStages, kWWarps},
};

int tc_num_configs() { return (int)(sizeof(kConfigs) / sizeof(kConfigs[0])); }
FoldConfig tc_config(int i) { return kConfigs[i]; }

cudaError_t launch_split_r(srw_ctx* h, cudaStream_t s) {
  const size_t n = (size_t)h->rec_pad * h->k_pad;
  split_r_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(h->d_R, h->n_rec, h->ld_r, h->rec_pad, h->k_pad,
                                                             h->d_rhi, h->d_rlo);
  split_r16_kernel<<<h->rec_pad, 256, 0, s>>>(h->d_R, h->n_rec, h->ld_r, h->k_pad, h->d_rhi16, h->d_rlo16, h->d_rinv);
  shat_k8_kernel<<<(h->k_pad + 255) / 256, 256, 0, s>>>(h->d_shat, h->k_pad, h->d_shat_k8);
  return launch_result();
}

cudaError_t tc_encode_maps(const srw_ctx* h, int bn, bool f16, CUtensorMap* hi, CUtensorMap* lo, int bk) {
  EncodeTiledFn encode = encode_fn();
  if (encode == nullptr) return cudaErrorNotSupported;
  if (bk != 64 && bk != 32) return cudaErrorInvalidValue;
  const cuuint64_t dims[2] = {(cuuint64_t)h->k_pad, (cuuint64_t)h->rec_pad};
  const cuuint64_t strides[1] = {(cuuint64_t)h->k_pad * 2};
  const cuuint32_t estr[2] = {1, 1};
  const cuuint32_t box[2] = {(cuuint32_t)bk, (cuuint32_t)bn};  // a box row is one swizzle span (128 or 64 bytes)
  for (int l = 0; l < 2; ++l) {
    void* base = f16 ? (l ? (void*)h->d_rlo16 : (void*)h->d_rhi16) : (l ? (void*)h->d_rlo : (void*)h->d_rhi);
    CUresult r = encode(l ? lo : hi, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base,
                        dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

cudaError_t tc_prepare(srw_ctx* h) {
  cudaError_t ea = set_attr_all<256>();
  if (ea == cudaSuccess) ea = set_attr_all<128>();
  if (ea != cudaSuccess) return ea;
  TcMaps* maps = new (std::nothrow) TcMaps();
  if (!maps) return cudaErrorMemoryAllocation;
  for (int ki = 0; ki < 2; ++ki)
  for (int bi = 0; bi < 2; ++bi) {
    const int bk = ki ? 32 : 64;
    cudaError_t e = tc_encode_maps(h, bi ? 256 : 128, false, &maps->hi[ki][bi], &maps->lo[ki][bi], bk);
    if (e == cudaSuccess) e = tc_encode_maps(h, bi ? 256 : 128, true, &maps->hi16[ki][bi], &maps->lo16[ki][bi], bk);
    if (e != cudaSuccess) {
      delete maps;
      return e;
    }
  }
  h->tmap = maps;
  return cudaSuccess;
}

void tc_release(srw_ctx* h) {
  delete static_cast<TcMaps*>(h->tmap);
  h->tmap = nullptr;
}

// Accumulation order of one rec tile's K blocks.  The tensor core's FP32
// accumulation drops the bits of every update below the accumulator's last
// place, so the error a row collects grows with the number of updates made
// after its sum has become large.  Walking the blocks from the tiny end of a
// row's response towards its peak keeps the sum small while most updates are
// made; which end that is depends on the response (a one-sided tail, several
// bands).  The choice is made here, at create time, by replaying the tile's
// accumulation of R (weights 1, steps of 16 true bins, each update rounded
// toward zero to FP32) in both directions and keeping the one whose summed
// error over the tile's rows is smaller; ties keep ascending order.
static bool descending_is_better(const std::vector<float>& R, int ld, int n_rec, int row0, int rows, int kb0,
                                 int kb1) {
  auto rz = [](double x) {
    float f = (float)x;
    if (std::fabs((double)f) > std::fabs(x)) f = std::nextafter(f, 0.f);
    return f;
  };
  double err[2] = {0.0, 0.0};
  for (int r = row0; r < row0 + rows && r < n_rec; ++r) {
    const float* row = R.data() + (size_t)r * ld;
    for (int dir = 0; dir < 2; ++dir) {
      float acc = 0.f;
      double exact = 0.0;
      const int nsteps = (kb1 - kb0) * (kBK / 16);
      for (int q = 0; q < nsteps; ++q) {
        const int step = dir ? (kb1 * (kBK / 16) - 1 - q) : (kb0 * (kBK / 16) + q);
        double part = 0.0;
        for (int k = step * 16; k < step * 16 + 16 && k < ld; ++k) part += (double)row[k];
        if (part == 0.0) continue;
        exact += part;
        acc = rz((double)acc + part);
      }
      err[dir] += std::fabs(exact - (double)acc);
    }
  }
  return err[1] < err[0];
}

// K-block range {first, end} of each rec tile of width bn: the blocks of 64
// true bins in which some row of the tile has a nonzero hi or lo element.
// Outside the range every product is an exact zero, so the folds skip those
// blocks without changing a bit of the accumulation.  A tile without any
// nonzero element keeps one block (its accumulator must still be written).
// The device copy holds the walk {first block, +-count} (see kb_at).
cudaError_t tc_block_ranges(srw_ctx* h, const std::vector<float>& R, cudaStream_t s) {
  const int n_kb = h->k_pad / kBK;
  unsigned char* d_flags = nullptr;
  const int max_tiles = (h->n_rec + 127) / 128;
  cudaError_t e = dev_malloc(&d_flags, (size_t)max_tiles * n_kb);
  if (e != cudaSuccess) return e;
  std::vector<unsigned char> flags((size_t)max_tiles * n_kb);
  // direction per group of 256 rows (both tile widths use it, so that every
  // output element accumulates the same updates in the same order whichever
  // width a launch uses; skipped blocks only ever add exact zeros)
  std::vector<char> down[2];
  for (int f16 = 0; f16 < 2 && e == cudaSuccess; ++f16)
    for (int bi = 1; bi >= 0 && e == cudaSuccess; --bi) {
      const int bn = bi ? 256 : 128, n_tiles = (h->n_rec + bn - 1) / bn;
      const uint4* hi = reinterpret_cast<const uint4*>(f16 ? (const void*)h->d_rhi16 : (const void*)h->d_rhi);
      const uint4* lo = reinterpret_cast<const uint4*>(f16 ? (const void*)h->d_rlo16 : (const void*)h->d_rlo);
      kb_flags_kernel<<<dim3(n_kb, n_tiles), 256, 0, s>>>(hi, lo, h->n_rec, h->k_pad, bn, d_flags);
      if ((e = launch_result()) != cudaSuccess) break;
      if ((e = cudaMemcpyAsync(flags.data(), d_flags, (size_t)n_tiles * n_kb, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
          (e = cudaStreamSynchronize(s)) != cudaSuccess)
        break;
      std::vector<int2>& r = h->kbr_h[f16][bi];
      r.assign(n_tiles, make_int2(0, 1));
      std::vector<int2> walk(n_tiles, make_int2(0, 1));
      for (int t = 0; t < n_tiles; ++t) {
        int first = -1, last = -1;
        for (int kb = 0; kb < n_kb; ++kb)
          if (flags[(size_t)t * n_kb + kb]) {
            if (first < 0) first = kb;
            last = kb;
          }
        if (first >= 0) {
          r[t] = make_int2(first, last + 1);
          if (bi) down[f16].push_back(descending_is_better(R, h->ld_r, h->n_rec, t * bn, bn, first, last + 1));
          walk[t] = down[f16][bi ? t : t / 2] ? make_int2(last, -(last + 1 - first))
                                              : make_int2(first, last + 1 - first);
        } else if (bi) {
          down[f16].push_back(0);
        }
      }
      if ((e = dev_malloc(&h->d_kbr[f16][bi], sizeof(int2) * n_tiles)) != cudaSuccess) break;
      h->device_bytes += sizeof(int2) * n_tiles;
      e = cudaMemcpy(h->d_kbr[f16][bi], walk.data(), sizeof(int2) * n_tiles, cudaMemcpyHostToDevice);
    }
  cudaFree(d_flags);
  return e;
}

double tc_block_fraction(const srw_ctx* h, int bn, bool f16) {
  const std::vector<int2>& r = h->kbr_h[f16 ? 1 : 0][bn == 256 ? 1 : 0];
  const int n_kb = h->k_pad / kBK;
  if (r.empty() || n_kb == 0) return 1.0;
  double used = 0.0;
  for (const int2& t : r) used += t.y - t.x;
  return used / ((double)r.size() * n_kb);
}

TcGroup tc_group_of(const srw_ctx* h, int bn, bool f16) {
  TcGroup G{};
  G.kbr = h->d_kbr[f16 ? 1 : 0][bn == 256 ? 1 : 0];
  G.map_hi = G.map_lo = nullptr;
  G.shat_k8 = reinterpret_cast<const float4*>(h->d_shat_k8);
  G.nb4 = h->d_nb4;
  G.c_data = h->d_cdata;
  G.parts_off = 0;
  G.n_rec = h->n_rec;
  G.k_pad = h->k_pad;
  G.P = 0;
  G.p_off = 0;
  G.bn = bn;
  G.n_tiles = (h->n_rec + bn - 1) / bn;
  const dfloat s2w = df_from_double(h->sin2w);
  G.sin2w_hi = s2w.hi;
  G.sin2w_lo = s2w.lo;
  G.cref = h->cref;
  G.rinv = h->d_rinv;
  for (int b = 0; b < kNB; ++b) G.wmax[b] = h->wmax[b];
  return G;
}

cudaError_t launch_fold_tc(const srw_ctx* h, const float* theta, int P, int precision, const FoldConfig& cfg,
                           double* parts, cudaStream_t s, int* n_parts, float* musig_out, cudaEvent_t ev_begin,
                           cudaEvent_t ev_end) {
  const TcMaps* maps = static_cast<const TcMaps*>(h->tmap);
  if (!maps) return cudaErrorNotSupported;
  const int bn = cfg.bn == 256 ? 256 : 128, bi = bn == 256 ? 1 : 0;
  const bool f16 = precision == SRW_FP16X3;
  TcLaunch L{};
  L.g0 = tc_group_of(h, bn, f16);
  L.g0.P = P;
  L.groups = nullptr;
  L.items = nullptr;
  L.n_items = ((P + kBM - 1) / kBM) * L.g0.n_tiles;
  L.coef = h->d_coef;
  L.parts = parts;
  L.musig_out = musig_out;
  L.status = h->d_status;
  L.inject = inject_timeout();
  // a response whose splits fill more than about half of L2 is streamed from HBM
  L.prefetch = (double)h->rec_pad * h->k_pad * 2.0 * 2.0 > kL2ResidentBytes ? 1 : 0;
  if (n_parts) *n_parts = L.g0.n_tiles;
  if (h->d_coef == nullptr || h->coef_cap < P) return cudaErrorInvalidValue;
  coef_kernel<<<(P + 255) / 256, 256, 0, s>>>(L.g0, theta, f16 ? 1 : 0, h->d_coef);
  const int grid = L.n_items < h->sm_count ? L.n_items : h->sm_count;
  cudaError_t e;
  // optional events around the fold kernel alone (not the coefficient pre-pass)
  if (ev_begin && (e = cudaEventRecord(ev_begin, s)) != cudaSuccess) return e;
  const int bk = cfg.bk == 32 ? 32 : 64, ki = bk == 32 ? 1 : 0;
  e = launch_single(bn, bk, precision, f16 ? maps->hi16[ki][bi] : maps->hi[ki][bi],
                    f16 ? maps->lo16[ki][bi] : maps->lo[ki][bi], L, grid, s);
  if (e == cudaSuccess && ev_end) e = cudaEventRecord(ev_end, s);
  return e;
}

cudaError_t launch_group_coef(const TcGroup* d_groups, int n_groups, int max_P, const float* theta, bool f16,
                              float4* out, cudaStream_t s) {
  if (n_groups < 1 || max_P < 1) return cudaSuccess;
  group_coef_kernel<<<dim3((max_P + 255) / 256, n_groups), 256, 0, s>>>(d_groups, theta, f16 ? 1 : 0, out);
  return launch_result();
}

cudaError_t launch_fold_tc_group(int bn_max, int precision, const TcGroup* d_groups, const int4* d_items, int n_slots,
                                 int n_cta, const float4* coef, double* parts, unsigned* status,
                                 cudaStream_t s) {
  if (n_cta < 1) return cudaSuccess;
  TcLaunch L{};
  L.groups = d_groups;
  L.items = d_items;
  L.n_items = n_slots;
  L.coef = coef;
  L.parts = parts;
  L.musig_out = nullptr;
  L.status = status;
  L.inject = inject_timeout();
  L.prefetch = 1;  // the configurations' responses together rarely stay in L2
  static const CUtensorMap unused{};  // grouped launches read each configuration's maps from its descriptor
  return launch_grouped(bn_max == 256 ? 256 : 128, precision, unused, unused, L, n_cta, s);
}

int tc_max_groups() { return kMaxGroups; }

}  // namespace srw
