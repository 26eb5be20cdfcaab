// Single-point fold + Poisson reduction, data set-up and partial-sum reduction.
//
// Fold (eq. visible_spectrum / eq. matrix_reweight):
//   mu_sig_j = sum_i R_ji W_i,  W_i = w_i(theta) E_SM,i
// Expectation (eq. mu_total) and -2 ln L (eq. logL):
//   mu_j = M_j (mu_sig_j + b_j),  -2lnL = C + 2 sum_j t(mu_j, n_j)
//
// The single-point fold is a GEMV bound by HBM bandwidth: R (n_rec x k_pad
// FP32) is read exactly once.  It is streamed into shared memory by the TMA
// engine (bulk async copies completing on mbarriers), so the number of bytes
// in flight per SM is set by the ring depth rather than by registers.  The
// Poisson term and the bin reduction are FP64 and fused into the same launch
// (the last block to finish sums the per-block partials in block order).

#include <algorithm>
#include <mutex>
#include <vector>
#include <string>

#include "dfloat.cuh"
#include "poisson.cuh"
#include "ptx.cuh"
#include "srw_internal.h"

namespace srw {
namespace {

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// One block per SM owns a contiguous range of rows.  A producer warp streams
// the rows' nonzero bands into a kGvStages-deep ring of 16 KB stages (several
// short bands share a stage, in a segment table built at create); the rows
// are dealt in turn to eight consumer warps, which multiply them by W (read
// through L1), keep FP32 partial sums over at most eight float4 a lane and
// fold them into a double-float per-lane accumulator; at the end of a row two
// shuffle rounds fold the 32 lanes into 8 shares, left in shared memory, and
// the epilogue adds them (a full warp reduction per row was a serial chain
// on the stream's critical path; 32 shares per row would not fit in shared
// memory at the largest row counts).  Every consumer warp releases every
// stage with one arrive.  Every wait is bounded (see ptx.cuh); a block that
// gives up raises kStatusTimeout.
// ---------------------------------------------------------------------------
constexpr int kGvConsumers = 8;
constexpr int kGvThreads = (kGvConsumers + 1) * 32;
constexpr int kGvChunk = 4096;  // floats per stage (16 KB)
constexpr int kGvStages = 6;
constexpr int kGvShares = 8;  // shares of a row a warp leaves (its 32 lanes folded in two shuffle rounds)
constexpr int kGvRowCost = 1024;  // floats: the fixed cost of one row's copy, see gemv_prepare

// One segment of a block's stream: `len` floats (a multiple of 32) of the
// block's row `row` from column k0, at float offset `off` of the block's ring
// stage number `stage`; `done` marks the row's last segment.  Segments come
// in stage order, and the segments of a row are consecutive.
struct GvSeg {
  int row, k0, len, off, stage;
  bool done;
};

// Create-time table entry {row | done << 30, k0, len, off | stage << 16}.
__device__ __forceinline__ GvSeg gv_unpack(int4 v) {
  return {v.x & 0x3fffffff, v.y, v.z, v.w & 0xffff, v.w >> 16, ((v.x >> 30) & 1) != 0};
}

// Without a table every row is streamed whole, cut into chunk-sized
// segments, one segment per stage.
__device__ __forceinline__ GvSeg gv_dense(int i, int ld, int chunk) {
  const int per_row = (ld + chunk - 1) / chunk, part = i % per_row, k0 = part * chunk;
  return {i / per_row, k0, min(chunk, ld - k0), 0, i, part == per_row - 1};
}

// Row stride of the per-row shares [share][row]: odd, so that the shares of a
// row land in different banks.
__host__ __device__ constexpr int gv_part_stride(int rows) { return rows | 1; }

__global__ void __launch_bounds__(kGvThreads, 1)
fold_point_kernel(const float* __restrict__ R, int n_rec, int ld, int rows_per_block, const float* __restrict__ W,
                  const double* __restrict__ muref, const double* __restrict__ n64, const double* __restrict__ b64,
                  const unsigned char* __restrict__ mask, const double* __restrict__ c_data,
                  float* __restrict__ musig_out, float* __restrict__ mu_out, double* __restrict__ parts,
                  unsigned* __restrict__ ticket, double* __restrict__ out, unsigned* __restrict__ status,
                  int inject, const int4* __restrict__ seg, const int* __restrict__ seg_start,
                  const int* __restrict__ row_start) {
  extern __shared__ __align__(128) unsigned char dsmem[];
  const int chunk = ld < kGvChunk ? ld : kGvChunk;
  const int ps = gv_part_stride(rows_per_block);
  float* sbuf = reinterpret_cast<float*>(dsmem);
  float2* spart = reinterpret_cast<float2*>(dsmem + sizeof(float) * (size_t)kGvStages * chunk);
  int4* sseg = reinterpret_cast<int4*>(spart + (size_t)kGvShares * ps);
  __shared__ __align__(8) uint64_t full[kGvStages], empty[kGvStages], never;
  __shared__ unsigned abort_flag;
  __shared__ double sred[kGvThreads / 32];
  __shared__ bool is_last;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // rows of this block: an even split, or (row_start) a split that balances
  // the blocks' estimated stream times (see gemv_prepare)
  const int r0 = row_start ? row_start[blockIdx.x] : blockIdx.x * rows_per_block;
  const int r1 = row_start ? row_start[blockIdx.x + 1] : min(n_rec, r0 + rows_per_block);
  const int nrows = r1 > r0 ? r1 - r0 : 0;
  // The epilogue's inputs of a thread's first row (row threadIdx.x) do not
  // depend on W: they are loaded here, so that their cold misses pass while R
  // streams instead of after it; rows beyond the block size load later.
  double ep_ref = 0.0, ep_b = 0.0, ep_n = 0.0, ep_c = 0.0;
  bool ep_on = true;
  if ((int)threadIdx.x < nrows) {
    const int j = r0 + threadIdx.x;
    if (muref != nullptr) ep_ref = __ldg(muref + j);
    if (b64 != nullptr) ep_b = __ldg(b64 + j);
    if (mask != nullptr) ep_on = __ldg(mask + j) != 0;
    if (out != nullptr) ep_n = __ldg(n64 + j);
  }
  if (out != nullptr && threadIdx.x == 0) ep_c = __ldg(c_data);  // used by the last block
  // the block's segments: from the create-time table (each row's nonzero
  // band, outside which R is exactly zero, short bands packed several to a
  // stage), staged in shared memory so that no walk waits on global memory;
  // else whole padded rows
  const int s0 = seg ? seg_start[blockIdx.x] : 0;
  const int nseg = seg ? seg_start[blockIdx.x + 1] - s0 : nrows * ((ld + chunk - 1) / chunk);
  if (seg)
    for (int i = threadIdx.x; i < nseg; i += blockDim.x) sseg[i] = seg[s0 + i];
  auto seg_at = [&](int i) { return seg ? gv_unpack(sseg[i]) : gv_dense(i, ld, chunk); };

  if (threadIdx.x == 0) {
    for (int st = 0; st < kGvStages; ++st) {
      ptx::mbar_init(&full[st], 1);
      ptx::mbar_init(&empty[st], kGvConsumers);
    }
    ptx::mbar_init(&never, 1);  // nothing arrives on it (injected timeout)
    abort_flag = 0u;
    ptx::fence_barrier_init();
  }
  __syncthreads();

  if (warp == kGvConsumers) {
    // ---- producer (one lane): every segment posts its bytes and its copy;
    // one arrive closes a stage
    if (lane == 0) {
      int cur = -1;
      bool ok = true;
      for (int i = 0; i < nseg; ++i) {
        const GvSeg g = seg_at(i);
        if (g.stage != cur) {
          if (cur >= 0) ptx::mbar_arrive(&full[cur % kGvStages]);
          cur = g.stage;
          if (cur >= kGvStages &&
              !ptx::mbar_wait(&empty[cur % kGvStages], ((cur / kGvStages) - 1) & 1, &abort_flag)) {
            atomicExch(&abort_flag, 1u);
            atomicOr(status, kStatusTimeout);
            ok = false;
            break;
          }
        }
        SRW_CHECK(status, g.row >= 0 && g.row < nrows && g.k0 >= 0 && g.len > 0 && g.k0 + g.len <= ld &&
                              (g.len & 31) == 0 && g.off >= 0 && g.off + g.len <= chunk);
        const int st = cur % kGvStages;
        ptx::mbar_expect_tx(&full[st], (uint32_t)g.len * 4u);
        ptx::bulk_g2s(sbuf + (size_t)st * chunk + g.off, R + (size_t)(r0 + g.row) * ld + g.k0, (uint32_t)g.len * 4u,
                      &full[st]);
      }
      if (ok && cur >= 0) ptx::mbar_arrive(&full[cur % kGvStages]);
      const int issued = ok ? cur + 1 : cur;  // stages whose copies were all posted
      // never let the block end with copies in flight
      for (int u = max(0, issued - kGvStages); u < issued; ++u)
        ptx::mbar_wait(&full[u % kGvStages], (u / kGvStages) & 1, nullptr, 100000000ull);
    }
  } else {
    // ---- consumers (no FP64 here: the chunk sums accumulate as double-floats)
    // W may come from a grid this one depends on programmatically: wait for it
    // (returns at once without such a dependency); the producer's R stream
    // does not depend on it and is already running
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // injected timeout (host-side fault injection, block 0): consumer warp 0
    // waits for an arrival that never comes, with a 1 ms limit, and gives up
    // exactly as when a copy never completes
    if (inject && blockIdx.x == 0 && warp == 0 && !ptx::mbar_wait(&never, 0, &abort_flag, 1000000ull)) {
      atomicExch(&abort_flag, 1u);
      atomicOr(status, kStatusTimeout);
    }
    dfloat lacc = {0.f, 0.f};
    int cur = -1;
    bool ok = true;
    for (int i = 0; i < nseg; ++i) {
      const GvSeg g = seg_at(i);
      if (g.stage != cur) {
        if (cur >= 0) {
          __syncwarp();
          if (lane == 0) ptx::mbar_arrive(&empty[cur % kGvStages]);
        }
        cur = g.stage;
        // warp-uniform: no lane runs on into the next stage or a __syncwarp alone
        ok = __all_sync(0xffffffffu, ptx::mbar_wait(&full[cur % kGvStages], (cur / kGvStages) & 1, &abort_flag));
        if (!ok) {
          if (lane == 0) {
            atomicExch(&abort_flag, 1u);
            atomicOr(status, kStatusTimeout);
          }
          break;
        }
      }
      // rows are dealt to the warps in turn: a warp sums whole rows (all
      // segments of a row go to the same warp), and the rows of different
      // warps stream in parallel
      if (g.row % kGvConsumers != warp) continue;
      const float4* buf = reinterpret_cast<const float4*>(sbuf + (size_t)(cur % kGvStages) * chunk + g.off);
      const float4* w4 = reinterpret_cast<const float4*>(W + g.k0);
      const int n4 = g.len / 4;
      for (int q0 = 0; q0 < n4; q0 += 8 * 32) {  // FP32 partials over at most 8 float4 a lane
        const int qe = min(n4, q0 + 8 * 32);
        float ax = 0.f, ay = 0.f, az = 0.f, aw = 0.f;
#pragma unroll 4
        for (int q = q0 + lane; q < qe; q += 32) {
          const float4 r = buf[q];
          const float4 w = __ldg(w4 + q);
          ax = fmaf(r.x, w.x, ax);
          ay = fmaf(r.y, w.y, ay);
          az = fmaf(r.z, w.z, az);
          aw = fmaf(r.w, w.w, aw);
        }
        lacc = df_add(lacc, (ax + ay) + (az + aw));
      }
      if (g.done) {  // two shuffle rounds fold the lanes into 8 shares; the epilogue adds them
        SRW_CHECK(status, g.row < rows_per_block);
        lacc = df_add(lacc, df_shfl_xor(lacc, 16));
        lacc = df_add(lacc, df_shfl_xor(lacc, 8));
        if (lane < kGvShares) spart[(size_t)lane * ps + g.row] = make_float2(lacc.hi, lacc.lo);
        lacc = {0.f, 0.f};
      }
    }
    if (ok && cur >= 0) {
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&empty[cur % kGvStages]);
    }
  }
  __syncthreads();

  // ---- epilogue: mu_j, FP64 Poisson terms, block partial (NaN for a block
  // that gave up, so that the point's value is NaN, never a wrong number)
  double t = abort_flag != 0u ? __longlong_as_double(0x7ff8000000000000LL) : 0.0;
  if (abort_flag == 0u) {
    for (int rl = threadIdx.x; rl < nrows; rl += kGvThreads) {
      const int j = r0 + rl;
      dfloat ms = {0.f, 0.f};  // the row's sum: the shares its warp left
      for (int l = 0; l < kGvShares; ++l) {
        const float2 v = spart[(size_t)l * ps + rl];
        ms = df_add(ms, dfloat{v.x, v.y});
      }
      const bool first = rl == (int)threadIdx.x;  // the row whose inputs are loaded
      // delta mode: W holds W(theta) - W_ref, and the FP64 reference fold is added back
      const double ref = first ? ep_ref : (muref != nullptr ? muref[j] : 0.0);
      const double musig = (double)ms.hi + (double)ms.lo + ref;
      const bool on = first ? ep_on : (mask == nullptr || mask[j] != 0);
      const double mu = on ? musig + (first ? ep_b : (b64 != nullptr ? b64[j] : 0.0)) : 0.0;
      if (musig_out) musig_out[j] = (float)musig;
      if (mu_out) mu_out[j] = (float)mu;
      if (on && out) {
        const double tj = poisson_term_f64(mu, first ? ep_n : n64[j]);
        if (isinf(tj)) atomicOr(status, kStatusDomain);
        t += tj;
      }
    }
  }
  if (out == nullptr) return;
  t = warp_sum_d(t);
  if (lane == 0) sred[warp] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kGvThreads / 32; ++w) s += sred[w];
    parts[blockIdx.x] = s;
    __threadfence();
    const unsigned prev = atomicAdd(ticket, 1u);
    is_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  // last block: fixed-order FP64 sum of all partials
  __threadfence();
  double s = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += kGvThreads) s += ((volatile double*)parts)[b];
  s = warp_sum_d(s);
  __syncthreads();
  if (lane == 0) sred[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < kGvThreads / 32; ++w) tot += sred[w];
    out[0] = 2.0 * tot + ep_c;
    *ticket = 0u;
  }
}

// out[p] = 2 sum_t parts[t][p] + C  (fixed order over t).
__global__ void reduce_parts_kernel(const double* __restrict__ parts, int n_parts, int P,
                                    const double* __restrict__ c_data, double* __restrict__ out,
                                    unsigned* __restrict__ status) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  double s = 0.0;
  SRW_CHECK(status, n_parts >= 1);
  for (int t = 0; t < n_parts; ++t) s += parts[(size_t)t * P + p];
  const double v = 2.0 * s + *c_data;
  if (isinf(v)) atomicOr(status, kStatusDomain);
  out[p] = v;
}

// --- data set-up --------------------------------------------------------------
__global__ void data_prepare_kernel(const double* __restrict__ bkg, int n_bkg, int n_rec,
                                    double* __restrict__ b64) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_rec) return;
  double b = 0.0;
  for (int k = 0; k < n_bkg; ++k) b += bkg[(size_t)k * n_rec + j];
  b64[j] = b;
}

// Per-bin constants of the batched epilogues: reference fold + background,
// in FP64 (SIMT fold) and as floats with the count and the mask (tensor fold).
__global__ void data_ref_kernel(const double* __restrict__ n64, const double* __restrict__ b64,
                                const double* __restrict__ muref, const unsigned char* __restrict__ mask, int n_rec,
                                const float* __restrict__ rinv, double* __restrict__ bref64, float4* __restrict__ nbm,
                                float2* __restrict__ nb2, float4* __restrict__ nb4) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_rec) return;
  const double br = b64[j] + muref[j];
  bref64[j] = br;
  const bool on = mask == nullptr || mask[j] != 0;
  nbm[j] = make_float4((float)n64[j], (float)br, on ? 1.f : 0.f, 0.f);
  nb2[j] = make_float2(on ? (float)n64[j] : -1.f, (float)br);
  // tensor-core epilogue: mu - n is formed from b + R W_ref - n, rounded once from FP64
  if (nb4) nb4[j] = make_float4(on ? (float)n64[j] : 0.f, (float)(on ? br - n64[j] : br), on ? 1.f : 0.f,
                                rinv ? rinv[j] : 1.f);
}

// C = 2 sum_j M_j [n_j - n_j ln n_j + lnGamma(n_j + 1)], one block.
__global__ void cdata_kernel(const double* __restrict__ n64, const unsigned char* __restrict__ mask, int n_rec,
                             double* __restrict__ c_out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int j = threadIdx.x; j < n_rec; j += blockDim.x) {
    if (mask != nullptr && mask[j] == 0) continue;
    const double n = n64[j];
    const double nlogn = n > 0.0 ? n * log(n) : 0.0;
    s += n - nlogn + lgamma(n + 1.0);
  }
  s = warp_sum_d(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *c_out = 2.0 * t;
  }
}

}  // namespace

static int gv_uniform_rows(const srw_ctx* h) {
  const int g = h->sm_count > 0 ? h->sm_count : 148;
  return (h->n_rec + g - 1) / g;
}

// Rows per block: the even split, or the largest block of the band-balanced split.
static int gv_rows_per_block(const srw_ctx* h) { return h->gv_blocks > 0 ? h->gv_max_rows : gv_uniform_rows(h); }

int fold_point_grid(const srw_ctx* h) {
  const int rpb = gv_uniform_rows(h);
  return (h->n_rec + rpb - 1) / rpb;
}

static size_t gv_smem(const srw_ctx* h) {
  const int chunk = h->ld_r < kGvChunk ? h->ld_r : kGvChunk;
  return sizeof(float) * (size_t)kGvStages * chunk +
         sizeof(float2) * kGvShares * (size_t)gv_part_stride(gv_rows_per_block(h)) +
         sizeof(int4) * (size_t)(h->gv_blocks > 0 ? h->gv_max_segs : 0);
}

// Per row of R its nonzero band [lo, hi): lo the first nonzero column rounded
// down to 4 floats (16-byte copies), the length rounded up to 32 floats and
// kept inside the padded row; an all-zero row keeps 32 columns.  The rows are
// split over the fold_point_grid blocks so that each takes about the same
// time to stream: a row costs its band plus kGvRowCost floats, the fixed cost
// of the bulk copy that brings it in (measured on GB300: a copy takes about
// 0.16 us plus 0.04 us per KB, one after another on an SM, so a block of many
// short rows is bound by its number of copies); each block's bands are cut
// into its stream segments: consecutive bands packed into stages of up to
// kGvChunk floats, a band that does not fit in the rest of a started stage
// opening the next one, a band longer than a stage cut into stage-sized
// pieces.
cudaError_t gemv_prepare(srw_ctx* h, const std::vector<float>& R) {
  const int n_rec = h->n_rec, ld = h->ld_r, chunk = ld < kGvChunk ? ld : kGvChunk;
  std::vector<int2> band(n_rec);
  long long total = 0;
  for (int r = 0; r < n_rec; ++r) {
    const float* row = R.data() + (size_t)r * ld;
    int first = -1, last = -1;
    for (int k = 0; k < ld; ++k)
      if (row[k] != 0.f) {
        if (first < 0) first = k;
        last = k;
      }
    int lo = first < 0 ? 0 : first / 4 * 4;
    int len = first < 0 ? 32 : (last + 1 - lo + 31) / 32 * 32;
    if (len > ld) len = ld;
    if (lo + len > ld) lo = ld - len;
    band[r] = make_int2(lo, lo + len);
    total += len + kGvRowCost;
  }
  const int nb = fold_point_grid(h);
  std::vector<int> start(nb + 1, n_rec);
  start[0] = 0;
  long long acc = 0;
  int b = 1, max_rows = 0;
  for (int r = 0; r < n_rec && b < nb; ++r) {
    acc += band[r].y - band[r].x + kGvRowCost;
    if (acc * nb >= total * b) start[b++] = r + 1;
  }
  for (int k = 0; k < nb; ++k) max_rows = std::max(max_rows, start[k + 1] - start[k]);
  // segments {row | done << 30, k0, len, off | stage << 16}, block by block
  std::vector<int4> seg;
  std::vector<int> seg_start(nb + 1, 0);
  int max_segs = 0;
  for (int k = 0; k < nb; ++k) {
    seg_start[k] = (int)seg.size();
    int stage = 0, fill = 0;
    for (int r = start[k]; r < start[k + 1]; ++r) {
      int k0 = band[r].x;
      while (k0 < band[r].y) {
        const int rem = band[r].y - k0;
        if (fill > 0 && rem > chunk - fill) {  // does not fit: next stage
          ++stage;
          fill = 0;
        }
        const int len = std::min(rem, chunk - fill);
        const int done = len == rem ? 1 : 0;
        if (stage >= 32768) return cudaErrorInvalidValue;
        seg.push_back(make_int4((r - start[k]) | (done << 30), k0, len, fill | (stage << 16)));
        fill += len;
        k0 += len;
        if (fill == chunk) {
          ++stage;
          fill = 0;
        }
      }
    }
    max_segs = std::max(max_segs, (int)seg.size() - seg_start[k]);
  }
  seg_start[nb] = (int)seg.size();
  cudaError_t e = cudaSuccess;
  if (!h->d_gv_seg && (e = dev_malloc(&h->d_gv_seg, sizeof(int4) * seg.size())) != cudaSuccess) return e;
  if (!h->d_gv_segs && (e = dev_malloc(&h->d_gv_segs, sizeof(int) * (size_t)(nb + 1))) != cudaSuccess) return e;
  if (!h->d_gv_rows && (e = dev_malloc(&h->d_gv_rows, sizeof(int) * (size_t)(nb + 1))) != cudaSuccess) return e;
  h->device_bytes += sizeof(int4) * seg.size() + 2 * sizeof(int) * (size_t)(nb + 1);
  if ((e = cudaMemcpy(h->d_gv_seg, seg.data(), sizeof(int4) * seg.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(h->d_gv_segs, seg_start.data(), sizeof(int) * (size_t)(nb + 1), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(h->d_gv_rows, start.data(), sizeof(int) * (size_t)(nb + 1), cudaMemcpyHostToDevice)) != cudaSuccess)
    return e;
  long long bytes = 0;
  for (const int2& x : band) bytes += 4LL * (x.y - x.x);
  h->gv_blocks = nb;
  h->gv_max_rows = max_rows;
  h->gv_max_segs = max_segs;
  h->gv_bytes = bytes;
  return cudaSuccess;
}

void fold_point_init() {
  cudaFuncSetAttribute(fold_point_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

cudaError_t launch_fold_point(const srw_ctx* h, const float* W, float* musig_out, float* mu_out, double* out,
                              cudaStream_t s, bool delta) {
  const size_t smem = gv_smem(h);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  const double* muref = delta ? h->d_muref64 : nullptr;
  fold_point_kernel<<<fold_point_grid(h), kGvThreads, smem, s>>>(
      h->d_R, h->n_rec, h->ld_r, gv_rows_per_block(h), W, muref, h->d_n64, h->d_b64, h->d_mask, h->d_cdata, musig_out,
      mu_out, h->d_part, h->d_ticket, out, h->d_status, inject_timeout(), h->gv_blocks > 0 ? h->d_gv_seg : nullptr,
      h->gv_blocks > 0 ? h->d_gv_segs : nullptr, h->gv_blocks > 0 ? h->d_gv_rows : nullptr);
  return launch_result();
}

cudaError_t launch_fold_point_after(const srw_ctx* h, const float* W, double* out, cudaStream_t s) {
  const size_t smem = gv_smem(h);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  const double* muref = h->d_muref64;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(fold_point_grid(h));
  cfg.blockDim = dim3(kGvThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, fold_point_kernel, (const float*)h->d_R, h->n_rec, h->ld_r,
                                           gv_rows_per_block(h), W, muref, (const double*)h->d_n64,
                                           (const double*)h->d_b64, (const unsigned char*)h->d_mask,
                                           (const double*)h->d_cdata, (float*)nullptr, (float*)nullptr, h->d_part,
                                           h->d_ticket, out, h->d_status, inject_timeout(),
                                           (const int4*)(h->gv_blocks > 0 ? h->d_gv_seg : nullptr),
                                           (const int*)(h->gv_blocks > 0 ? h->d_gv_segs : nullptr),
                                           (const int*)(h->gv_blocks > 0 ? h->d_gv_rows : nullptr));
  return e != cudaSuccess ? e : launch_result();
}

cudaError_t launch_reduce_parts(const srw_ctx* h, const double* parts, int n_parts, int P, double* out,
                                cudaStream_t s) {
  const int thr = 256;
  reduce_parts_kernel<<<(P + thr - 1) / thr, thr, 0, s>>>(parts, n_parts, P, h->d_cdata, out, h->d_status);
  return launch_result();
}

cudaError_t launch_set_data(srw_ctx* h, const double* d_bkg, int n_bkg, cudaStream_t s) {
  const int thr = 256;
  data_prepare_kernel<<<(h->n_rec + thr - 1) / thr, thr, 0, s>>>(d_bkg, n_bkg, h->n_rec, h->d_b64);
  cdata_kernel<<<1, 1024, 0, s>>>(h->d_n64, h->d_mask, h->n_rec, h->d_cdata);
  return launch_data_ref(h, s);
}

cudaError_t launch_data_ref(srw_ctx* h, cudaStream_t s) {
  const int thr = 256;
  data_ref_kernel<<<(h->n_rec + thr - 1) / thr, thr, 0, s>>>(h->d_n64, h->d_b64, h->d_muref64, h->d_mask, h->n_rec,
                                                             h->d_rinv, h->d_bref64, h->d_nbm, h->d_nb2, h->d_nb4);
  cudaError_t e = launch_result();
  if (e == cudaSuccess && h->d_lin) e = launch_linear_consts(h, s);
  return e;
}

// out[p][j] += mu_ref[j]: folded spectra of the batched path from deviations.
__global__ void add_ref_kernel(float* __restrict__ out, const double* __restrict__ muref, int P, int n_rec) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)P * n_rec) return;
  out[idx] += (float)muref[idx % n_rec];
}

cudaError_t launch_add_ref(const srw_ctx* h, float* out, int P, cudaStream_t s) {
  const size_t n = (size_t)P * h->n_rec;
  add_ref_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, h->d_muref64, P, h->n_rec);
  return launch_result();
}

}  // namespace srw

// ---------------------------------------------------------------------------
// Allocation-free single-point likelihood.
//
// For callers that cannot allocate device memory themselves: code that runs
// inside another framework's memory manager, which owns every device
// allocation, or code that must not call cudaMalloc/cudaFree because those
// calls can synchronise the whole device.  They pass all inputs and the output
// as device pointers; the scratch the kernels need (per-block partial sums,
// the data-only constant of -2 ln L, the last-block ticket and the status
// word) lives in the file-scope array below, which every GPU that loads this
// library holds until the process exits.
// ---------------------------------------------------------------------------
namespace srw {
namespace {

constexpr int kNoAllocMaxBlocks = 1024;  // partial sums: one per block of the fold
constexpr int kNoAllocMaxRec = 65536;    // reconstructed bins
struct NoAllocScratch {
  double parts[kNoAllocMaxBlocks];
  double c_data;
  unsigned ticket;
  unsigned status;
};
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

struct NoAllocDevice {
  NoAllocScratch* scratch = nullptr;  // device address of g_noalloc_scratch
  int sm_count = 0;
  bool ready = false;
};
constexpr int kNoAllocMaxDevices = 64;
NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];

}  // namespace
}  // namespace srw

static std::mutex g_noalloc_mutex;
static thread_local std::string g_noalloc_err;

extern "C" srw_status srw_loglik_point_noalloc(const float* R, int n_rec, int ld, const float* W,
                                               const double* counts, const double* bkg, const unsigned char* mask,
                                               double* out, void* stream) {
  using namespace srw;
  auto bad = [](const char* m) {
    g_noalloc_err = m;
    return SRW_EINVAL;
  };
  if (!R || !W || !counts || !out) return bad("R, W, counts and out must be device pointers");
  if (n_rec < 1 || n_rec > kNoAllocMaxRec) return bad("n_rec must lie in [1, 65536]");
  if (ld < 64 || ld % 64 != 0) return bad("ld must be a positive multiple of 64");
  if (((uintptr_t)R % 16) != 0 || ((uintptr_t)W % 16) != 0) return bad("R and W must be 16-byte aligned");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    g_noalloc_err = cudaGetErrorString(e);
    return SRW_ECUDA;
  }
  if (dev < 0 || dev >= kNoAllocMaxDevices) return bad("device index out of range");
  NoAllocDevice& nd = g_noalloc_dev[dev];
  {
    // once per device, with that device current: resolve the device address
    // of the scratch array (its host-side name is only a stand-in)
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!nd.ready) {
      void* p = nullptr;
      if ((e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess ||
          (e = cudaDeviceGetAttribute(&nd.sm_count, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
          (e = cudaFuncSetAttribute(fold_point_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)) !=
              cudaSuccess) {
        g_noalloc_err = cudaGetErrorString(e);
        return SRW_ECUDA;
      }
      nd.scratch = static_cast<NoAllocScratch*>(p);
      nd.ready = true;
    }
  }
  const int g = nd.sm_count > 0 ? nd.sm_count : 148;
  const int rpb = (n_rec + g - 1) / g;
  const int grid = (n_rec + rpb - 1) / rpb;
  if (grid > kNoAllocMaxBlocks) return bad("too many blocks for the scratch array");
  const int chunk = ld < kGvChunk ? ld : kGvChunk;
  const size_t smem =
      sizeof(float) * (size_t)kGvStages * chunk + sizeof(float2) * kGvShares * (size_t)gv_part_stride(rpb);
  if (smem > 200 * 1024) return bad("n_rec too large for the fold's shared memory");
  cudaStream_t s = (cudaStream_t)stream;
  NoAllocScratch* sc = nd.scratch;
  // the array keeps the previous call's contents: the ticket and the status must start at zero
  if ((e = cudaMemsetAsync(&sc->ticket, 0, 2 * sizeof(unsigned), s)) != cudaSuccess) {
    g_noalloc_err = cudaGetErrorString(e);
    return SRW_ECUDA;
  }
  cdata_kernel<<<1, 1024, 0, s>>>(counts, mask, n_rec, &sc->c_data);
  fold_point_kernel<<<grid, kGvThreads, smem, s>>>(R, n_rec, ld, rpb, W, nullptr, counts, bkg, mask, &sc->c_data,
                                                    nullptr, nullptr, sc->parts, &sc->ticket, out, &sc->status,
                                                    inject_timeout(), nullptr, nullptr, nullptr);
  if ((e = launch_result()) != cudaSuccess) {
    g_noalloc_err = cudaGetErrorString(e);
    return SRW_ECUDA;
  }
  return SRW_OK;
}

extern "C" const char* srw_noalloc_last_error(void) { return g_noalloc_err.c_str(); }
