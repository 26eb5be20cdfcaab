// Grouped evaluation: several detector configurations in one persistent
// tensor-core fold launch (srw_group_* in srw.h).
//
// Each configuration g keeps its own handle (binning, BF16 response, data,
// reference point).  A work item is one 128-point x bn-bin tile of one
// configuration; its cost is proportional to the configuration's K blocks.
// The host schedule sorts the items longest-first (keeping the items of one
// rec tile of one configuration adjacent, so the CTAs that run them at the
// same time share that response slice in L2) and gives each to the least-
// loaded CTA; every CTA then walks its own list in the persistent kernel,
// stored with a grid stride (CTA b's k-th item at slot k * n_cta + b, each
// list closed by a stop item).

#include <algorithm>
#include <cmath>
#include <new>
#include <queue>
#include <string>
#include <vector>

#include "srw_internal.h"

namespace srw {
namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;

// Relative cost of one item in K blocks of a 256-wide tile: a 128-wide tile
// does half the MMAs but the same weighted-spectrum production, and each item
// pays a fixed prologue / epilogue.
double item_cost(int n_kb, int bn) { return bn == 256 ? n_kb + 2.0 : 0.93 * n_kb + 1.0; }

__global__ void group_reduce_kernel(const GroupPart* __restrict__ gp, const double* __restrict__ parts,
                                    double* __restrict__ out, unsigned* __restrict__ status) {
  const GroupPart G = gp[blockIdx.y];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= G.P) return;
  const double* src = parts + G.parts_off + p;
  double s = 0.0;
  for (int t = 0; t < G.n_parts; ++t) s += src[(size_t)t * G.P];
  const double v = 2.0 * s + *G.c_data;
  if (isinf(v)) atomicOr(status, kStatusDomain);
  out[G.p_off + p] = v;
}

}  // namespace

cudaError_t launch_group_reduce(const GroupPart* d_gparts, int n_groups, int max_P, const double* parts,
                                double* out, unsigned* status, cudaStream_t s) {
  if (n_groups < 1 || max_P < 1) return cudaSuccess;
  const int thr = 256;
  group_reduce_kernel<<<dim3((max_P + thr - 1) / thr, n_groups), thr, 0, s>>>(d_gparts, parts, out, status);
  return srw::launch_result();
}

}  // namespace srw

using srw::GroupPart;
using srw::TcGroup;

struct srw_group_plan {
  bool built = false;
  int candidate = 1;
  int bn_max = 256;
  std::vector<int> bn;
  int n_items = 0, n_slots = 0, n_cta = 0;
  size_t n_parts = 0;
  TcGroup* d_groups = nullptr;
  CUtensorMap* d_maps = nullptr;
  int4* d_items = nullptr;  // grid-stride slots
  GroupPart* d_gparts = nullptr;
};

struct srw_group_ctx {
  int device = 0, sm_count = 0, n = 0;
  std::vector<srw_handle> hs;
  std::vector<int> P, p_off;
  int P_total = 0, P_max = 0;
  std::vector<unsigned long long> versions;
  bool tensor_ok = true;
  srw_group_plan plan[3];           // SRW_BF16, SRW_BF16X3, SRW_FP16X3
  std::vector<int> tuned_bn[3];     // candidate 3: tile width per configuration chosen by measurement
  GroupPart* d_simt_gparts = nullptr;  // SRW_FP32
  size_t simt_parts = 0;
  double* d_parts = nullptr;
  size_t parts_cap = 0;
  float4* d_coef = nullptr;         // [points][2] W-producer coefficients and FP16 scales
  float* d_theta = nullptr;         // staging for host calls
  double* d_out = nullptr;
  unsigned* d_status = nullptr;
  cudaStream_t own_stream = nullptr;
  int profile = 0;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  std::string err;
};

namespace {

using srw::item_cost;
using srw::kBK;
using srw::kBM;

srw_status gfail(srw_group g, srw_status s, const std::string& msg) {
  if (g) g->err = msg;
  return s;
}

srw_status gcuda(srw_group g, cudaError_t e, const char* what) {
  return gfail(g, e == cudaErrorMemoryAllocation ? SRW_ENOMEM : SRW_ECUDA,
               std::string(what) + ": " + cudaGetErrorString(e));
}

#define G_CUDA(g, call, what)                           \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return gcuda(g, e_, what);   \
  } while (0)

template <class T>
void gfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void free_plan(srw_group_plan& pl) {
  gfree(pl.d_groups);
  gfree(pl.d_maps);
  gfree(pl.d_items);
  gfree(pl.d_gparts);
  pl.built = false;
}

void invalidate(srw_group g) {
  for (auto& pl : g->plan) free_plan(pl);
  gfree(g->d_simt_gparts);
  g->simt_parts = 0;
}

// Data and reference changes of a member handle change its descriptor.
void refresh_if_changed(srw_group g) {
  bool changed = false;
  for (int i = 0; i < g->n; ++i)
    if (g->hs[i]->version != g->versions[i]) changed = true;
  if (!changed) return;
  invalidate(g);
  for (int i = 0; i < g->n; ++i) g->versions[i] = g->hs[i]->version;
}

srw_status ensure_parts(srw_group g, size_t n) {
  if (n <= g->parts_cap && g->d_parts) return SRW_OK;
  gfree(g->d_parts);
  g->parts_cap = 0;  // a growth that fails leaves no buffer: the next call allocates again
  G_CUDA(g, srw::dev_malloc(&g->d_parts, sizeof(double) * n), "grouped partial sums");
  g->parts_cap = n;
  return SRW_OK;
}

// Tile widths of one candidate schedule.
// Cost of all rec tiles of handle h at width bn: each tile runs only its
// K-block range.
double tiles_cost(const srw_ctx* h, int bn, bool f16) {
  const std::vector<int2>& r = h->kbr_h[f16 ? 1 : 0][bn == 256 ? 1 : 0];
  double c = 0.0;
  for (const int2& t : r) c += item_cost(t.y - t.x, bn);
  return c;
}

void candidate_widths(srw_group g, int cand, int pi, bool f16, int* bn_max, std::vector<int>& bn) {
  bn.assign(g->n, 256);
  *bn_max = 256;
  if (cand == 3 && (int)g->tuned_bn[pi].size() == g->n) {
    bn = g->tuned_bn[pi];
    *bn_max = *std::max_element(bn.begin(), bn.end());
    return;
  }
  if (cand == 3) cand = 1;  // not tuned yet: the cost model's widths
  if (cand == 2) {
    bn.assign(g->n, 128);
    *bn_max = 128;
    return;
  }
  if (cand == 1) {
    for (int i = 0; i < g->n; ++i) {
      bn[i] = tiles_cost(g->hs[i], 128, f16) < tiles_cost(g->hs[i], 256, f16) ? 128 : 256;
    }
  }
}

srw_status build_plan(srw_group g, int pi, int cand) {
  srw_group_plan& pl = g->plan[pi];
  free_plan(pl);
  pl.candidate = cand;
  const bool f16 = pi + 1 == SRW_FP16X3;
  candidate_widths(g, cand, pi, f16, &pl.bn_max, pl.bn);

  struct Item {
    double cost;
    int g, m0, n0;
  };
  std::vector<Item> all;
  std::vector<TcGroup> desc(g->n);
  std::vector<GroupPart> gparts(g->n);
  std::vector<CUtensorMap> maps(2 * (size_t)g->n);
  long long parts_off = 0;
  for (int i = 0; i < g->n; ++i) {
    const srw_ctx* h = g->hs[i];
    const int bn = pl.bn[i];
    TcGroup G = srw::tc_group_of(h, bn, f16);
    G.P = g->P[i];
    G.p_off = g->p_off[i];
    G.parts_off = parts_off;
    desc[i] = G;
    gparts[i] = GroupPart{parts_off, G.n_tiles, G.P, G.p_off, 0, h->d_cdata};
    parts_off += (long long)G.n_tiles * G.P;
    const cudaError_t e = srw::tc_encode_maps(h, bn, f16, &maps[2 * (size_t)i], &maps[2 * (size_t)i + 1]);
    if (e != cudaSuccess) return gcuda(g, e, "tensor maps");
    const std::vector<int2>& kr = h->kbr_h[f16 ? 1 : 0][bn == 256 ? 1 : 0];
    const int m_tiles = (G.P + kBM - 1) / kBM;
    for (int nt = 0; nt < G.n_tiles; ++nt) {
      const double cost = item_cost(kr[nt].y - kr[nt].x, bn);
      for (int mt = 0; mt < m_tiles; ++mt) all.push_back({cost, i, mt * kBM, nt * bn});
    }
  }
  // longest first; equal costs keep (configuration, rec tile, point tile) order
  std::stable_sort(all.begin(), all.end(), [](const Item& a, const Item& b) { return a.cost > b.cost; });
  const int n_cta = (int)std::min<size_t>((size_t)g->sm_count, all.size());
  std::vector<std::vector<int4>> per(n_cta);
  typedef std::pair<double, int> Load;
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
  for (int b = 0; b < n_cta; ++b) heap.push({0.0, b});
  for (const Item& it : all) {
    Load l = heap.top();
    heap.pop();
    per[l.second].push_back(make_int4(it.g, it.m0, it.n0, 0));
    heap.push({l.first + it.cost, l.second});
  }
  size_t kmax = 0;
  for (int b = 0; b < n_cta; ++b) kmax = std::max(kmax, per[b].size());
  kmax += 1;  // room for every list's stop item
  std::vector<int4> items(kmax * n_cta, make_int4(-1, 0, 0, 0));
  for (int b = 0; b < n_cta; ++b)
    for (size_t k = 0; k < per[b].size(); ++k) items[k * n_cta + b] = per[b][k];

  G_CUDA(g, srw::dev_malloc(&pl.d_maps, sizeof(CUtensorMap) * maps.size()), "alloc maps");
  for (int i = 0; i < g->n; ++i) {
    desc[i].map_hi = pl.d_maps + 2 * (size_t)i;
    desc[i].map_lo = pl.d_maps + 2 * (size_t)i + 1;
  }
  G_CUDA(g, srw::dev_malloc(&pl.d_groups, sizeof(TcGroup) * desc.size()), "alloc descriptors");
  G_CUDA(g, srw::dev_malloc(&pl.d_gparts, sizeof(GroupPart) * gparts.size()), "alloc descriptors");
  G_CUDA(g, srw::dev_malloc(&pl.d_items, sizeof(int4) * std::max<size_t>(1, items.size())), "alloc items");
  G_CUDA(g, cudaMemcpy(pl.d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice), "upload");
  G_CUDA(g, cudaMemcpy(pl.d_groups, desc.data(), sizeof(TcGroup) * desc.size(), cudaMemcpyHostToDevice), "upload");
  G_CUDA(g, cudaMemcpy(pl.d_gparts, gparts.data(), sizeof(GroupPart) * gparts.size(), cudaMemcpyHostToDevice),
         "upload");
  if (!items.empty())
    G_CUDA(g, cudaMemcpy(pl.d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice), "upload");
  pl.n_items = (int)all.size();
  pl.n_slots = (int)items.size();
  pl.n_cta = n_cta;
  pl.n_parts = (size_t)parts_off;
  pl.built = true;
  return SRW_OK;
}

srw_status build_simt(srw_group g) {
  std::vector<GroupPart> gp(g->n);
  long long off = 0;
  for (int i = 0; i < g->n; ++i) {
    const int np = srw::fold_simt_parts(g->hs[i]->n_rec);
    gp[i] = GroupPart{off, np, g->P[i], g->p_off[i], 0, g->hs[i]->d_cdata};
    off += (long long)np * g->P[i];
  }
  G_CUDA(g, srw::dev_malloc(&g->d_simt_gparts, sizeof(GroupPart) * gp.size()), "alloc descriptors");
  G_CUDA(g, cudaMemcpy(g->d_simt_gparts, gp.data(), sizeof(GroupPart) * gp.size(), cudaMemcpyHostToDevice), "upload");
  g->simt_parts = (size_t)off;
  return SRW_OK;
}

srw_status check_status(srw_group g, cudaStream_t s, bool* domain) {
  unsigned st = 0;
  G_CUDA(g, cudaMemcpyAsync(&st, g->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "status read");
  G_CUDA(g, cudaStreamSynchronize(s), "stream sync");
  if (st) G_CUDA(g, cudaMemsetAsync(g->d_status, 0, sizeof(unsigned), s), "status reset");
  if (st & srw::kStatusTimeout) return gfail(g, SRW_ETIMEOUT, "a bounded device wait expired; the fold aborted");
  if (domain) *domain = (st & srw::kStatusDomain) != 0;
  return SRW_OK;
}

// Launches the grouped evaluation of all points (device pointers).
srw_status run(srw_group g, const float* th, double* o, int precision, cudaStream_t s) {
  if (precision == SRW_FP32) {
    if (!g->d_simt_gparts) {
      srw_status st = build_simt(g);
      if (st != SRW_OK) return st;
    }
    srw_status st = ensure_parts(g, g->simt_parts);
    if (st != SRW_OK) return st;
    size_t off = 0;
    for (int i = 0; i < g->n; ++i) {
      if (g->P[i] == 0) continue;
      int np = 0;
      G_CUDA(g, srw::launch_fold_simt(g->hs[i], th + (size_t)g->p_off[i] * 5, g->P[i], g->d_parts + off, s, &np),
             "SIMT fold");
      off += (size_t)np * g->P[i];
    }
    G_CUDA(g, srw::launch_group_reduce(g->d_simt_gparts, g->n, g->P_max, g->d_parts, o, g->d_status, s), "reduce");
    return SRW_OK;
  }
  srw_group_plan& pl = g->plan[precision - 1];
  if (!pl.built) {
    srw_status st = build_plan(g, precision - 1, pl.candidate);
    if (st != SRW_OK) return st;
  }
  srw_status st = ensure_parts(g, pl.n_parts);
  if (st != SRW_OK) return st;
  G_CUDA(g, srw::launch_group_coef(pl.d_groups, g->n, g->P_max, th, precision == SRW_FP16X3, g->d_coef, s),
         "point coefficients");
  if (g->profile) G_CUDA(g, cudaEventRecord(g->ev[0], s), "event");
  G_CUDA(g, srw::launch_fold_tc_group(pl.bn_max, precision, pl.d_groups, pl.d_items, pl.n_slots, pl.n_cta, g->d_coef,
                                      g->d_parts, g->d_status, s),
         "grouped fold");
  if (g->profile) G_CUDA(g, cudaEventRecord(g->ev[1], s), "event");
  G_CUDA(g, srw::launch_group_reduce(pl.d_gparts, g->n, g->P_max, g->d_parts, o, g->d_status, s), "reduce");
  return SRW_OK;
}

srw_status check_precision(srw_group g, int precision) {
  if (precision < SRW_FP32 || precision > SRW_FP16X3) return gfail(g, SRW_EINVAL, "bad precision");
  if (precision != SRW_FP32 && !g->tensor_ok)
    return gfail(g, SRW_EUNSUPPORTED, "tensor-core fold unavailable on this device");
  return SRW_OK;
}

}  // namespace

extern "C" {

srw_status srw_group_create(const srw_handle* handles, int n, const int* P, srw_group* out) {
  if (!out) return SRW_EINVAL;
  *out = nullptr;
  if (!handles || !P || n < 1) return SRW_EINVAL;
  if (n > srw::tc_max_groups()) return SRW_EINVAL;
  long long total = 0;
  int pmax = 0;
  for (int i = 0; i < n; ++i) {
    if (!handles[i] || P[i] < 0 || !handles[i]->has_data) return SRW_EINVAL;
    if (handles[i]->device != handles[0]->device) return SRW_EINVAL;
    total += P[i];
    pmax = std::max(pmax, P[i]);
  }
  if (total < 1 || total > 0x7fffffffLL / 5) return SRW_EINVAL;
  srw_group g = new (std::nothrow) srw_group_ctx();
  if (!g) return SRW_ENOMEM;
  g->n = n;
  g->device = handles[0]->device;
  g->sm_count = handles[0]->sm_count;
  g->hs.assign(handles, handles + n);
  g->P.assign(P, P + n);
  g->p_off.resize(n);
  int off = 0;
  for (int i = 0; i < n; ++i) {
    g->p_off[i] = off;
    off += P[i];
    g->tensor_ok = g->tensor_ok && handles[i]->tensor_ok;
    g->versions.push_back(handles[i]->version);
  }
  g->P_total = (int)total;
  g->P_max = pmax;
  cudaError_t e = cudaSetDevice(g->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->own_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = srw::dev_malloc(&g->d_status, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(g->d_status, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = srw::dev_malloc(&g->d_theta, sizeof(float) * 5 * total);
  if (e == cudaSuccess) e = srw::dev_malloc(&g->d_coef, 2 * sizeof(float4) * total);
  if (e == cudaSuccess) e = srw::dev_malloc(&g->d_out, sizeof(double) * total);
  if (e != cudaSuccess) {
    srw_group_destroy(g);
    return e == cudaErrorMemoryAllocation ? SRW_ENOMEM : SRW_ECUDA;
  }
  *out = g;
  return SRW_OK;
}

srw_status srw_group_loglik(srw_group g, const float* theta, double* out, int where, srw_precision precision,
                            void* stream) {
  if (!g) return SRW_EINVAL;
  if (!theta || !out) return gfail(g, SRW_EINVAL, "theta/out is NULL");
  if (where != SRW_HOST && where != SRW_DEVICE) return gfail(g, SRW_EINVAL, "where must be SRW_HOST or SRW_DEVICE");
  srw_status st = check_precision(g, (int)precision);
  if (st != SRW_OK) return st;
  refresh_if_changed(g);
  cudaStream_t s = stream ? (cudaStream_t)stream : g->own_stream;
  const float* th = theta;
  double* o = out;
  if (where == SRW_HOST) {
    if (!srw::all_finite(theta, (size_t)g->P_total * 5)) return gfail(g, SRW_EINVAL, "theta must be finite");
    // a host-pointer call reports the device status of this call only
    G_CUDA(g, cudaMemsetAsync(g->d_status, 0, sizeof(unsigned), s), "status reset");
    G_CUDA(g, cudaMemcpyAsync(g->d_theta, theta, sizeof(float) * 5 * (size_t)g->P_total, cudaMemcpyHostToDevice, s),
           "theta upload");
    th = g->d_theta;
    o = g->d_out;
  }
  st = run(g, th, o, (int)precision, s);
  if (st != SRW_OK) return st;
  if (where == SRW_HOST) {
    G_CUDA(g, cudaMemcpyAsync(out, o, sizeof(double) * (size_t)g->P_total, cudaMemcpyDeviceToHost, s), "download");
    bool domain = false;
    st = check_status(g, s, &domain);
    if (st != SRW_OK) return st;
    if (domain) return gfail(g, SRW_EDOMAIN, "expected count <= 0 in a bin with data: value is +inf");
  } else if (!stream) {
    G_CUDA(g, cudaStreamSynchronize(s), "sync");
  }
  return SRW_OK;
}

srw_status srw_group_autotune(srw_group g, srw_precision precision, void* stream, int* chosen) {
  if (!g) return SRW_EINVAL;
  if (chosen) *chosen = 0;
  srw_status st = check_precision(g, (int)precision);
  if (st != SRW_OK) return st;
  if (precision == SRW_FP32) return SRW_OK;
  refresh_if_changed(g);
  cudaStream_t s = stream ? (cudaStream_t)stream : g->own_stream;
  // deterministic in-box points for timing
  std::vector<float> th((size_t)g->P_total * 5);
  for (size_t q = 0; q < th.size(); ++q)
    th[q] = (float)(0.3 * std::sin(0.7 * (double)q + 0.1)) + (q % 5 == 4 ? 1.5f : 0.f);
  G_CUDA(g, cudaMemcpyAsync(g->d_theta, th.data(), sizeof(float) * th.size(), cudaMemcpyHostToDevice, s), "upload");
  cudaEvent_t e0, e1;
  G_CUDA(g, cudaEventCreate(&e0), "event");
  G_CUDA(g, cudaEventCreate(&e1), "event");
  const int pi = (int)precision - 1;
  // time the plan built for candidate c (+inf if it fails or a wait timed out)
  auto time_plan = [&](int c) {
    if (build_plan(g, pi, c) != SRW_OK) return 1e30f;
    if (run(g, g->d_theta, g->d_out, (int)precision, s) != SRW_OK) return 1e30f;  // warm-up
    cudaEventRecord(e0, s);
    bool ok = true;
    for (int r = 0; r < 3 && ok; ++r) ok = run(g, g->d_theta, g->d_out, (int)precision, s) == SRW_OK;
    cudaEventRecord(e1, s);
    bool dom = false;
    if (!ok || check_status(g, s, &dom) != SRW_OK) return 1e30f;  // a timed-out schedule is never chosen
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
  };
  float best = 1e30f;
  int best_c = 1;
  for (int c = 0; c < 3; ++c) {
    const float ms = time_plan(c);
    if (ms < best) {
      best = ms;
      best_c = c;
    }
  }
  // candidate 3: from the best fixed schedule, flip the tile width of one
  // configuration at a time (the most expensive ones first, at most 16) and
  // keep each flip that shortens the launch by more than 1 %
  {
    int bn_max = 256;
    std::vector<int> bn;
    candidate_widths(g, best_c, pi, pi + 1 == SRW_FP16X3, &bn_max, bn);
    std::vector<std::pair<double, int>> order;
    for (int i = 0; i < g->n; ++i)
      if (g->P[i] > 0)
        order.push_back({tiles_cost(g->hs[i], bn[i], pi + 1 == SRW_FP16X3) * (double)g->P[i], i});
    std::sort(order.rbegin(), order.rend());
    if (order.size() > 16) order.resize(16);
    g->tuned_bn[pi] = bn;
    float cur = best;
    for (const auto& o : order) {
      const int i = o.second;
      g->tuned_bn[pi][i] = bn[i] == 256 ? 128 : 256;
      const float ms = time_plan(3);
      if (ms < 0.99f * cur) {
        cur = ms;
        bn[i] = g->tuned_bn[pi][i];
      } else {
        g->tuned_bn[pi][i] = bn[i];
      }
    }
    if (cur < best) {
      best = cur;
      best_c = 3;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  st = build_plan(g, pi, best_c);
  if (st != SRW_OK) return st;
  if (chosen) *chosen = best_c;
  return SRW_OK;
}

srw_status srw_group_set_schedule(srw_group g, srw_precision precision, int candidate) {
  if (!g) return SRW_EINVAL;
  if (precision != SRW_BF16 && precision != SRW_BF16X3 && precision != SRW_FP16X3)
    return gfail(g, SRW_EINVAL, "schedules exist for the tensor-core precisions only");
  if (candidate < 0 || candidate > 3) return gfail(g, SRW_EINVAL, "candidate must be 0, 1, 2 or 3");
  refresh_if_changed(g);
  return build_plan(g, (int)precision - 1, candidate);
}

srw_status srw_group_schedule(srw_group g, srw_precision precision, int* bn_max, int* bn, int* n_items, int* n_cta,
                              int* candidate) {
  if (!g) return SRW_EINVAL;
  if (precision != SRW_BF16 && precision != SRW_BF16X3 && precision != SRW_FP16X3)
    return gfail(g, SRW_EINVAL, "schedules exist for the tensor-core precisions only");
  refresh_if_changed(g);
  srw_group_plan& pl = g->plan[(int)precision - 1];
  if (!pl.built) {
    srw_status st = build_plan(g, (int)precision - 1, pl.candidate);
    if (st != SRW_OK) return st;
  }
  if (bn_max) *bn_max = pl.bn_max;
  if (bn)
    for (int i = 0; i < g->n; ++i) bn[i] = pl.bn[i];
  if (n_items) *n_items = pl.n_items;
  if (n_cta) *n_cta = pl.n_cta;
  if (candidate) *candidate = pl.candidate;
  return SRW_OK;
}

srw_status srw_group_profile(srw_group g, int enable) {
  if (!g) return SRW_EINVAL;
  if (enable && !g->ev[0]) {
    G_CUDA(g, cudaEventCreate(&g->ev[0]), "event create");
    G_CUDA(g, cudaEventCreate(&g->ev[1]), "event create");
  }
  g->profile = enable ? 1 : 0;
  return SRW_OK;
}

srw_status srw_group_profile_read(srw_group g, float* fold_ms) {
  if (!g || !fold_ms) return gfail(g, SRW_EINVAL, "NULL argument");
  if (!g->profile) return gfail(g, SRW_EINVAL, "profiling is not enabled");
  G_CUDA(g, cudaEventSynchronize(g->ev[1]), "event sync");
  G_CUDA(g, cudaEventElapsedTime(fold_ms, g->ev[0], g->ev[1]), "event elapsed");
  return SRW_OK;
}

const char* srw_group_last_error(srw_group g) { return g ? g->err.c_str() : "NULL group"; }

srw_status srw_group_destroy(srw_group g) {
  if (!g) return SRW_OK;
  cudaSetDevice(g->device);
  if (g->own_stream) cudaStreamSynchronize(g->own_stream);
  invalidate(g);
  gfree(g->d_parts);
  gfree(g->d_theta);
  gfree(g->d_coef);
  gfree(g->d_out);
  gfree(g->d_status);
  for (auto& ev : g->ev)
    if (ev) cudaEventDestroy(ev);
  if (g->own_stream) cudaStreamDestroy(g->own_stream);
  delete g;
  return SRW_OK;
}

}  // extern "C"
