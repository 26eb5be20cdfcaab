// C-ABI entry points of the srw library: validation, device tables, dispatch
// and the per-signature CUDA-graph cache.  See include/srw.h for the contract.

#include <algorithm>
#include <cmath>
#include <cstring>
#include <fstream>
#include <numeric>
#include <sstream>
#include <string>
#include <vector>

#include "srw_internal.h"

namespace srw {


static thread_local std::string g_create_err;

srw_status fail(srw_ctx* h, srw_status s, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_err = msg;
  return s;
}

srw_status cuda_fail(srw_ctx* h, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(h, e == cudaErrorMemoryAllocation ? SRW_ENOMEM : SRW_ECUDA, m);
}

ModelView model_view(const srw_ctx* h) {
  ModelView m;
  m.n_t = h->n_t;
  m.n_rec = h->n_rec;
  m.n_nodes = h->n_nodes;
  m.k_pad = h->k_pad;
  m.ld_r = h->ld_r;
  m.midpoint = h->midpoint;
  m.t_min = (float)h->t_min;
  m.t_min64 = h->t_min;
  m.node_a = h->d_node_a;
  m.node_w = h->d_node_w;
  m.node_c = h->d_node_c;
  m.node_wlo = h->d_node_wlo;
  m.node64 = h->d_node64;
  m.bin_count = h->d_bin_count;
  m.bin_f = h->d_bin_f;
  m.bin_l = h->d_bin_l;
  m.bin64 = h->d_bin64;
  m.ssm32 = h->d_ssm32;
  m.esm32 = h->d_esm32;
  m.R = h->d_R;
  return m;
}

DataView data_view(const srw_ctx* h) {
  DataView d;
  d.n_rec = h->n_rec;
  d.n64 = h->d_n64;
  d.b64 = h->d_b64;
  d.nbm = h->d_nbm;
  d.mask = h->d_mask;
  d.c_data = h->d_cdata;
  return d;
}

template <class T>
static cudaError_t dalloc(srw_ctx* h, T** p, size_t n) {
  cudaError_t e = dev_malloc((void**)p, sizeof(T) * std::max<size_t>(n, 1));
  if (e == cudaSuccess) h->device_bytes += sizeof(T) * std::max<size_t>(n, 1);
  return e;
}

template <class T>
static void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

static float int_bits_as_float(int v) {
  float f;
  std::memcpy(&f, &v, sizeof f);
  return f;
}

static void split_df(double x, float* hi, float* lo) {
  *hi = (float)x;
  *lo = (float)(x - (double)*hi);
}

// Monomials (batched folds) and coupling products (spectrum kernel) of the
// reference point, in FP64 split into hi + lo floats.  Without a reference
// point the monomials are those of the theta-independent term alone
// (c = 1 for the nu_mu spectrum, 0 otherwise): it is folded once in FP64 and
// the folds never carry it, so their constant-monomial coefficient is always
// exactly zero.  The spectrum kernel's coupling products are zero then.
static void set_reference_coefs(srw_ctx* h) {
  const double s = h->sin2w;
  const double* t = nullptr;
  double th[5];
  for (int k = 0; k < 5; ++k) th[k] = (double)h->theta_ref[k];
  t = th;
  const double gle = 0.5 + s + t[0], gre = s + t[1], glt = -0.5 + s + t[2], grt = s + t[3];
  const double glm = -0.5 + s, grm = s, mu2 = t[4] * t[4];
  const double c[kNB] = {gle * gle, gre * gre, -gle * gre, glt * glt, grt * grt, -glt * grt, 1.0, mu2};
  const double g[10] = {gle * gle, glm * glm, glt * glt, gre * gre, grm * grm, grt * grt,
                        gle * gre, glm * grm, glt * grt, h->kappa * mu2};
  for (int b = 0; b < kNB; ++b) {
    if (h->use_ref) split_df(c[b], &h->cref.hi[b], &h->cref.lo[b]);
    else {
      h->cref.hi[b] = b == 6 ? 1.f : 0.f;
      h->cref.lo[b] = 0.f;
    }
  }
  for (int k = 0; k < 10; ++k) {
    if (h->use_ref) split_df(g[k], &h->gref[0][k], &h->gref[1][k]);
    else h->gref[0][k] = h->gref[1][k] = 0.f;
  }
}

static bool finite_all(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

static void destroy_graphs(srw_ctx* h) {
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
}

static void release(srw_ctx* h) {
  destroy_graphs(h);
  tc_release(h);
  dfree(h->d_node_a); dfree(h->d_node_w); dfree(h->d_node_c); dfree(h->d_node_wlo); dfree(h->d_shat_lo); dfree(h->d_shat_k8); dfree(h->d_node64); dfree(h->d_bin_count); dfree(h->d_bin_f);
  dfree(h->d_bin_l); dfree(h->d_bin64); dfree(h->d_basis); dfree(h->d_ssm64); dfree(h->d_esm64);
  for (int f = 0; f < 2; ++f)
    for (int b = 0; b < 2; ++b) dfree(h->d_kbr[f][b]);
  dfree(h->d_ssm32); dfree(h->d_esm32); dfree(h->d_shat); dfree(h->d_R); dfree(h->d_rhi); dfree(h->d_rlo); dfree(h->d_rhi16); dfree(h->d_rlo16); dfree(h->d_rinv); dfree(h->d_coef); dfree(h->d_linM); dfree(h->d_lin); dfree(h->d_linp);
  dfree(h->d_n64); dfree(h->d_b64); dfree(h->d_muref64); dfree(h->d_bref64); dfree(h->d_nbm); dfree(h->d_nb2); dfree(h->d_nb4); dfree(h->d_mask); dfree(h->d_cdata);
  dfree(h->d_W); dfree(h->d_S); dfree(h->d_musig); dfree(h->d_mu); dfree(h->d_part); dfree(h->d_ticket);
  dfree(h->d_status); dfree(h->d_gv_seg); dfree(h->d_simt_kr); dfree(h->d_gv_segs); dfree(h->d_gv_rows); dfree(h->d_bpart); dfree(h->d_theta); dfree(h->d_out); dfree(h->d_theta0);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  h->own_stream = nullptr;
  for (auto& ev : h->ev_fold)
    if (ev) cudaEventDestroy(ev);
  h->ev_fold[0] = h->ev_fold[1] = nullptr;
}

#define SRW_CUDA(h, call, what)                      \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
  } while (0)

static cudaStream_t pick_stream(srw_ctx* h, void* stream) {
  return stream ? (cudaStream_t)stream : h->own_stream;
}

// Grows the staging buffers for host-pointer calls; invalidates graphs that
// referenced the old buffers.
static srw_status ensure_staging(srw_ctx* h, int P) {
  if (P <= h->stage_cap && h->d_theta && h->d_out) return SRW_OK;
  int cap = std::max(P, 2 * h->stage_cap);
  destroy_graphs(h);
  dfree(h->d_theta);
  dfree(h->d_out);
  h->stage_cap = 0;  // a growth that fails leaves no buffer: the next call allocates again
  SRW_CUDA(h, dev_malloc(&h->d_theta, sizeof(float) * 5 * (size_t)cap), "staging theta");
  SRW_CUDA(h, dev_malloc(&h->d_out, sizeof(double) * (size_t)cap), "staging out");
  h->stage_cap = cap;
  return SRW_OK;
}

// Per-point coefficient buffer of the tensor-core folds (two float4 a point).
static srw_status ensure_coef(srw_ctx* h, int P) {
  if (P <= h->coef_cap && h->d_coef) return SRW_OK;
  const int cap = std::max(P, 2 * h->coef_cap);
  destroy_graphs(h);
  dfree(h->d_coef);
  h->coef_cap = 0;
  SRW_CUDA(h, dev_malloc(&h->d_coef, 2 * sizeof(float4) * (size_t)cap), "point coefficients");
  h->coef_cap = cap;
  return SRW_OK;
}

static srw_status ensure_bparts(srw_ctx* h, size_t n) {
  if (n <= h->bpart_cap && h->d_bpart) return SRW_OK;
  size_t cap = std::max(n, 2 * h->bpart_cap);
  destroy_graphs(h);
  dfree(h->d_bpart);
  h->bpart_cap = 0;
  // the debug build keeps canary doubles after the buffer (checked by host-pointer calls)
  const size_t extra = kDebugChecks ? kCanaryDoubles : 0;
  SRW_CUDA(h, dev_malloc(&h->d_bpart, sizeof(double) * (cap + extra)), "batched partials");
  h->bpart_cap = cap;
  if (kDebugChecks) {
    std::vector<unsigned long long> c(kCanaryDoubles, kCanaryBits);
    SRW_CUDA(h, cudaMemcpy(h->d_bpart + cap, c.data(), sizeof(double) * kCanaryDoubles, cudaMemcpyHostToDevice),
             "canary");
  }
  return SRW_OK;
}

static srw_status check_status_word(srw_ctx* h, cudaStream_t s, bool* domain) {
  unsigned st = 0;
  unsigned long long canary[kCanaryDoubles];
  SRW_CUDA(h, cudaMemcpyAsync(&st, h->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "status read");
  if (kDebugChecks && h->d_bpart)
    SRW_CUDA(h, cudaMemcpyAsync(canary, h->d_bpart + h->bpart_cap, sizeof(canary), cudaMemcpyDeviceToHost, s),
             "canary read");
  SRW_CUDA(h, cudaStreamSynchronize(s), "stream sync");
  if (st) SRW_CUDA(h, cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), s), "status reset");
  if (st & kStatusCheck) return fail(h, SRW_ECHECK, "a debug bounds check failed in a kernel");
  if (kDebugChecks && h->d_bpart)
    for (int k = 0; k < kCanaryDoubles; ++k)
      if (canary[k] != kCanaryBits) return fail(h, SRW_ECHECK, "the canary after the batched partial sums was overwritten");
  if (st & kStatusTimeout) return fail(h, SRW_ETIMEOUT, "a bounded device wait expired; the fold aborted");
  if (domain) *domain = (st & kStatusDomain) != 0;
  return SRW_OK;
}

// Replays the cached graph for this call signature, capturing it first if needed.
template <class Body>
static srw_status run_graph(srw_ctx* h, int path, int precision, int P, const void* theta, void* out,
                            cudaStream_t s, Body body) {
  for (auto& g : h->graphs) {
    if (g.path == path && g.precision == precision && g.P == P && g.theta == theta && g.out == out &&
        g.stream == s && g.prof == h->profile) {
      SRW_CUDA(h, cudaGraphLaunch(g.exec, s), "graph launch");
      return SRW_OK;
    }
  }
  cudaGraph_t graph = nullptr;
  fault_take_timeout_fired();  // clear: only an injection inside this capture counts
  SRW_CUDA(h, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
  cudaError_t eb = body(s);
  cudaError_t ee = cudaStreamEndCapture(s, &graph);
  if (eb != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(h, eb, "kernel launch during capture");
  }
  if (ee != cudaSuccess) return cuda_fail(h, ee, "end capture");
  cudaGraphExec_t exec = nullptr;
  cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) return cuda_fail(h, ei, "graph instantiate");
  if (fault_take_timeout_fired()) {
    // a graph captured with an injected timeout runs once and is not cached
    // (its destruction is deferred by CUDA until the launch completes)
    const cudaError_t el = cudaGraphLaunch(exec, s);
    cudaGraphExecDestroy(exec);
    if (el != cudaSuccess) return cuda_fail(h, el, "graph launch");
    return SRW_OK;
  }
  if (h->graphs.size() >= 32) {
    cudaGraphExecDestroy(h->graphs.front().exec);
    h->graphs.erase(h->graphs.begin());
  }
  h->graphs.push_back(GraphEntry{path, precision, P, h->profile, theta, out, s, exec});
  SRW_CUDA(h, cudaGraphLaunch(exec, s), "graph launch");
  return SRW_OK;
}

// Node and bin tables of a set of sources (replaces any previous tables).
// Every "does node n reach bin i" decision is made here in FP64 and handed to
// the kernels as integers: k_n = number of bins that lie entirely below
// T_max(E_n) (integrated mode) or whose centre lies below it (midpoint mode).
// Bins i < k_n are complete, bin k_n is clipped at T_max (integrated mode; its
// integrals are precomputed in FP64 per node), bins above get nothing.  Nodes
// are sorted by T_max descending, so k_n does not increase with n and the
// nodes reaching bin i are the prefix k_n >= i.
static cudaError_t upload_tables(srw_ctx* h, const srw_binning* bin, const srw_source* sources, int n_sources,
                                 cudaStream_t s) {
  dfree(h->d_node_a); dfree(h->d_node_w); dfree(h->d_node_c); dfree(h->d_node_wlo); dfree(h->d_node64);
  dfree(h->d_bin_count); dfree(h->d_bin_f); dfree(h->d_bin_l); dfree(h->d_bin64);
  const int n_t = bin->n_t;
  const double t_min = h->t_min, f_tau = h->f_tau;
  int N = 0;
  for (int k = 0; k < n_sources; ++k) N += sources[k].n_nodes;
  h->n_nodes = N;
  // ---- nodes: flavour weights in FP64, sorted by T_max descending
  std::vector<double> E(N), w(N), pe(N), pm(N), pt(N), tmax(N);
  {
    int q = 0;
    for (int k = 0; k < n_sources; ++k)
      for (int n = 0; n < sources[k].n_nodes; ++n, ++q) {
        E[q] = sources[k].e[n];
        w[q] = sources[k].w[n];
        const double p = sources[k].pee[n];
        pe[q] = p;
        pm[q] = (1.0 - p) * (1.0 - f_tau);
        pt[q] = (1.0 - p) * f_tau;
        tmax[q] = 2.0 * E[q] * E[q] / (kMe + 2.0 * E[q]);
      }
  }
  std::vector<int> order(N);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return tmax[a] > tmax[b]; });
  std::vector<float4> node_a(N), node_w(N), node_c(N), node_wlo(N);
  std::vector<double> node64(5 * (size_t)N);
  for (int q = 0; q < N; ++q) {
    const int o = order[q];
    const double e = E[o];
    const double wq[4] = {w[o] * pe[o], w[o] * pm[o], w[o] * pt[o], w[o]};
    node_w[q] = make_float4((float)wq[0], (float)wq[1], (float)wq[2], (float)wq[3]);
    node_wlo[q] = make_float4((float)(wq[0] - (double)node_w[q].x), (float)(wq[1] - (double)node_w[q].y),
                              (float)(wq[2] - (double)node_w[q].z), (float)(wq[3] - (double)node_w[q].w));
    node64[q] = e;
    node64[(size_t)N + q] = w[o] * pe[o];
    node64[2 * (size_t)N + q] = w[o] * pm[o];
    node64[3 * (size_t)N + q] = w[o] * pt[o];
    node64[4 * (size_t)N + q] = w[o];
  }
  // ---- bins
  std::vector<float4> bin_f(n_t);
  std::vector<float> bin_l(n_t);
  std::vector<double> bin64(2 * (size_t)n_t);
  std::vector<double> edge_hi(n_t), edge_c(n_t);
  for (int i = 0; i < n_t; ++i) {
    const double lo = bin->t_edges[i], hi = bin->t_edges[i + 1];
    bin64[i] = lo;
    bin64[(size_t)n_t + i] = hi;
    edge_hi[i] = hi;
    edge_c[i] = 0.5 * (lo + hi);
    if (h->midpoint) {
      const double tc = 0.5 * (lo + hi);
      // bins whose centre is below the threshold carry zero width
      bin_f[i] = make_float4((float)tc, tc >= t_min ? (float)(hi - lo) : 0.f, 0.f, 0.f);
      bin_l[i] = 0.f;
    } else {
      const double a = std::max(lo, t_min);
      if (!(hi > a)) {
        bin_f[i] = make_float4(1.f, 1.f, 0.f, 0.f);  // below threshold: zero-width bin
        bin_l[i] = 0.f;
        continue;
      }
      bin_f[i] = make_float4((float)a, (float)hi, (float)(hi - a), (float)(0.5 * (hi - a) * (a + hi)));
      bin_l[i] = (float)std::log1p((hi - a) / a);
    }
  }
  std::vector<int> kn(N);
  for (int q = 0; q < N; ++q) {
    const double tm = tmax[order[q]], e = E[order[q]];
    const std::vector<double>& ref = h->midpoint ? edge_c : edge_hi;
    // number of bins with edge (hi or centre) below T_max: hi <= tm, centre < tm
    int k;
    if (h->midpoint)
      k = (int)(std::lower_bound(ref.begin(), ref.end(), tm) - ref.begin());
    else
      k = (int)(std::upper_bound(ref.begin(), ref.end(), tm) - ref.begin());
    kn[q] = k;
    node_a[q] = make_float4((float)e, (float)(1.0 / e), int_bits_as_float(k), (float)(kMe / (e * e)));
    node_c[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!h->midpoint && k < n_t) {
      const double a = std::max(bin->t_edges[k], t_min), b = tm;
      if (b > a) {
        const double d = b - a, u = 1.0 - a / e, v = 1.0 - b / e;
        node_c[q] = make_float4((float)d, (float)(0.5 * d * (a + b)), (float)(d * (u * u + u * v + v * v) / 3.0),
                                (float)(std::log1p(d / a) - d / e));
      }
    }
  }
  // nodes with k_n >= i reach bin i (complete or clipped): a prefix because k_n is non-increasing
  std::vector<int> bin_count(n_t + 1, 0);
  for (int q = 0; q < N; ++q) bin_count[std::min(kn[q], n_t)] += 1;
  for (int i = n_t - 1; i >= 0; --i) bin_count[i] += bin_count[i + 1];
  bin_count.resize(n_t);
  for (int i = 0; i < n_t; ++i)
    if (!h->midpoint && !(bin->t_edges[i + 1] > std::max(bin->t_edges[i], t_min))) bin_count[i] = 0;

  cudaError_t e;
#define TAB(call) \
  if ((e = (call)) != cudaSuccess) return e
  TAB(dalloc(h, &h->d_node_a, N));
  TAB(dalloc(h, &h->d_node_w, N));
  TAB(dalloc(h, &h->d_node_c, N));
  TAB(dalloc(h, &h->d_node_wlo, N));
  TAB(dalloc(h, &h->d_node64, 5 * (size_t)N));
  TAB(dalloc(h, &h->d_bin_count, n_t));
  TAB(dalloc(h, &h->d_bin_f, n_t));
  TAB(dalloc(h, &h->d_bin_l, n_t));
  TAB(dalloc(h, &h->d_bin64, 2 * (size_t)n_t));
  TAB(cudaMemcpyAsync(h->d_node_a, node_a.data(), sizeof(float4) * N, cudaMemcpyHostToDevice, s));
  TAB(cudaMemcpyAsync(h->d_node_w, node_w.data(), sizeof(float4) * N, cudaMemcpyHostToDevice, s));
  TAB(cudaMemcpyAsync(h->d_node_c, node_c.data(), sizeof(float4) * N, cudaMemcpyHostToDevice, s));
  TAB(cudaMemcpyAsync(h->d_node_wlo, node_wlo.data(), sizeof(float4) * N, cudaMemcpyHostToDevice, s));
  TAB(cudaMemcpyAsync(h->d_node64, node64.data(), sizeof(double) * node64.size(), cudaMemcpyHostToDevice, s));
  TAB(cudaMemcpyAsync(h->d_bin_count, bin_count.data(), sizeof(int) * n_t, cudaMemcpyHostToDevice, s));
  TAB(cudaMemcpyAsync(h->d_bin_f, bin_f.data(), sizeof(float4) * n_t, cudaMemcpyHostToDevice, s));
  TAB(cudaMemcpyAsync(h->d_bin_l, bin_l.data(), sizeof(float) * n_t, cudaMemcpyHostToDevice, s));
  TAB(cudaMemcpyAsync(h->d_bin64, bin64.data(), sizeof(double) * bin64.size(), cudaMemcpyHostToDevice, s));
#undef TAB
  return cudaStreamSynchronize(s);  // the host tables go out of scope
}

// Device arrays sized by the fold axis (h->n_t columns, padded to k_pad) and
// the reconstructed bins.
static cudaError_t alloc_axis(srw_ctx* h, cudaStream_t s) {
  const int n_t = h->n_t, n_rec = h->n_rec;
  h->k_pad = (n_t + 63) / 64 * 64;
  h->ld_r = h->k_pad;
  const size_t ld = h->ld_r;
  cudaError_t e;
#define AX(call) \
  if ((e = (call)) != cudaSuccess) return e
  AX(dalloc(h, &h->d_basis, (size_t)kNB * n_t));
  AX(dalloc(h, &h->d_ssm64, n_t));
  AX(dalloc(h, &h->d_esm64, n_t));
  AX(dalloc(h, &h->d_ssm32, n_t));
  AX(dalloc(h, &h->d_esm32, h->k_pad));
  AX(dalloc(h, &h->d_shat, (size_t)kNB * h->k_pad));
  AX(dalloc(h, &h->d_shat_lo, (size_t)kNB * h->k_pad));
  AX(dalloc(h, &h->d_R, (size_t)n_rec * ld));
  AX(dalloc(h, &h->d_W, h->k_pad));
  AX(dalloc(h, &h->d_S, n_t));
  AX(dalloc(h, &h->d_musig, n_rec));
  AX(dalloc(h, &h->d_muref64, n_rec));
  AX(dalloc(h, &h->d_mu, n_rec));
  h->part_cap = fold_point_grid(h);
  AX(dalloc(h, &h->d_part, h->part_cap));
  AX(dalloc(h, &h->d_ticket, 1));
  AX(dalloc(h, &h->d_status, 1));
  AX(dalloc(h, &h->d_theta0, 8));
  AX(cudaMemsetAsync(h->d_ticket, 0, sizeof(unsigned), s));
  AX(cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), s));
  AX(cudaMemsetAsync(h->d_theta0, 0, sizeof(float) * 8, s));
  AX(cudaMemsetAsync(h->d_W, 0, sizeof(float) * h->k_pad, s));
  AX(cudaMemsetAsync(h->d_esm32, 0, sizeof(float) * h->k_pad, s));
  AX(cudaMemsetAsync(h->d_ssm32, 0, sizeof(float) * n_t, s));
  AX(cudaMemsetAsync(h->d_R, 0, sizeof(float) * (size_t)n_rec * ld, s));
#undef AX
  return cudaSuccess;
}

// Joint response (eq. Rij) of every component on the concatenated axis:
// per-component FP64 coefficient spectra, the live-time-corrected histogram
// sums, the event numbers N_k, then R_cat, the concatenated coefficient
// spectra and the weights' baseline E = 1 (W_c = S_c(theta) / S_SM,c).
static srw_status build_joint(srw_ctx* h, const srw_binning* bin, const srw_source* sources, int n_src,
                              const srw_joint_response* jr, cudaStream_t s) {
  const int n_t = bin->n_t, n_rec = h->n_rec;
  cudaError_t e;
#define JC(call, what)                                        \
  do {                                                        \
    if ((e = (call)) != cudaSuccess) return cuda_fail(h, e, what); \
  } while (0)
  // ---- coefficient spectra of each component (G0, FP64)
  std::vector<double> basis_all((size_t)n_src * kNB * n_t);
  h->n_t = n_t;
  JC(dalloc(h, &h->d_basis, (size_t)kNB * n_t), "alloc basis");
  for (int k = 0; k < n_src; ++k) {
    JC(upload_tables(h, bin, &sources[k], 1, s), "node tables");
    JC(launch_basis_fp64(h, s), "basis kernel");
    JC(cudaMemcpyAsync(basis_all.data() + (size_t)k * kNB * n_t, h->d_basis, sizeof(double) * kNB * n_t,
                       cudaMemcpyDeviceToHost, s), "basis download");
    JC(cudaStreamSynchronize(s), "basis sync");
  }
  dfree(h->d_node_a); dfree(h->d_node_w); dfree(h->d_node_c); dfree(h->d_node_wlo); dfree(h->d_node64);
  dfree(h->d_bin_count); dfree(h->d_bin_f); dfree(h->d_bin_l); dfree(h->d_bin64); dfree(h->d_basis);
  int total_nodes = 0;
  for (int k = 0; k < n_src; ++k) total_nodes += sources[k].n_nodes;
  h->n_nodes = total_nodes;
  h->device_bytes = 0;  // every persistent array so far was temporary
  // SM spectra and their integrals F_k (FP64, host): c(SM) of the unshifted couplings
  const double s2 = h->sin2w, gle = 0.5 + s2, gre = s2, glt = -0.5 + s2, grt = s2;
  const double csm[kNB] = {gle * gle, gre * gre, -gle * gre, glt * glt, grt * grt, -glt * grt, 1.0, 0.0};
  std::vector<double> F(n_src, 0.0);
  for (int k = 0; k < n_src; ++k)
    for (int i = 0; i < n_t; ++i) {
      double v = 0.0;
      for (int b = 0; b < kNB; ++b) v += csm[b] * basis_all[((size_t)k * kNB + b) * n_t + i];
      F[k] += v;
    }

  // ---- histogram sums (FP64, device)
  const size_t cells = (size_t)n_rec * n_t;
  double *d_hist = nullptr, *d_mask = nullptr, *d_live = nullptr, *d_col = nullptr;
  int* d_cols = nullptr;
  auto free_tmp = [&]() {
    dfree(d_hist); dfree(d_mask); dfree(d_live); dfree(d_col); dfree(d_cols);
  };
  auto jfail = [&](cudaError_t ce, const char* what) {
    free_tmp();
    return cuda_fail(h, ce, what);
  };
#define JT(call, what)                               \
  do {                                               \
    if ((e = (call)) != cudaSuccess) return jfail(e, what); \
  } while (0)
  JT(dev_malloc(&d_hist, sizeof(double) * cells * n_src), "alloc histograms");
  JT(dev_malloc(&d_mask, sizeof(double) * (size_t)n_rec * n_src), "alloc masks");
  JT(dev_malloc(&d_live, sizeof(double) * n_rec), "alloc live time");
  JT(dev_malloc(&d_col, sizeof(double) * 2 * (size_t)n_t * n_src), "alloc column sums");
  std::vector<double> ones(std::max(n_rec, 1), 1.0), live(n_rec, 1.0);
  if (jr->live) std::copy(jr->live, jr->live + n_rec, live.begin());
  JT(cudaMemcpyAsync(d_live, live.data(), sizeof(double) * n_rec, cudaMemcpyHostToDevice, s), "upload live time");
  for (int k = 0; k < n_src; ++k) {
    const double* m = (jr->mask && jr->mask[k]) ? jr->mask[k] : ones.data();
    JT(cudaMemcpyAsync(d_hist + cells * k, jr->hist[k], sizeof(double) * cells, cudaMemcpyHostToDevice, s),
       "upload histogram");
    JT(cudaMemcpyAsync(d_mask + (size_t)n_rec * k, m, sizeof(double) * n_rec, cudaMemcpyHostToDevice, s),
       "upload mask");
    JT(launch_joint_colsums(d_hist + cells * k, d_mask + (size_t)n_rec * k, d_live, n_rec, n_t,
                            d_col + 2 * (size_t)n_t * k, d_col + 2 * (size_t)n_t * k + n_t, s),
       "histogram sums");
  }
  std::vector<double> col(2 * (size_t)n_t * n_src);
  JT(cudaMemcpyAsync(col.data(), d_col, sizeof(double) * col.size(), cudaMemcpyDeviceToHost, s), "download sums");
  JT(cudaStreamSynchronize(s), "sums sync");
  std::vector<double> Z(n_src, 0.0), Y(n_src, 0.0), N(n_src, 0.0), scale(n_src, 1.0);
  std::vector<std::vector<int>> cols(n_src);
  int K = 0;
  for (int k = 0; k < n_src; ++k) {
    const double* cz = col.data() + 2 * (size_t)n_t * k;
    const double* cy = cz + n_t;
    for (int i = 0; i < n_t; ++i) {
      Z[k] += cz[i];
      Y[k] += cy[i];
      if (cz[i] > 0.0) cols[k].push_back(i);
    }
    if (!(Z[k] > 0.0)) {
      free_tmp();
      return fail(h, SRW_EINVAL, "the histogram of component " + std::to_string(k) + " holds no events");
    }
    if (jr->scale) scale[k] = jr->scale[k];
    K += (int)cols[k].size();
  }
  if (K > 49152) {
    free_tmp();
    return fail(h, SRW_EINVAL, "the concatenated (component, true bin) axis exceeds 49152 columns");
  }
  // N_k: given, or lambda F_k with the SM signal sum_j M_j sum_k N_k sum_i R^(k)_ij = exposure
  double lambda = 0.0;
  if (jr->events) {
    for (int k = 0; k < n_src; ++k) N[k] = jr->events[k];
  } else {
    double per = 0.0;
    for (int k = 0; k < n_src; ++k) per += F[k] * scale[k] * Y[k] / Z[k];
    if (!(per > 0.0) || !std::isfinite(per)) {
      free_tmp();
      return fail(h, SRW_EINVAL, "the SM signal of the components folds to zero: cannot normalise the exposure");
    }
    lambda = h->exposure / per;
    for (int k = 0; k < n_src; ++k) N[k] = lambda * F[k];
  }
  h->lambda = lambda;

  // ---- the concatenated axis
  h->n_t = K;
  JT(alloc_axis(h, s), "alloc");
  std::vector<int> all_cols;
  all_cols.reserve(K);
  h->col_src.clear();
  h->col_bin.clear();
  for (int k = 0; k < n_src; ++k)
    for (int i : cols[k]) {
      all_cols.push_back(i);
      h->col_src.push_back(k);
      h->col_bin.push_back(i);
    }
  JT(dev_malloc(&d_cols, sizeof(int) * std::max(K, 1)), "alloc columns");
  JT(cudaMemcpyAsync(d_cols, all_cols.data(), sizeof(int) * K, cudaMemcpyHostToDevice, s), "upload columns");
  int col0 = 0;
  for (int k = 0; k < n_src; ++k) {
    const int nk = (int)cols[k].size();
    JT(launch_joint_gather(d_hist + cells * k, d_mask + (size_t)n_rec * k, d_live, n_rec, n_t, d_cols + col0, nk,
                           N[k] * scale[k] / Z[k], h->d_R, h->ld_r, col0, s),
       "joint response gather");
    col0 += nk;
  }
  std::vector<double> basis_cat((size_t)kNB * K), esm(K, 1.0);
  for (int c = 0; c < K; ++c) {
    const int k = h->col_src[c], i = h->col_bin[c];
    for (int b = 0; b < kNB; ++b) basis_cat[(size_t)b * K + c] = basis_all[((size_t)k * kNB + b) * n_t + i];
  }
  JT(cudaMemcpyAsync(h->d_basis, basis_cat.data(), sizeof(double) * basis_cat.size(), cudaMemcpyHostToDevice, s),
     "upload basis");
  JT(cudaMemcpyAsync(h->d_esm64, esm.data(), sizeof(double) * K, cudaMemcpyHostToDevice, s), "upload baseline");
  h->has_esm_input = 1;
  JT(launch_build_shat(h, s), "shat kernels");
  JT(cudaStreamSynchronize(s), "joint sync");
  free_tmp();
#undef JT
#undef JC
  return SRW_OK;
}

// Checks shared by srw_create and srw_create_joint.
static srw_status validate_model(const srw_binning* bin, const srw_source* sources, int n_sources,
                                 const srw_options* opt) {
  if (bin->n_t < 1 || bin->n_rec < 1 || !bin->t_edges)
    return fail(nullptr, SRW_EINVAL, "n_t and n_rec must be >= 1 and t_edges non-NULL");
  if (bin->n_t > 49152) return fail(nullptr, SRW_EINVAL, "n_t above the supported maximum 49152");
  if (n_sources < 1) return fail(nullptr, SRW_EINVAL, "need at least one source");
  const int n_t = bin->n_t;
  if (!finite_all(bin->t_edges, (size_t)n_t + 1) || bin->t_edges[0] < 0.0)
    return fail(nullptr, SRW_EINVAL, "t_edges must be finite and >= 0");
  for (int i = 0; i < n_t; ++i)
    if (!(bin->t_edges[i + 1] > bin->t_edges[i])) return fail(nullptr, SRW_EINVAL, "t_edges must ascend strictly");
  if (!std::isfinite(bin->t_min > 0.0 ? bin->t_min : 1e-3)) return fail(nullptr, SRW_EINVAL, "t_min must be finite");
  if (!(opt->exposure > 0.0) || !std::isfinite(opt->exposure))
    return fail(nullptr, SRW_EINVAL, "exposure must be finite and > 0");
  const double sin2w = opt->sin2w > 0.0 ? opt->sin2w : 0.23121;
  const double f_tau = opt->f_tau >= 0.0 ? opt->f_tau : 0.5;
  if (!(sin2w < 1.0) || !(f_tau <= 1.0)) return fail(nullptr, SRW_EINVAL, "sin2w must be < 1 and f_tau <= 1");
  long long n_nodes = 0;
  for (int k = 0; k < n_sources; ++k) {
    const srw_source& s = sources[k];
    if (s.n_nodes < 1 || !s.e || !s.w || !s.pee) return fail(nullptr, SRW_EINVAL, "source with no nodes or NULL arrays");
    for (int n = 0; n < s.n_nodes; ++n) {
      if (!(s.e[n] > 0.0) || !std::isfinite(s.e[n])) return fail(nullptr, SRW_EINVAL, "node energies must be > 0");
      if (!(s.w[n] >= 0.0) || !std::isfinite(s.w[n])) return fail(nullptr, SRW_EINVAL, "node weights must be >= 0");
      if (!(s.pee[n] >= 0.0 && s.pee[n] <= 1.0)) return fail(nullptr, SRW_EINVAL, "P_ee must lie in [0, 1]");
    }
    n_nodes += s.n_nodes;
  }
  if (n_nodes > (1 << 26)) return fail(nullptr, SRW_EINVAL, "too many nodes");
  return SRW_OK;
}

static srw_status validate_joint(const srw_binning* bin, int n_sources, const srw_joint_response* jr,
                                 const srw_options* opt) {
  if (!jr->hist) return fail(nullptr, SRW_EINVAL, "joint response without histograms");
  if (opt->e_true_sm) return fail(nullptr, SRW_EINVAL, "e_true_sm is not used with a joint response: pass NULL");
  const size_t cells = (size_t)bin->n_rec * bin->n_t;
  for (int k = 0; k < n_sources; ++k) {
    const double* hk = jr->hist[k];
    if (!hk) return fail(nullptr, SRW_EINVAL, "NULL histogram");
    for (size_t q = 0; q < cells; ++q)
      if (!(hk[q] >= 0.0) || !std::isfinite(hk[q])) return fail(nullptr, SRW_EINVAL, "histograms must be finite and >= 0");
    if (jr->mask && jr->mask[k])
      for (int j = 0; j < bin->n_rec; ++j)
        if (!(jr->mask[k][j] > 0.0) || !std::isfinite(jr->mask[k][j]))
          return fail(nullptr, SRW_EINVAL, "live-time corrections must be finite and > 0");
    if (jr->scale && (!(jr->scale[k] > 0.0) || !std::isfinite(jr->scale[k])))
      return fail(nullptr, SRW_EINVAL, "scale factors must be finite and > 0");
    if (jr->events && (!(jr->events[k] > 0.0) || !std::isfinite(jr->events[k])))
      return fail(nullptr, SRW_EINVAL, "event numbers must be finite and > 0");
  }
  if (jr->live)
    for (int j = 0; j < bin->n_rec; ++j)
      if (!(jr->live[j] >= 0.0) || !std::isfinite(jr->live[j]))
        return fail(nullptr, SRW_EINVAL, "live-time factors must be finite and >= 0");
  return SRW_OK;
}

// srw_create (R != NULL, conditional response) and srw_create_joint (jr != NULL).
static srw_status create_impl(const srw_binning* bin, const srw_source* sources, int n_sources, const float* R,
                              const srw_joint_response* jr, const srw_options* opt, srw_handle* out) {
  g_create_err.clear();
  if (!out) return fail(nullptr, SRW_EINVAL, "out handle pointer is NULL");
  *out = nullptr;
  if (!bin || !sources || (!R && !jr) || !opt) return fail(nullptr, SRW_EINVAL, "NULL binning/sources/response/options");
  srw_status vs = validate_model(bin, sources, n_sources, opt);
  if (vs != SRW_OK) return vs;
  const int n_t = bin->n_t, n_rec = bin->n_rec;
  if (R) {
    for (size_t q = 0; q < (size_t)n_rec * n_t; ++q)
      if (!(R[q] >= 0.f) || !std::isfinite(R[q])) return fail(nullptr, SRW_EINVAL, "R must be finite and >= 0");
    if (opt->e_true_sm) {
      if (!finite_all(opt->e_true_sm, n_t)) return fail(nullptr, SRW_EINVAL, "e_true_sm must be finite");
      for (int i = 0; i < n_t; ++i)
        if (opt->e_true_sm[i] < 0.0) return fail(nullptr, SRW_EINVAL, "e_true_sm must be >= 0");
    }
  } else if ((vs = validate_joint(bin, n_sources, jr, opt)) != SRW_OK) {
    return vs;
  }

  int dev = 0, ndev = 0;
  cudaError_t ce = cudaGetDeviceCount(&ndev);
  if (ce != cudaSuccess || ndev == 0) return fail(nullptr, SRW_ECUDA, "no CUDA device available");
  if ((ce = cudaGetDevice(&dev)) != cudaSuccess) return fail(nullptr, SRW_ECUDA, "cudaGetDevice failed");
  cudaDeviceProp prop;
  if ((ce = cudaGetDeviceProperties(&prop, dev)) != cudaSuccess) return fail(nullptr, SRW_ECUDA, "device properties");
  if (!(prop.major == 10 && prop.minor == 3))
    return fail(nullptr, SRW_EUNSUPPORTED, "libsrw is compiled for sm_103a (GB300); device is sm_" +
                                               std::to_string(prop.major) + std::to_string(prop.minor));

  srw_ctx* h = new (std::nothrow) srw_ctx();
  if (!h) return fail(nullptr, SRW_ENOMEM, "host allocation");
  h->device = dev;
  h->sm_count = prop.multiProcessorCount;
  h->cc_major = prop.major;
  h->cc_minor = prop.minor;
  h->n_t = n_t;
  h->n_rec = n_rec;
  h->midpoint = bin->midpoint ? 1 : 0;
  h->rec_pad = (n_rec + 255) / 256 * 256;
  h->t_min = bin->t_min > 0.0 ? bin->t_min : 1e-3;
  h->sin2w = opt->sin2w > 0.0 ? opt->sin2w : 0.23121;
  h->f_tau = opt->f_tau >= 0.0 ? opt->f_tau : 0.5;
  h->exposure = opt->exposure;
  h->joint = jr ? 1 : 0;
  h->has_esm_input = (!jr && opt->e_true_sm) ? 1 : 0;
  h->kappa = (kPi * kAlpha * kAlpha / (kMe * kMe)) / (2.0 * kGF * kGF * kMe / kPi) * kMuUnit * kMuUnit;

  auto bail = [&](srw_status st) {
    std::string msg = h->err;
    release(h);
    delete h;
    fail(nullptr, st, msg);
    return st;
  };
#define CREATE_CUDA(call, what)                       \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return bail(cuda_fail(h, e_, what)); \
  } while (0)

  CREATE_CUDA(cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking), "stream create");
  cudaStream_t s = h->own_stream;
  fold_point_init();

  if (!jr) {
    CREATE_CUDA(upload_tables(h, bin, sources, n_sources, s), "node tables");
    CREATE_CUDA(alloc_axis(h, s), "alloc");
    CREATE_CUDA(cudaMemcpy2DAsync(h->d_R, (size_t)h->ld_r * sizeof(float), R, (size_t)n_t * sizeof(float),
                                  (size_t)n_t * sizeof(float), n_rec, cudaMemcpyHostToDevice, s), "upload R");
    if (h->has_esm_input)
      CREATE_CUDA(cudaMemcpyAsync(h->d_esm64, opt->e_true_sm, sizeof(double) * n_t, cudaMemcpyHostToDevice, s), "upload");
    // ---- G0 coefficient spectra (FP64), S_SM, E_SM, shat; then S_SM of the FP32 kernel
    CREATE_CUDA(launch_basis_fp64(h, s), "basis kernel");
    CREATE_CUDA(launch_build_shat(h, s), "shat kernels");
    CREATE_CUDA(launch_spectrum_point(h, h->d_theta0, nullptr, nullptr, h->d_ssm32, s), "SM spectrum kernel");
  } else {
    srw_status st = build_joint(h, bin, sources, n_sources, jr, s);
    if (st != SRW_OK) return bail(st);
  }
  CREATE_CUDA(dalloc(h, &h->d_linM, (size_t)n_rec * kNB), "alloc rank-8 matrix");
  CREATE_CUDA(dalloc(h, &h->d_lin, 3 * (size_t)n_rec), "alloc rank-8 constants");
  CREATE_CUDA(dalloc(h, &h->d_linp, (size_t)n_rec), "alloc rank-8 constants");
  CREATE_CUDA(launch_linear_m(h, s), "rank-8 matrix");
  set_reference_coefs(h);  // reference point: the SM (theta = 0)
  CREATE_CUDA(launch_reference_fold(h, s), "reference fold");
  CREATE_CUDA(cudaStreamSynchronize(s), "create sync");
  if (!jr && !h->has_esm_input && !(h->lambda > 0.0))
    return bail(fail(h, SRW_EINVAL, "the SM spectrum folded through R is zero: cannot normalise the exposure"));

  // ---- R on the host once: the GEMV's nonzero bands, the folds' K-block ranges
  std::vector<float> Rh((size_t)n_rec * h->ld_r);
  CREATE_CUDA(cudaMemcpy(Rh.data(), h->d_R, sizeof(float) * Rh.size(), cudaMemcpyDeviceToHost), "read R");
  CREATE_CUDA(gemv_prepare(h, Rh), "GEMV bands");
  CREATE_CUDA(simt_prepare(h, Rh), "FP32 fold K ranges");
  // ---- tensor-core path: BF16 hi/lo split of R and TMA descriptors
  if (tc_supported(h)) {
    CREATE_CUDA(dalloc(h, &h->d_rhi, (size_t)h->rec_pad * h->k_pad), "alloc R hi");
    CREATE_CUDA(dalloc(h, &h->d_rlo, (size_t)h->rec_pad * h->k_pad), "alloc R lo");
    CREATE_CUDA(dalloc(h, &h->d_shat_k8, (size_t)kNB * h->k_pad), "alloc shat k-major");
    CREATE_CUDA(dalloc(h, &h->d_rhi16, (size_t)h->rec_pad * h->k_pad), "alloc R hi (FP16)");
    CREATE_CUDA(dalloc(h, &h->d_rlo16, (size_t)h->rec_pad * h->k_pad), "alloc R lo (FP16)");
    CREATE_CUDA(dalloc(h, &h->d_rinv, (size_t)h->n_rec), "alloc R row scales");
    {  // bound of the coefficient spectra for the FP16 scales of the weighted spectra
      std::vector<float> sh((size_t)kNB * h->k_pad);
      CREATE_CUDA(cudaMemcpy(sh.data(), h->d_shat, sizeof(float) * sh.size(), cudaMemcpyDeviceToHost), "read shat");
      for (int b = 0; b < kNB; ++b) {
        float m = 0.f;
        for (int k = 0; k < h->k_pad; ++k) m = std::max(m, std::fabs(sh[(size_t)b * h->k_pad + k]));
        h->wmax[b] = m;
      }
    }
    CREATE_CUDA(launch_split_r(h, s), "split R");
    CREATE_CUDA(tc_block_ranges(h, Rh, s), "K-block ranges");
    CREATE_CUDA(tc_prepare(h), "tensor map encode");
    h->tensor_ok = true;
  }
  h->cfg[0] = FoldConfig{0, 128, 16, 1, 0};
  h->cfg[1] = h->cfg[2] = h->cfg[3] = tc_config(0);
  *out = h;
  return SRW_OK;
#undef CREATE_CUDA
}

}  // namespace srw

using namespace srw;

extern "C" {

const char* srw_status_string(srw_status s) {
  switch (s) {
    case SRW_OK: return "ok";
    case SRW_EINVAL: return "invalid argument";
    case SRW_ENOMEM: return "out of memory";
    case SRW_ECUDA: return "CUDA error";
    case SRW_ENODATA: return "no data set";
    case SRW_EDOMAIN: return "expected count <= 0 where data > 0";
    case SRW_ETIMEOUT: return "device wait timed out";
    case SRW_EUNSUPPORTED: return "unsupported device";
    case SRW_ECHECK: return "debug bounds check failed";
  }
  return "unknown status";
}

const char* srw_last_error(srw_handle h) { return h ? h->err.c_str() : g_create_err.c_str(); }

srw_status srw_create(const srw_binning* bin, const srw_source* sources, int n_sources, const float* R,
                      const srw_options* opt, srw_handle* out) {
  if (!R) {
    g_create_err = "NULL R";
    if (out) *out = nullptr;
    return SRW_EINVAL;
  }
  return create_impl(bin, sources, n_sources, R, nullptr, opt, out);
}

srw_status srw_create_joint(const srw_binning* bin, const srw_source* sources, int n_sources,
                            const srw_joint_response* response, const srw_options* opt, srw_handle* out) {
  if (!response) {
    g_create_err = "NULL joint response";
    if (out) *out = nullptr;
    return SRW_EINVAL;
  }
  return create_impl(bin, sources, n_sources, nullptr, response, opt, out);
}

srw_status srw_joint_layout(srw_handle h, int* n_columns, int* source, int* bin) {
  if (!h) return fail(nullptr, SRW_EINVAL, "NULL handle");
  if (!n_columns) return fail(h, SRW_EINVAL, "n_columns is NULL");
  *n_columns = h->n_t;
  for (int c = 0; c < h->n_t; ++c) {
    if (source) source[c] = h->joint ? h->col_src[c] : 0;
    if (bin) bin[c] = h->joint ? h->col_bin[c] : c;
  }
  return SRW_OK;
}

srw_status srw_set_data(srw_handle h, const double* counts, const double* bkg, int n_bkg,
                        const unsigned char* mask) {
  if (!h) return fail(nullptr, SRW_EINVAL, "NULL handle");
  if (!counts) return fail(h, SRW_EINVAL, "counts is NULL");
  if (n_bkg < 0 || (n_bkg > 0 && !bkg)) return fail(h, SRW_EINVAL, "bad background arguments");
  const int n_rec = h->n_rec;
  for (int j = 0; j < n_rec; ++j)
    if (!(counts[j] >= 0.0) || !std::isfinite(counts[j])) return fail(h, SRW_EINVAL, "counts must be finite and >= 0");
  if (n_bkg > 0 && !finite_all(bkg, (size_t)n_bkg * n_rec)) return fail(h, SRW_EINVAL, "backgrounds must be finite");
  cudaStream_t s = h->own_stream;
  // each buffer once; after a call whose allocation failed part-way, the next
  // call allocates the ones still missing
  if (!h->d_n64) SRW_CUDA(h, dalloc(h, &h->d_n64, n_rec), "alloc data");
  if (!h->d_b64) SRW_CUDA(h, dalloc(h, &h->d_b64, n_rec), "alloc data");
  if (!h->d_nbm) SRW_CUDA(h, dalloc(h, &h->d_nbm, n_rec), "alloc data");
  if (!h->d_nb2) SRW_CUDA(h, dalloc(h, &h->d_nb2, n_rec), "alloc data");
  if (!h->d_nb4) SRW_CUDA(h, dalloc(h, &h->d_nb4, n_rec), "alloc data");
  if (!h->d_cdata) SRW_CUDA(h, dalloc(h, &h->d_cdata, 1), "alloc data");
  if (!h->d_bref64) SRW_CUDA(h, dalloc(h, &h->d_bref64, n_rec), "alloc data");
  if (mask && !h->d_mask) SRW_CUDA(h, dalloc(h, &h->d_mask, n_rec), "alloc mask");
  // from here on the data change: a failure leaves the handle without data
  // (SRW_ENODATA) rather than with a mix of the old and the new
  h->has_data = 0;
  if (!mask) dfree(h->d_mask);
  destroy_graphs(h);
  double* d_bkg = nullptr;
  SRW_CUDA(h, cudaMemcpyAsync(h->d_n64, counts, sizeof(double) * n_rec, cudaMemcpyHostToDevice, s), "upload counts");
  if (mask) SRW_CUDA(h, cudaMemcpyAsync(h->d_mask, mask, n_rec, cudaMemcpyHostToDevice, s), "upload mask");
  if (n_bkg > 0) {
    SRW_CUDA(h, dev_malloc_async(&d_bkg, sizeof(double) * (size_t)n_bkg * n_rec, s), "alloc bkg");
    SRW_CUDA(h, cudaMemcpyAsync(d_bkg, bkg, sizeof(double) * (size_t)n_bkg * n_rec, cudaMemcpyHostToDevice, s), "upload bkg");
  }
  SRW_CUDA(h, launch_set_data(h, d_bkg, n_bkg, s), "data kernels");
  if (d_bkg) SRW_CUDA(h, cudaFreeAsync(d_bkg, s), "free bkg");
  SRW_CUDA(h, cudaStreamSynchronize(s), "set_data sync");
  h->has_data = 1;
  ++h->version;
  return SRW_OK;
}

srw_status srw_spectrum(srw_handle h, const float* theta, int stage, float* out, int where, void* stream) {
  if (!h) return fail(nullptr, SRW_EINVAL, "NULL handle");
  if (!theta || !out) return fail(h, SRW_EINVAL, "theta/out is NULL");
  if (stage < 0 || stage > 3) return fail(h, SRW_EINVAL, "stage must be 0..3");
  if (where != SRW_HOST && where != SRW_DEVICE) return fail(h, SRW_EINVAL, "where must be SRW_HOST or SRW_DEVICE");
  if (stage == 3 && !h->has_data) return fail(h, SRW_ENODATA, "stage 3 needs srw_set_data");
  cudaStream_t s = pick_stream(h, stream);
  const float* th = theta;
  if (where == SRW_HOST) {
    for (int k = 0; k < 5; ++k)
      if (!std::isfinite(theta[k])) return fail(h, SRW_EINVAL, "theta must be finite");
    srw_status st = ensure_staging(h, 1);
    if (st != SRW_OK) return st;
    SRW_CUDA(h, cudaMemcpyAsync(h->d_theta, theta, sizeof(float) * 5, cudaMemcpyHostToDevice, s), "theta upload");
    th = h->d_theta;
  }
  const bool dev = where == SRW_DEVICE;
  const int n_out = stage <= 1 ? h->n_t : h->n_rec;
  float* dst = dev ? out : (stage == 0 ? h->d_S : stage == 1 ? h->d_W : stage == 2 ? h->d_musig : h->d_mu);
  if (h->joint) {
    // per-component spectra / weights on the concatenated axis from the FP64
    // coefficient spectra; the fold of the weights' deviation from the reference
    if (stage <= 1) {
      SRW_CUDA(h, launch_basis_eval(h, th, stage, dst, s), "spectrum kernel");
    } else {
      SRW_CUDA(h, launch_weights_from_basis(h, th, h->d_W, s), "weights kernel");
      SRW_CUDA(h, launch_fold_point(h, h->d_W, stage == 2 ? dst : nullptr, stage == 3 ? dst : nullptr, nullptr, s, true),
               "fold kernel");
    }
  } else if (stage == 0) {
    SRW_CUDA(h, launch_spectrum_point(h, th, dst, nullptr, nullptr, s), "spectrum kernel");
  } else {
    // stage 1 returns the full W; stages 2 and 3 fold the deviation from the reference point
    float* Wbuf = (stage == 1 && dev) ? out : h->d_W;
    SRW_CUDA(h, launch_spectrum_point(h, th, nullptr, Wbuf, nullptr, s, stage >= 2), "spectrum kernel");
    // the spectrum kernel forms a deviation only with a reference point set
    if (stage == 2) SRW_CUDA(h, launch_fold_point(h, h->d_W, dst, nullptr, nullptr, s, h->use_ref != 0), "fold kernel");
    if (stage == 3) SRW_CUDA(h, launch_fold_point(h, h->d_W, nullptr, dst, nullptr, s, h->use_ref != 0), "fold kernel");
  }
  if (!dev) {
    SRW_CUDA(h, cudaMemcpyAsync(out, dst, sizeof(float) * n_out, cudaMemcpyDeviceToHost, s), "download");
    SRW_CUDA(h, cudaStreamSynchronize(s), "sync");
  } else if (!stream) {
    SRW_CUDA(h, cudaStreamSynchronize(s), "sync");
  }
  return SRW_OK;
}

static srw_status loglik_impl(srw_handle h, const float* theta, int P, double* out, int where, int precision,
                              void* stream, bool points_only) {
  if (!h) return fail(nullptr, SRW_EINVAL, "NULL handle");
  if (!theta || !out) return fail(h, SRW_EINVAL, "theta/out is NULL");
  if (P < 1) return fail(h, SRW_EINVAL, "P must be >= 1");
  if (precision < SRW_FP32 || precision > SRW_FP16X3) return fail(h, SRW_EINVAL, "bad precision");
  if (!h->has_data) return fail(h, SRW_ENODATA, "call srw_set_data first");
  if (where != SRW_HOST && where != SRW_DEVICE) return fail(h, SRW_EINVAL, "where must be SRW_HOST or SRW_DEVICE");
  if (precision != SRW_FP32 && !h->tensor_ok)
    return fail(h, SRW_EUNSUPPORTED, "tensor-core fold unavailable on this device");
  cudaStream_t s = pick_stream(h, stream);
  const float* th = theta;
  double* o = out;
  if (where == SRW_HOST) {
    // theta is checked for finiteness on the host while the device works (see
    // below); every kernel takes it only in arithmetic, so a non-finite value
    // does no harm before the call fails
    srw_status st = ensure_staging(h, P);
    if (st != SRW_OK) return st;
    // a host-pointer call reports the device status of this call only
    SRW_CUDA(h, cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), s), "status reset");
    SRW_CUDA(h, cudaMemcpyAsync(h->d_theta, theta, sizeof(float) * 5 * (size_t)P, cudaMemcpyHostToDevice, s),
             "theta upload");
    th = h->d_theta;
    o = h->d_out;
  }

  srw_status st = SRW_OK;
  if (points_only) {
    st = run_graph(h, 3, precision, P, th, o, s, [&](cudaStream_t cs) {
      for (int p = 0; p < P; ++p) {
        cudaError_t e = h->joint ? launch_weights_from_basis(h, th + 5 * (size_t)p, h->d_W, cs)
                                 : launch_spectrum_point(h, th + 5 * (size_t)p, nullptr, h->d_W, nullptr, cs, true);
        if (e != cudaSuccess) return e;
        if ((e = launch_fold_point(h, h->d_W, nullptr, nullptr, o + p, cs, h->joint || h->use_ref)) != cudaSuccess)
          return e;
      }
      return cudaSuccess;
    });
  } else if (h->profile) {
    // profiling: direct launches (no graph), with events around the fold
    // kernel alone, so that srw_profile_read gives that kernel's device time
    if (P == 1 && precision == SRW_FP32) {
      cudaError_t e = launch_weights_from_basis(h, th, h->d_W, s);
      if (e == cudaSuccess) e = cudaEventRecord(h->ev_fold[0], s);
      if (e == cudaSuccess) e = launch_fold_point(h, h->d_W, nullptr, nullptr, o, s, true);
      if (e == cudaSuccess) e = cudaEventRecord(h->ev_fold[1], s);
      if (e != cudaSuccess) return cuda_fail(h, e, "profiled single-point fold");
    } else {
      const int n_parts_max = precision == SRW_FP32 ? fold_simt_parts(h->n_rec) : (h->rec_pad / 128);
      st = ensure_bparts(h, (size_t)n_parts_max * P);
      if (st == SRW_OK && precision != SRW_FP32) st = ensure_coef(h, P);
      if (st != SRW_OK) return st;
      int n_parts = 0;
      cudaError_t e = cudaSuccess;
      if (precision == SRW_FP32) {
        e = cudaEventRecord(h->ev_fold[0], s);
        if (e == cudaSuccess) e = launch_fold_simt(h, th, P, h->d_bpart, s, &n_parts);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_fold[1], s);
      } else {
        e = launch_fold_tc(h, th, P, precision, h->cfg[precision], h->d_bpart, s, &n_parts, nullptr, h->ev_fold[0],
                           h->ev_fold[1]);
      }
      if (e == cudaSuccess) e = launch_reduce_parts(h, h->d_bpart, n_parts, P, o, s);
      if (e != cudaSuccess) return cuda_fail(h, e, "profiled batched fold");
    }
  } else if (P == 1 && precision == SRW_FP32) {
    st = run_graph(h, 1, precision, P, th, o, s, [&](cudaStream_t cs) {
      // W(theta) - W_ref from the coefficient spectra, then the HBM-streaming
      // fold, launched as a programmatic dependent: it streams R while the
      // weights kernel runs
      cudaError_t e = launch_weights_from_basis(h, th, h->d_W, cs);
      if (e != cudaSuccess) return e;
      return launch_fold_point_after(h, h->d_W, o, cs);
    });
  } else {
    const int n_parts_max = precision == SRW_FP32 ? fold_simt_parts(h->n_rec) : (h->rec_pad / 128);
    st = ensure_bparts(h, (size_t)n_parts_max * P);
    if (st == SRW_OK && precision != SRW_FP32) st = ensure_coef(h, P);
    if (st != SRW_OK) return st;
    const FoldConfig cfg = h->cfg[precision];
    st = run_graph(h, 2, precision, P, th, o, s, [&](cudaStream_t cs) {
      int n_parts = 0;
      cudaError_t e = precision == SRW_FP32 ? launch_fold_simt(h, th, P, h->d_bpart, cs, &n_parts)
                                            : launch_fold_tc(h, th, P, precision, cfg, h->d_bpart, cs, &n_parts);
      if (e != cudaSuccess) return e;
      return launch_reduce_parts(h, h->d_bpart, n_parts, P, o, cs);
    });
  }
  if (st != SRW_OK) return st;
  if (where == SRW_HOST) {
    // a non-finite theta fails the call before anything is written to out
    if (!all_finite(theta, (size_t)P * 5)) {
      SRW_CUDA(h, cudaStreamSynchronize(s), "sync");
      return fail(h, SRW_EINVAL, "theta must be finite");
    }
    SRW_CUDA(h, cudaMemcpyAsync(out, o, sizeof(double) * (size_t)P, cudaMemcpyDeviceToHost, s), "download");
    bool domain = false;
    st = check_status_word(h, s, &domain);
    if (st != SRW_OK) return st;
    if (domain) return fail(h, SRW_EDOMAIN, "expected count <= 0 in a bin with data: value is +inf");
  } else if (!stream) {
    SRW_CUDA(h, cudaStreamSynchronize(s), "sync");
  }
  return SRW_OK;
}

srw_status srw_loglik(srw_handle h, const float* theta, int P, double* out, int where, srw_precision precision,
                      void* stream) {
  return loglik_impl(h, theta, P, out, where, (int)precision, stream, false);
}

srw_status srw_loglik_points(srw_handle h, const float* theta, int P, double* out, int where, void* stream) {
  return loglik_impl(h, theta, P, out, where, SRW_FP32, stream, true);
}

srw_status srw_loglik_linear(srw_handle h, const float* theta, int P, double* out, double* grad, int where,
                             void* stream) {
  if (!h) return fail(nullptr, SRW_EINVAL, "NULL handle");
  if (!theta || !out) return fail(h, SRW_EINVAL, "theta/out is NULL");
  if (P < 1) return fail(h, SRW_EINVAL, "P must be >= 1");
  if (!h->has_data) return fail(h, SRW_ENODATA, "call srw_set_data first");
  if (where != SRW_HOST && where != SRW_DEVICE) return fail(h, SRW_EINVAL, "where must be SRW_HOST or SRW_DEVICE");
  cudaStream_t s = pick_stream(h, stream);
  const float* th = theta;
  double *o = out, *g = grad, *d_g = nullptr;
  if (where == SRW_HOST) {
    if (!all_finite(theta, (size_t)P * 5)) return fail(h, SRW_EINVAL, "theta must be finite");
    srw_status st = ensure_staging(h, P);
    if (st != SRW_OK) return st;
    // a host-pointer call reports the device status of this call only
    SRW_CUDA(h, cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), s), "status reset");
    SRW_CUDA(h, cudaMemcpyAsync(h->d_theta, theta, sizeof(float) * 5 * (size_t)P, cudaMemcpyHostToDevice, s),
             "theta upload");
    th = h->d_theta;
    o = h->d_out;
    if (grad) {
      SRW_CUDA(h, dev_malloc_async(&d_g, sizeof(double) * 5 * (size_t)P, s), "alloc gradient");
      g = d_g;
    }
  }
  cudaError_t e = launch_linear_loglik(h, th, P, o, g, s);
  if (e != cudaSuccess) {
    if (d_g) cudaFreeAsync(d_g, s);
    return cuda_fail(h, e, "rank-8 evaluation");
  }
  if (where == SRW_HOST) {
    SRW_CUDA(h, cudaMemcpyAsync(out, o, sizeof(double) * (size_t)P, cudaMemcpyDeviceToHost, s), "download");
    if (grad) {
      SRW_CUDA(h, cudaMemcpyAsync(grad, d_g, sizeof(double) * 5 * (size_t)P, cudaMemcpyDeviceToHost, s), "download");
      SRW_CUDA(h, cudaFreeAsync(d_g, s), "free gradient");
    }
    bool domain = false;
    srw_status st = check_status_word(h, s, &domain);
    if (st != SRW_OK) return st;
    if (domain) return fail(h, SRW_EDOMAIN, "expected count <= 0 in a bin with data: value is +inf");
  } else if (!stream) {
    SRW_CUDA(h, cudaStreamSynchronize(s), "sync");
  }
  return SRW_OK;
}

srw_status srw_loglik_profiled(srw_handle h, const float* theta, int P, double sigma_alpha, double* out,
                               double* alpha, int where, void* stream) {
  if (!h) return fail(nullptr, SRW_EINVAL, "NULL handle");
  if (!theta || !out) return fail(h, SRW_EINVAL, "theta/out is NULL");
  if (P < 1) return fail(h, SRW_EINVAL, "P must be >= 1");
  if (!(sigma_alpha >= 0.0) || !std::isfinite(sigma_alpha)) return fail(h, SRW_EINVAL, "sigma_alpha must be >= 0");
  if (!h->has_data) return fail(h, SRW_ENODATA, "call srw_set_data first");
  if (where != SRW_HOST && where != SRW_DEVICE) return fail(h, SRW_EINVAL, "where must be SRW_HOST or SRW_DEVICE");
  cudaStream_t s = pick_stream(h, stream);
  const float* th = theta;
  double *o = out, *a = alpha, *d_a = nullptr;
  if (where == SRW_HOST) {
    if (!all_finite(theta, (size_t)P * 5)) return fail(h, SRW_EINVAL, "theta must be finite");
    srw_status st = ensure_staging(h, P);
    if (st != SRW_OK) return st;
    // a host-pointer call reports the device status of this call only
    SRW_CUDA(h, cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), s), "status reset");
    SRW_CUDA(h, cudaMemcpyAsync(h->d_theta, theta, sizeof(float) * 5 * (size_t)P, cudaMemcpyHostToDevice, s),
             "theta upload");
    th = h->d_theta;
    o = h->d_out;
    if (alpha) {
      SRW_CUDA(h, dev_malloc_async(&d_a, sizeof(double) * (size_t)P, s), "alloc alpha");
      a = d_a;
    }
  }
  cudaError_t e = launch_linear_profiled(h, th, P, sigma_alpha, o, a, s);
  if (e != cudaSuccess) {
    if (d_a) cudaFreeAsync(d_a, s);
    return cuda_fail(h, e, "profiled evaluation");
  }
  if (where == SRW_HOST) {
    SRW_CUDA(h, cudaMemcpyAsync(out, o, sizeof(double) * (size_t)P, cudaMemcpyDeviceToHost, s), "download");
    if (alpha) {
      SRW_CUDA(h, cudaMemcpyAsync(alpha, d_a, sizeof(double) * (size_t)P, cudaMemcpyDeviceToHost, s), "download");
      SRW_CUDA(h, cudaFreeAsync(d_a, s), "free alpha");
    }
    bool domain = false;
    srw_status st = check_status_word(h, s, &domain);
    if (st != SRW_OK) return st;
    if (domain) return fail(h, SRW_EDOMAIN, "expected count <= 0 in a bin with data: value is +inf");
  } else if (!stream) {
    SRW_CUDA(h, cudaStreamSynchronize(s), "sync");
  }
  return SRW_OK;
}

srw_status srw_spectrum_batch(srw_handle h, const float* theta, int P, float* out, int where, srw_precision precision,
                              void* stream) {
  if (!h) return fail(nullptr, SRW_EINVAL, "NULL handle");
  if (!theta || !out) return fail(h, SRW_EINVAL, "theta/out is NULL");
  if (P < 1) return fail(h, SRW_EINVAL, "P must be >= 1");
  if (precision < SRW_FP32 || precision > SRW_FP16X3) return fail(h, SRW_EINVAL, "bad precision");
  if (where != SRW_HOST && where != SRW_DEVICE) return fail(h, SRW_EINVAL, "where must be SRW_HOST or SRW_DEVICE");
  if (precision != SRW_FP32 && !h->tensor_ok)
    return fail(h, SRW_EUNSUPPORTED, "tensor-core fold unavailable on this device");
  cudaStream_t s = pick_stream(h, stream);
  const float* th = theta;
  float* o = out;
  float* d_tmp = nullptr;
  if (precision != SRW_FP32) {
    srw_status st = ensure_coef(h, P);
    if (st != SRW_OK) return st;
  }
  if (where == SRW_HOST) {
    if (!all_finite(theta, (size_t)P * 5)) return fail(h, SRW_EINVAL, "theta must be finite");
    srw_status st = ensure_staging(h, P);
    if (st != SRW_OK) return st;
    // a host-pointer call reports the device status of this call only
    SRW_CUDA(h, cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), s), "status reset");
    SRW_CUDA(h, cudaMemcpyAsync(h->d_theta, theta, sizeof(float) * 5 * (size_t)P, cudaMemcpyHostToDevice, s),
             "theta upload");
    th = h->d_theta;
    SRW_CUDA(h, dev_malloc_async(&d_tmp, sizeof(float) * (size_t)P * h->n_rec, s), "alloc spectra");
    o = d_tmp;
  }
  int n_parts = 0;
  cudaError_t e = precision == SRW_FP32
                      ? launch_fold_simt(h, th, P, nullptr, s, &n_parts, o)
                      : launch_fold_tc(h, th, P, (int)precision, h->cfg[precision], nullptr, s, &n_parts, o);
  if (e == cudaSuccess) e = launch_add_ref(h, o, P, s);
  if (e != cudaSuccess) {
    if (d_tmp) cudaFreeAsync(d_tmp, s);
    return cuda_fail(h, e, "batched fold");
  }
  if (where == SRW_HOST) {
    SRW_CUDA(h, cudaMemcpyAsync(out, d_tmp, sizeof(float) * (size_t)P * h->n_rec, cudaMemcpyDeviceToHost, s),
             "download");
    SRW_CUDA(h, cudaFreeAsync(d_tmp, s), "free spectra");
    bool dom = false;
    srw_status st = check_status_word(h, s, &dom);
    if (st != SRW_OK) return st;
  } else if (!stream) {
    SRW_CUDA(h, cudaStreamSynchronize(s), "sync");
  }
  return SRW_OK;
}

srw_status srw_get_basis(srw_handle h, double* out) {
  if (!h) return fail(nullptr, SRW_EINVAL, "NULL handle");
  if (!out) return fail(h, SRW_EINVAL, "out is NULL");
  SRW_CUDA(h, cudaMemcpy(out, h->d_basis, sizeof(double) * kNB * (size_t)h->n_t, cudaMemcpyDeviceToHost), "download");
  return SRW_OK;
}

srw_status srw_fold_work(srw_handle h, srw_precision precision, int tile, double* executed_fraction) {
  if (!h) return fail(nullptr, SRW_EINVAL, "NULL handle");
  if (!executed_fraction) return fail(h, SRW_EINVAL, "executed_fraction is NULL");
  if (precision < SRW_FP32 || precision > SRW_FP16X3) return fail(h, SRW_EINVAL, "bad precision");
  if (tile != 0 && tile != 128 && tile != 256) return fail(h, SRW_EINVAL, "tile must be 0, 128 or 256");
  *executed_fraction = 1.0;
  if (precision != SRW_FP32 && h->tensor_ok)
    *executed_fraction = tc_block_fraction(h, tile ? tile : h->cfg[precision].bn, precision == SRW_FP16X3);
  return SRW_OK;
}

srw_status srw_gemv_work(srw_handle h, long long* bytes) {
  if (!h) return fail(nullptr, SRW_EINVAL, "NULL handle");
  if (!bytes) return fail(h, SRW_EINVAL, "bytes is NULL");
  *bytes = h->gv_blocks > 0 ? h->gv_bytes : 4LL * h->n_rec * h->ld_r;
  return SRW_OK;
}

srw_status srw_info(srw_handle h, srw_info_t* info) {
  if (!h || !info) return fail(h, SRW_EINVAL, "NULL argument");
  info->n_t = h->n_t;
  info->n_rec = h->n_rec;
  info->n_nodes = h->n_nodes;
  info->k_pad = h->k_pad;
  info->device = h->device;
  info->sm_count = h->sm_count;
  info->tensor_path = h->tensor_ok ? 1 : 0;
  info->lambda = h->has_esm_input ? 0.0 : h->lambda;
  info->device_bytes = h->device_bytes;
  return SRW_OK;
}

srw_status srw_autotune(srw_handle h, int P, srw_precision precision, const char* cache_path, void* stream,
                        int* chosen) {
  if (!h) return fail(nullptr, SRW_EINVAL, "NULL handle");
  if (P < 1) return fail(h, SRW_EINVAL, "P must be >= 1");
  if (!h->has_data) return fail(h, SRW_ENODATA, "call srw_set_data first");
  if (chosen) *chosen = 0;
  if (precision == SRW_FP32 || !h->tensor_ok) return SRW_OK;  // single SIMT configuration
  const int pr = (int)precision;
  std::string key;
  {
    std::ostringstream k;
    k << "srw-fold prec=" << pr << " M=" << P << " N=" << h->n_rec << " K=" << h->k_pad << " sm=" << h->sm_count;
    key = k.str();
  }
  if (cache_path) {
    std::ifstream in(cache_path);
    std::string line;
    while (std::getline(in, line)) {
      if (line.compare(0, key.size(), key) == 0 && line.size() > key.size() + 1) {
        const int idx = std::atoi(line.c_str() + key.size() + 1);
        if (idx >= 0 && idx < tc_num_configs()) {
          h->cfg[pr] = tc_config(idx);
          h->cfg_index[pr] = idx;
          destroy_graphs(h);
          if (chosen) *chosen = idx;
          return SRW_OK;
        }
      }
    }
  }
  cudaStream_t s = pick_stream(h, stream);
  srw_status st = ensure_staging(h, P);
  if (st != SRW_OK) return st;
  const int n_parts_max = h->rec_pad / 128;
  st = ensure_bparts(h, (size_t)n_parts_max * P);
  if (st == SRW_OK) st = ensure_coef(h, P);
  if (st != SRW_OK) return st;
  // deterministic in-box points for timing
  std::vector<float> th((size_t)P * 5);
  for (size_t q = 0; q < th.size(); ++q) th[q] = (float)(0.3 * std::sin(0.7 * (double)q + 0.1)) + (q % 5 == 4 ? 1.5f : 0.f);
  SRW_CUDA(h, cudaMemcpyAsync(h->d_theta, th.data(), sizeof(float) * th.size(), cudaMemcpyHostToDevice, s), "upload");
  cudaEvent_t e0, e1;
  SRW_CUDA(h, cudaEventCreate(&e0), "event");
  SRW_CUDA(h, cudaEventCreate(&e1), "event");
  float best = 1e30f;
  int best_i = -1, n_timed = 0;
  for (int i = 0; i < tc_num_configs(); ++i) {
    const FoldConfig c = tc_config(i);
    ++n_timed;
    int n_parts = 0;
    cudaError_t e = launch_fold_tc(h, h->d_theta, P, pr, c, h->d_bpart, s, &n_parts);  // warm-up
    if (e != cudaSuccess) continue;
    cudaEventRecord(e0, s);
    for (int r = 0; r < 3; ++r) launch_fold_tc(h, h->d_theta, P, pr, c, h->d_bpart, s, &n_parts);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    bool dom = false;
    if (check_status_word(h, s, &dom) != SRW_OK) continue;  // a timed-out configuration is never chosen
    if (ms < best) {
      best = ms;
      best_i = i;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best_i < 0) return fail(h, SRW_ECUDA, "no fold configuration ran");
  h->cfg_timed[pr] = n_timed;
  h->cfg[pr] = tc_config(best_i);
  h->cfg_index[pr] = best_i;
  destroy_graphs(h);
  if (chosen) *chosen = best_i;
  if (cache_path) {
    std::ofstream o(cache_path, std::ios::app);
    o << key << " " << best_i << "\n";
  }
  return SRW_OK;
}

srw_status srw_fold_config(int index, int* tile, int* k_block, int* stages) {
  if (index < 0 || index >= tc_num_configs()) return SRW_EINVAL;
  const FoldConfig c = tc_config(index);
  if (tile) *tile = c.bn;
  if (k_block) *k_block = c.bk;
  if (stages) *stages = c.stages;
  return SRW_OK;
}

srw_status srw_get_fold_config(srw_handle h, srw_precision precision, int* index, int* timed) {
  if (!h) return fail(nullptr, SRW_EINVAL, "NULL handle");
  if (precision == SRW_FP32 || precision < SRW_FP32 || precision > SRW_FP16X3)
    return fail(h, SRW_EINVAL, "precision must be a tensor-core precision");
  int idx = h->cfg_index[precision];
  if (idx < 0)  // the default of the precision
    for (int i = 0; i < tc_num_configs(); ++i) {
      const FoldConfig c = tc_config(i);
      if (c.bn == h->cfg[precision].bn && c.bk == h->cfg[precision].bk && c.stages == h->cfg[precision].stages) {
        idx = i;
        break;
      }
    }
  if (index) *index = idx;
  if (timed) *timed = h->cfg_timed[precision];
  return SRW_OK;
}

srw_status srw_set_fold_config(srw_handle h, srw_precision precision, int index) {
  if (!h) return fail(nullptr, SRW_EINVAL, "NULL handle");
  if (precision == SRW_FP32 || precision < SRW_FP32 || precision > SRW_FP16X3)
    return fail(h, SRW_EINVAL, "precision must be a tensor-core precision");
  if (index < 0 || index >= tc_num_configs()) return fail(h, SRW_EINVAL, "no such fold configuration");
  h->cfg[precision] = tc_config(index);
  h->cfg_index[precision] = index;
  destroy_graphs(h);
  return SRW_OK;
}

srw_status srw_set_reference(srw_handle h, const float* theta_ref) {
  if (!h) return fail(nullptr, SRW_EINVAL, "NULL handle");
  if (theta_ref) {
    for (int k = 0; k < 5; ++k)
      if (!std::isfinite(theta_ref[k])) return fail(h, SRW_EINVAL, "theta_ref must be finite");
    for (int k = 0; k < 5; ++k) h->theta_ref[k] = theta_ref[k];
    h->use_ref = 1;
  } else {
    h->use_ref = 0;
  }
  set_reference_coefs(h);
  destroy_graphs(h);
  cudaStream_t s = h->own_stream;
  SRW_CUDA(h, launch_reference_fold(h, s), "reference fold");
  if (h->has_data) SRW_CUDA(h, launch_data_ref(h, s), "data kernels");
  SRW_CUDA(h, cudaStreamSynchronize(s), "sync");
  ++h->version;
  return SRW_OK;
}

srw_status srw_profile(srw_handle h, int enable) {
  if (!h) return fail(nullptr, SRW_EINVAL, "NULL handle");
  if (enable && !h->ev_fold[0]) {
    SRW_CUDA(h, cudaEventCreate(&h->ev_fold[0]), "event create");
    SRW_CUDA(h, cudaEventCreate(&h->ev_fold[1]), "event create");
  }
  h->profile = enable ? 1 : 0;
  return SRW_OK;
}

srw_status srw_profile_read(srw_handle h, float* fold_ms) {
  if (!h || !fold_ms) return fail(h, SRW_EINVAL, "NULL argument");
  if (!h->profile) return fail(h, SRW_EINVAL, "profiling is not enabled");
  SRW_CUDA(h, cudaEventSynchronize(h->ev_fold[1]), "event sync");
  SRW_CUDA(h, cudaEventElapsedTime(fold_ms, h->ev_fold[0], h->ev_fold[1]), "event elapsed");
  return SRW_OK;
}

srw_status srw_check(srw_handle h, void* stream) {
  if (!h) return fail(nullptr, SRW_EINVAL, "NULL handle");
  bool domain = false;
  srw_status st = check_status_word(h, pick_stream(h, stream), &domain);
  if (st != SRW_OK) return st;
  if (domain) return fail(h, SRW_EDOMAIN, "expected count <= 0 in a bin with data: a value is +inf");
  return SRW_OK;
}

srw_status srw_destroy(srw_handle h) {
  if (!h) return SRW_OK;
  cudaSetDevice(h->device);
  if (h->own_stream) cudaStreamSynchronize(h->own_stream);
  release(h);
  delete h;
  return SRW_OK;
}

}  // extern "C"
