// Internal state and launchers of the srw library (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <cstring>
#include <vector>

#include "../../include/srw.h"

namespace srw {

// Physical constants (CODATA 2018).
constexpr double kMe = 0.51099895000;           // electron mass [MeV]
constexpr double kAlpha = 1.0 / 137.035999084;  // fine-structure constant
constexpr double kGF = 1.1663787e-11;           // Fermi constant [MeV^-2]
constexpr double kPi = 3.14159265358979323846;
constexpr double kMuUnit = 1.0e-11;             // mu_hat unit: 1e-11 Bohr magnetons

// Number of coefficient spectra: the recoil spectrum is
//   S(theta) = sum_b c_b(theta) B_b,
//   c = {gLe^2, gRe^2, -gLe gRe, gLt^2, gRt^2, -gLt gRt, 1, mu_hat^2}.
constexpr int kNB = 8;

// Status bits written by kernels into the context's device status word.
constexpr unsigned kStatusTimeout = 1u;
constexpr unsigned kStatusDomain = 2u;
constexpr unsigned kStatusCheck = 4u;  // a debug-build bounds check failed

// Debug-build bounds checks (compiled with -DSRW_DEBUG_CHECKS, the library
// libsrw_debug.so): a failed check sets kStatusCheck in the kernel's status
// word and the kernel carries on (no trap: the GPU and the context stay
// usable); host-pointer calls and srw_check then report SRW_ECHECK.  In the
// release build the checks compile to nothing.
#ifdef SRW_DEBUG_CHECKS
#define SRW_CHECK(status_ptr, cond)                                \
  do {                                                             \
    if (!(cond)) atomicOr((status_ptr), ::srw::kStatusCheck);      \
  } while (0)
constexpr bool kDebugChecks = true;
#else
#define SRW_CHECK(status_ptr, cond) \
  do {                              \
  } while (0)
constexpr bool kDebugChecks = false;
#endif
// Canary doubles after the batched partial sums (debug build): a write past
// the end of that buffer changes them, which host-pointer calls detect.
constexpr int kCanaryDoubles = 64;
constexpr unsigned long long kCanaryBits = 0x7ff4dead5ca1ab1eull;  // a signalling-NaN pattern

// Device-side view of the theta-independent model tables.
struct ModelView {
  int n_t, n_rec, n_nodes, k_pad, ld_r, midpoint;
  float t_min;
  double t_min64;
  // nodes sorted by T_max descending
  const float4* node_a;  // {E, 1/E, k_n (int bits), m_e/E^2}; k_n = #bins with T_hi <= T_max(E)
  const float4* node_w;  // {w P_e, w P_mu, w P_tau, w}
  const float4* node_wlo;  // FP32 residuals of node_w (node_w + node_wlo = FP64 value)
  const float4* node_c;  // FP64-exact integrals over the clipped bin k_n: {I0, I1, J, MM}
  const double* node64;  // [5][n_nodes]: E, w P_e, w P_mu, w P_tau, w (FP64, same order)
  const int* bin_count;  // per bin: nodes [0, count) may contribute
  const float4* bin_f;   // {a = max(T_lo, t_min), b = T_hi, I0 = b - a, I1 = (b-a)(a+b)/2}
  const float* bin_l;    // log(b/a) per bin (from FP64)
  const double* bin64;   // [2][n_t]: T_lo, T_hi (FP64)
  const float* ssm32;    // [n_t] S_SM from the FP32 spectrum kernel (weights denominator)
  const float* esm32;    // [n_t] E_SM baseline
  const float* R;        // [n_rec][ld_r] FP32, zero padded
};

// Data view for the likelihood epilogues.
struct DataView {
  int n_rec;
  const double* n64;     // counts
  const double* b64;     // summed background
  const float4* nbm;     // {n_j, b_j, mask_j, 0} as floats for the batched epilogue
  const unsigned char* mask;
  const double* c_data;  // device scalar: 2 sum [n - n ln n + lnGamma(n+1)]
};

struct GraphEntry {
  int path, precision, P, prof;
  const void* theta;
  void* out;
  cudaStream_t stream;
  cudaGraphExec_t exec;
};

// Coupling monomials of the reference point (double-float), subtracted from
// those of each theta: the batched folds compute R (W(theta) - W_ref) and add
// the FP64 reference fold R W_ref.
struct CoefRef {
  float hi[kNB], lo[kNB];
};

// One detector configuration of a tensor-core fold launch.  A launch over a
// single handle carries one by value; a grouped launch (several handles, one
// persistent grid) reads an array of them from device memory.
struct TcGroup {
  const CUtensorMap* map_hi;   // R hi / lo maps, box 64 K x bn rows (grouped launches; global memory)
  const CUtensorMap* map_lo;
  const float4* shat_k8;       // [k_pad][8] coefficient spectra, k-major
  const float4* nb4;           // [n_rec] {n_j (0 where masked), b_j + R W_ref - n_j, mask 1/0, 1/r_j (FP16 row scale)}
  const double* c_data;        // data constant of -2 ln L (device scalar)
  long long parts_off;         // partial sums of the group: parts + parts_off, [n_tiles][P]
  int n_rec, k_pad, P, p_off;  // p_off: first point of the group in the launch's theta / out
  int bn, n_tiles;             // rec tile width (128 or 256) and number of rec tiles
  float sin2w_hi, sin2w_lo;
  CoefRef cref;
  const float* rinv;           // SRW_FP16X3: [n_rec] inverse power-of-two row scales of R
  const int2* kbr;             // [n_tiles] K-block walk {first block, +-count} over the tile's nonzero response
  float wmax[kNB];             // SRW_FP16X3: max_i |shat_b,i| (bound of the weighted-spectrum deviations)
};

// Where the per-tile partial sums of one configuration live, for the final
// reduction of a grouped call.
struct GroupPart {
  long long parts_off;
  int n_parts, P, p_off, pad;
  const double* c_data;
};

// Tile configuration of the batched fold.
struct FoldConfig {
  int kind;      // 0 = SIMT FP32, 1 = tcgen05
  int bn;        // rec-bin tile (N)
  int bk;        // true bins per pipeline stage (K block)
  int stages;    // pipeline depth (shared-memory stages)
  int w_warps;   // producer warps for the weighted-spectrum operand
};

}  // namespace srw

struct srw_ctx {
  int device = 0, sm_count = 0, cc_major = 0, cc_minor = 0;
  int n_t = 0, n_rec = 0, n_nodes = 0, midpoint = 0;
  int ld_r = 0;     // FP32 R row pitch (multiple of 4 floats)
  int k_pad = 0;    // recoil dimension padded to 64 for the BF16 operands
  int rec_pad = 0;  // n_rec padded to 256 rows for the BF16 split R
  double t_min = 1e-3, sin2w = 0.23121, f_tau = 0.5, exposure = 0, lambda = 0, kappa = 0;
  int has_esm_input = 0;
  int has_data = 0;
  int joint = 0;                   // srw_create_joint: the fold axis is (component, true bin)
  std::vector<int> col_src, col_bin;  // joint: component and true bin of every column
  unsigned long long version = 0;  // bumped when data or the reference point change
  size_t device_bytes = 0;

  // model tables
  float4* d_node_a = nullptr;
  float4* d_node_w = nullptr;
  float4* d_node_c = nullptr;
  float4* d_node_wlo = nullptr;
  double* d_node64 = nullptr;
  int* d_bin_count = nullptr;
  float4* d_bin_f = nullptr;
  float* d_bin_l = nullptr;
  double* d_bin64 = nullptr;
  double* d_basis = nullptr;   // [8][n_t] FP64 coefficient spectra
  double* d_ssm64 = nullptr;   // [n_t] FP64 S_SM
  double* d_esm64 = nullptr;   // [n_t] FP64 E_SM
  float* d_ssm32 = nullptr;
  float* d_esm32 = nullptr;
  float* d_shat = nullptr;     // [8][k_pad] FP32 pre-weighted basis (W = sum_b c_b shat_b)
  float* d_shat_lo = nullptr;  // [8][k_pad] FP32 residuals of shat
  float* d_shat_k8 = nullptr;  // [k_pad][8] FP32 shat, k-major (tensor-core W producers)
  float* d_R = nullptr;        // [n_rec][ld_r]
  __nv_bfloat16* d_rhi = nullptr;  // [rec_pad][k_pad]
  __nv_bfloat16* d_rlo = nullptr;
  __half* d_rhi16 = nullptr;       // [rec_pad][k_pad] FP16 split of R scaled by row (SRW_FP16X3)
  __half* d_rlo16 = nullptr;
  float* d_rinv = nullptr;         // [n_rec] inverse row scales of the FP16 split
  int2* d_kbr[2][2] = {};          // [FP16 split?][bn == 256] K-block range of each rec tile
  std::vector<int2> kbr_h[2][2];   // host copies (grouped scheduling, work accounting)
  float wmax[8] = {};              // max_i |shat_b,i|
  float4* d_coef = nullptr;        // [P][2] per-point W-producer coefficients and FP16 scales (batched scratch)
  double* d_linM = nullptr;        // [n_rec][8] M = R shat^T (FP64) of the rank-8 evaluator
  float4* d_lin = nullptr;         // [3 n_rec] per-bin constants of the rank-8 evaluator
  float4* d_linp = nullptr;        // [n_rec] {mu_ref, b, n, 0} for the profiled evaluation
  int coef_cap = 0;

  // data
  double* d_n64 = nullptr;
  double* d_b64 = nullptr;
  float4* d_nbm = nullptr;
  float2* d_nb2 = nullptr;     // {n_j or -1 where masked, b_j + R W_ref} (surrogate epilogue)
  float4* d_nb4 = nullptr;     // {n_j (0 where masked), b_j + R W_ref - n_j, mask 1/0, 1/r_j} (tensor-core epilogue)
  unsigned char* d_mask = nullptr;
  double* d_cdata = nullptr;

  // scratch (device)
  float* d_W = nullptr;        // [ld_r] weighted true spectrum of the point path
  float* d_S = nullptr;        // [n_t] spectrum of the point path
  float* d_musig = nullptr;    // [n_rec]
  float* d_mu = nullptr;       // [n_rec]
  double* d_part = nullptr;    // partial sums (point path: per block)
  int part_cap = 0;
  unsigned* d_ticket = nullptr;
  unsigned* d_status = nullptr;
  int4* d_gv_seg = nullptr;    // single-point GEMV: stream segments of every block (rows' nonzero bands)
  int* d_gv_segs = nullptr;    // [gv_blocks + 1] first segment of each GEMV block
  int* d_gv_rows = nullptr;    // [gv_blocks + 1] first row of each GEMV block (band-balanced split)
  int2* d_simt_kr = nullptr;   // FP32 batched fold: K-tile range [first, end) of each 128-bin rec tile
  int gv_blocks = 0, gv_max_rows = 0, gv_max_segs = 0;
  long long gv_bytes = 0;      // bytes of R the GEMV streams (the bands)
  double* d_bpart = nullptr;   // batched partials [n_tiles][P]
  size_t bpart_cap = 0;
  float* d_theta = nullptr;    // staging for host theta
  double* d_out = nullptr;     // staging for host out
  int stage_cap = 0;
  float* d_theta0 = nullptr;   // 5 zeros

  cudaStream_t own_stream = nullptr;
  std::vector<srw::GraphEntry> graphs;
  srw::FoldConfig cfg[4];      // per precision
  int cfg_index[4] = {-1, -1, -1, -1};
  int cfg_timed[4] = {0, 0, 0, 0};  // candidates the last srw_autotune timed, per precision
  bool tensor_ok = false;
  void* tmap = nullptr;        // TMA descriptors for R hi/lo (tcgen05 path)
  int profile = 0;             // record events around the fold launch
  int use_ref = 1;             // fold deviations from the reference point
  float theta_ref[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  srw::CoefRef cref{};          // monomials of theta_ref (zeros when use_ref == 0)
  float gref[2][10] = {};       // coupling products of theta_ref for the spectrum kernel (hi, lo)
  double* d_muref64 = nullptr;  // [n_rec] R W_ref in FP64
  double* d_bref64 = nullptr;   // [n_rec] R W_ref + background (FP64)
  cudaEvent_t ev_fold[2] = {nullptr, nullptr};
  std::string err;
};

namespace srw {

// fault.cu: host-side fault injection (see srw_fault_inject in srw.h).
// True when an armed fault of `kind` fires at this event (it then disarms).
bool fault_fire(int kind);
// True if a timeout fault fired on this thread since the last call (clears it).
bool fault_take_timeout_fired();

// Device allocation of the library (subject to SRW_FAULT_ALLOC injection).
template <class T>
inline cudaError_t dev_malloc(T** p, size_t bytes) {
  if (fault_fire(SRW_FAULT_ALLOC)) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}
template <class T>
inline cudaError_t dev_malloc_async(T** p, size_t bytes, cudaStream_t s) {
  if (fault_fire(SRW_FAULT_ALLOC)) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocAsync(reinterpret_cast<void**>(p), bytes, s);
}
// Status of the kernel launch just made (subject to SRW_FAULT_LAUNCH injection).
inline cudaError_t launch_result() {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && fault_fire(SRW_FAULT_LAUNCH)) return cudaErrorLaunchFailure;
  return e;
}
// 1 when this fold launch is to take an injected timeout (SRW_FAULT_TIMEOUT).
inline int inject_timeout() { return fault_fire(SRW_FAULT_TIMEOUT) ? 1 : 0; }

srw_status fail(srw_ctx* h, srw_status s, const std::string& msg);
srw_status cuda_fail(srw_ctx* h, cudaError_t e, const char* what);

ModelView model_view(const srw_ctx* h);
DataView data_view(const srw_ctx* h);

// spectrum.cu
cudaError_t launch_basis_fp64(const srw_ctx* h, cudaStream_t s);
cudaError_t launch_spectrum_point(const srw_ctx* h, const float* theta, float* S_out, float* W_out,
                                  float* ssm_out, cudaStream_t s, bool delta = false);
cudaError_t launch_reference_fold(srw_ctx* h, cudaStream_t s);
cudaError_t launch_weights_from_basis(const srw_ctx* h, const float* theta, float* W, cudaStream_t s);
cudaError_t launch_build_shat(srw_ctx* h, cudaStream_t s);

// joint.cu: per-component joint response (eq. Rij) on the concatenated axis.
// colZ_i = sum_j N_ji / M_j and colY_i = sum_j live_j N_ji / M_j (FP64).
cudaError_t launch_joint_colsums(const double* hist, const double* mask, const double* live, int n_rec, int n_t,
                                 double* colZ, double* colY, cudaStream_t s);
// R[j][col0 + c] = live_j factor N_{j, cols[c]} / M_j, rounded to FP32.
cudaError_t launch_joint_gather(const double* hist, const double* mask, const double* live, int n_rec, int n_t,
                                const int* cols, int n_cols, double factor, float* R, int ld, int col0,
                                cudaStream_t s);
// Spectra of one point from the FP64 coefficient spectra over the handle's
// axis: mode 0 S_c(theta), mode 1 W_c = S_c(theta) / S_SM,c E_SM,c (E_SM,c where S_SM,c = 0).
cudaError_t launch_basis_eval(const srw_ctx* h, const float* theta, int mode, float* out, cudaStream_t s);

// likelihood.cu
cudaError_t launch_set_data(srw_ctx* h, const double* d_bkg, int n_bkg, cudaStream_t s);
cudaError_t launch_data_ref(srw_ctx* h, cudaStream_t s);
cudaError_t launch_add_ref(const srw_ctx* h, float* out, int P, cudaStream_t s);
int fold_point_grid(const srw_ctx* h);
// Nonzero bands of R's rows and the band-balanced row split of the GEMV
// (R: the device R copied to the host, n_rec x ld_r).
// True when every one of the n floats is finite (exponent field not all ones):
// one branch-free pass over their bits, which the host compiler vectorises
// (a per-element isfinite with an early exit does not).
inline bool all_finite(const float* x, size_t n) {
  uint32_t bad = 0u;
  for (size_t q = 0; q < n; ++q) {
    uint32_t b;
    std::memcpy(&b, x + q, sizeof b);
    bad |= (uint32_t)((b & 0x7f800000u) == 0x7f800000u);
  }
  return bad == 0u;
}

cudaError_t gemv_prepare(srw_ctx* h, const std::vector<float>& R);
cudaError_t simt_prepare(srw_ctx* h, const std::vector<float>& R);
void fold_point_init();
int fold_simt_parts(int n_rec);
cudaError_t launch_fold_point(const srw_ctx* h, const float* W, float* musig_out, float* mu_out, double* out,
                              cudaStream_t s, bool delta = false);
// The single-point fold (delta mode) as a programmatic dependent of the
// preceding kernel on s: it starts while that kernel runs and waits for W.
cudaError_t launch_fold_point_after(const srw_ctx* h, const float* W, double* out, cudaStream_t s);
cudaError_t launch_reduce_parts(const srw_ctx* h, const double* parts, int n_parts, int P, double* out,
                                cudaStream_t s);

// fold_simt.cu
cudaError_t launch_fold_simt(const srw_ctx* h, const float* theta, int P, double* parts, cudaStream_t s,
                             int* n_parts, float* musig_out = nullptr);

// fold_tc.cu
bool tc_supported(const srw_ctx* h);
cudaError_t tc_prepare(srw_ctx* h);
void tc_release(srw_ctx* h);
int tc_num_configs();
FoldConfig tc_config(int i);
cudaError_t launch_fold_tc(const srw_ctx* h, const float* theta, int P, int precision, const FoldConfig& cfg,
                           double* parts, cudaStream_t s, int* n_parts, float* musig_out = nullptr,
                           cudaEvent_t ev_begin = nullptr, cudaEvent_t ev_end = nullptr);
cudaError_t launch_split_r(srw_ctx* h, cudaStream_t s);
// linear.cu: exact rank-8 evaluation mu = mu_ref + b + M (c(theta) - c_ref).
cudaError_t launch_linear_m(srw_ctx* h, cudaStream_t s);
cudaError_t launch_linear_consts(srw_ctx* h, cudaStream_t s);
cudaError_t launch_linear_loglik(const srw_ctx* h, const float* theta, int P, double* out, double* grad,
                                 cudaStream_t s);
cudaError_t launch_linear_profiled(const srw_ctx* h, const float* theta, int P, double sigma_alpha, double* out,
                                   double* alpha, cudaStream_t s);
// Per-point power-of-two scales of the FP16 split for a grouped launch.
cudaError_t launch_group_coef(const TcGroup* d_groups, int n_groups, int max_P, const float* theta, bool f16,
                              float4* out,
                                cudaStream_t s);
int tc_max_groups();
// Descriptor of handle h as a configuration with rec tile bn (maps left null)
// for the FP16 split (f16) or the BF16 split.
TcGroup tc_group_of(const srw_ctx* h, int bn, bool f16);
// Per rec tile, the K blocks where the split response has nonzero elements
// (both splits, both tile widths); blocks outside hold only zeros.
cudaError_t tc_block_ranges(srw_ctx* h, const std::vector<float>& R, cudaStream_t s);
// Fraction of the (rec tile, K block) pairs a batched fold executes.
double tc_block_fraction(const srw_ctx* h, int bn, bool f16);
// Tensor maps of h's hi / lo response (FP16 split if f16, else BF16) with a
// box of bk (64 or 32) K x bn rows.
cudaError_t tc_encode_maps(const srw_ctx* h, int bn, bool f16, CUtensorMap* hi, CUtensorMap* lo, int bk = 64);
// One persistent launch of n_cta CTAs over several configurations.  Slot
// k * n_cta + b of items (n_slots in all) is CTA b's k-th item {group, m0,
// n0, 0}; a group < 0 ends that CTA's list.  bn_max (128 or 256) bounds every
// group's bn.
cudaError_t launch_fold_tc_group(int bn_max, int precision, const TcGroup* d_groups, const int4* d_items, int n_slots,
                                 int n_cta, const float4* coef, double* parts, unsigned* status,
                                 cudaStream_t s);
// -2 ln L of every point of a grouped call from its per-tile partial sums.
cudaError_t launch_group_reduce(const GroupPart* d_gparts, int n_groups, int max_P, const double* parts,
                                double* out, unsigned* status, cudaStream_t s);

}  // namespace srw
