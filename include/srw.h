/*
 * srw.h - spectrum-reweighting likelihood for solar neutrino-electron
 * scattering on NVIDIA GB300 (sm_103a).  C ABI.
 *
 * Implements the per-parameter-point likelihood of arXiv 2607.00488 ("GPU-
 * accelerated spectrum reweighting for new-physics searches in solar
 * neutrino-electron scattering"):
 *   (a) recoil spectrum S_i(theta) per true-recoil bin from the flavour-
 *       weighted nu-e cross section (Sec. II, eqs. sm_cross_section,
 *       g_tilde, xs_mm, xs_total; Sec. III.A eq. fT) and the bin weights
 *       w_i = S_i(theta)/S_i(SM) (eqs. fT_norm, reweight_factor);
 *   (b) the fold through a fixed response R (eq. matrix_reweight,
 *       eq. visible_spectrum, eq. fNp_reweight);
 *   (c) the Poisson -2 ln L against binned data plus background templates
 *       (eqs. mu_total, logL; the Gaussian pull terms stay with the caller,
 *       as in Sec. IV.B).
 *
 * Parameter point layout (float32, 5 per point):
 *   theta = { eps_L_ee, eps_R_ee, eps_L_tautau, eps_R_tautau, mu_hat }
 *   with mu_hat = mu_nu / (1e-11 Bohr magnetons).  The NSI couplings shift
 *   the chiral couplings g_{L,R} of nu_e and nu_tau (eq. g_tilde); nu_mu
 *   keeps its SM couplings.
 *
 * Conventions
 *   - Energies are in MeV.  Cross sections are in units of
 *     sigma0 = 2 G_F^2 m_e / pi; the absolute scale cancels in the weights.
 *   - Every input array is COPIED by the library during the call that takes
 *     it; the caller keeps ownership and may free it on return.
 *   - Output buffers are owned by the caller.
 *   - `where` = SRW_HOST: pointers are host memory and the call returns when
 *     the result is in host memory.  `where` = SRW_DEVICE: pointers are
 *     device memory on the handle's device, and the call is asynchronous,
 *     stream-ordered on `stream` (a cudaStream_t; NULL = a stream owned by
 *     the handle, synchronised before return).  Any other `where` value, a
 *     NULL handle or required pointer, a point count below 1 or a precision
 *     outside srw_precision returns SRW_EINVAL before any device work; a
 *     likelihood call on a handle without srw_set_data returns SRW_ENODATA.
 *     The sizes of the caller's buffers are not known to the library: they
 *     must hold what the call's arguments say it reads and writes.
 *   - No C++ exception crosses this boundary.  Every call returns a status;
 *     srw_last_error() gives a message for the last failure on a handle.
 *   - A handle is not thread-safe: use one host thread (and one stream) per
 *     handle at a time.
 *   - All hot-path work runs in the library's CUDA kernels.  If no CUDA
 *     device is usable, srw_create fails with SRW_ECUDA; there is no CPU
 *     fallback.
 */
#ifndef SRW_H_
#define SRW_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct srw_ctx* srw_handle;

typedef enum {
  SRW_OK = 0,
  SRW_EINVAL = 1,       /* invalid argument: null pointer, size, NaN, unsorted edges */
  SRW_ENOMEM = 2,       /* device or host allocation failed */
  SRW_ECUDA = 3,        /* a CUDA runtime/driver call failed (message in srw_last_error) */
  SRW_ENODATA = 4,      /* srw_loglik before srw_set_data */
  SRW_EDOMAIN = 5,      /* some mu_j <= 0 with n_j > 0 (or mu_j < 0): that point's -2lnL is +inf */
  SRW_ETIMEOUT = 6,     /* a bounded device-side wait expired; the kernel aborted cleanly */
  SRW_EUNSUPPORTED = 7, /* the device cannot run the requested path (needs sm_103) */
  SRW_ECHECK = 8        /* debug build only: an index bounds check or a buffer canary failed */
} srw_status;

typedef enum { SRW_HOST = 0, SRW_DEVICE = 1 } srw_where;

/* Arithmetic of the response fold in the batched path.
 *   SRW_FP32   : FP32 SIMT products, FP32 accumulation with compensated
 *                chunk sums.
 *   SRW_BF16   : R and the weighted spectra rounded to BF16 on the tcgen05
 *                tensor cores, FP32 accumulation in tensor memory.
 *   SRW_BF16X3 : both operands split x = hi + lo (BF16 each, round to
 *                nearest even); the three products hi*hi + hi*lo + lo*hi
 *                accumulate in FP32 on the tensor cores.  The split keeps
 *                about 16 significant bits of each operand.
 *   SRW_FP16X3 : the same three products with FP16 hi and lo (about 22
 *                significant bits), each operand first scaled by an exact
 *                power of two into FP16 range: every row of R by its own
 *                factor (fixed at srw_create), the weighted-spectrum
 *                deviations of each point by a factor from a bound on their
 *                size; the epilogue divides both out exactly.  Same tensor-
 *                core work as SRW_BF16X3.
 * The -2lnL bin reduction accumulates in FP64 for every precision. */
typedef enum { SRW_FP32 = 0, SRW_BF16 = 1, SRW_BF16X3 = 2, SRW_FP16X3 = 3 } srw_precision;

/* Recoil binning (Sec. III.A).  The lower integration limit of every bin is
 * max(T_lo, t_min): t_min > 0 is the analysis threshold that regulates the
 * 1/T magnetic-moment term (Sec. II.C).  midpoint = 0 integrates the cross
 * section over each bin in closed form (default); midpoint = 1 evaluates it at
 * the bin centre times the bin width (eq. fT literally; a bin counts for a
 * node iff t_min <= T_c < T_max(E)). */
typedef struct {
  int n_t;                /* number of true-recoil bins, >= 1 */
  const double* t_edges;  /* n_t + 1 strictly ascending edges, t_edges[0] >= 0, MeV */
  int n_rec;              /* number of reconstructed bins, >= 1 */
  double t_min;           /* threshold, MeV, > 0 (1e-3 if <= 0 is passed) */
  int midpoint;           /* 0 = bin-integrated (default), 1 = midpoint */
} srw_binning;

/* One solar-neutrino component k (Sec. II.A, eq. rate_sm; Sec. III.A,
 * eq. fT): energy nodes E_n with weights w_n = phi_k(E_n) dE_n (a line is a
 * single node) and survival probability P_ee(E_n).  The nu_mu / nu_tau split
 * of 1 - P_ee is (1 - f_tau, f_tau). */
typedef struct {
  int n_nodes;            /* >= 1 */
  const double* e;        /* n_nodes neutrino energies, MeV, > 0 */
  const double* w;        /* n_nodes weights, >= 0, arbitrary units */
  const double* pee;      /* n_nodes survival probabilities in [0, 1] */
} srw_source;

typedef struct {
  double sin2w;           /* weak mixing angle sin^2(theta_W); <= 0 selects 0.23121 */
  double f_tau;           /* nu_tau fraction of 1 - P_ee; < 0 selects 0.5 */
  double exposure;        /* expected signal events after the response at theta = 0 (> 0) */
  const double* e_true_sm;/* optional n_t baseline true-recoil SM histogram (the MC
                             baseline E_true^SM of eq. matrix_reweight); NULL: use
                             lambda * S_SM with sum_j (R E_SM)_j = exposure */
} srw_options;

/* Create a likelihood context on the current CUDA device.
 *   R: n_rec x n_t row-major float32, host memory: the conditional response
 *      R[j][i] = P(reconstructed bin j | true bin i) (eq. visible_spectrum;
 *      column sums are the efficiency).  Must be finite and >= 0.
 * Builds, on the device, the FP64 coefficient spectra of the recoil spectrum
 * (the spectrum is a polynomial in the couplings and mu_hat^2), the SM
 * spectrum, the baseline E_SM, and the BF16 hi/lo split of R.
 * Errors: SRW_EINVAL (bad sizes/values), SRW_ENOMEM, SRW_ECUDA. */
srw_status srw_create(const srw_binning* binning, const srw_source* sources, int n_sources,
                      const float* R, const srw_options* options, srw_handle* out);

/* Per-component joint response (Sec. III.B-C, eqs. Rij, fNp_reweight,
 * mu_total).  Component k (sources[k] of srw_create_joint) comes with the 2-D
 * histogram N^(k) of a detector simulation of its SM events, from which
 *   R^(k)_ij = (N^(k)_ij / M^(k)_j) / sum_{i'j'} (N^(k)_i'j' / M^(k)_j') * s^(k)
 * (eq. Rij; i = true recoil bin, j = reconstructed bin), and its expected
 * counts are
 *   mu_j = M_j sum_k N_k sum_i R^(k)_ij S^(k)_i(theta) / S^(k)_i(SM) + background_j,
 * which is eq. mu_total with eq. fNp_reweight when the rate of a component
 * follows its integrated cross section over the recoil bins: the
 * normalisation prefactor of eq. fNp_reweight then cancels against
 * rate_k(theta) / rate_k(SM), and N_k = MT rate_k(SM).  Where S^(k)_i(SM) = 0
 * the weight is 1.  All arrays are host memory, row-major [n_rec][n_t] like
 * the conditional R of srw_create. */
typedef struct {
  const double* const* hist;  /* n_sources pointers to N^(k), n_rec x n_t, finite and >= 0; every
                                 histogram must hold some events */
  const double* const* mask;  /* NULL, or n_sources pointers (an entry may be NULL = all ones) to the
                                 live-time corrections M^(k)_j, n_rec values, finite and > 0 */
  const double* scale;        /* n_sources scale factors s^(k) > 0, or NULL (all 1) */
  const double* live;         /* n_rec common live-time factors M_j >= 0 of eq. mu_total, or NULL (all 1) */
  const double* events;       /* n_sources SM event numbers N_k > 0, or NULL: N_k = lambda F_k with
                                 F_k = sum_i S^(k)_i(SM) and lambda such that the SM signal
                                 sum_j mu_j - background_j equals options->exposure */
} srw_joint_response;

/* Create a likelihood context whose fold runs over the concatenated
 * (component, true bin) axis: one contraction sum over c = (k, i) of
 * R_cat[j][c] W_c(theta) with R_cat[j][(k,i)] = M_j N_k R^(k)_ij and
 * W_(k,i) = S^(k)_i(theta) / S^(k)_i(SM) (eq. fNp_reweight for every
 * component at once).  Only true bins where a component's histogram has
 * events enter the axis; its length is the handle's n_t (srw_info) and
 * srw_joint_layout maps it back.  Every entry point taking a handle works on
 * the result; srw_spectrum stage 0 / 1 return the per-component spectra /
 * weights on the concatenated axis, srw_get_basis the concatenated
 * coefficient spectra.  options->e_true_sm must be NULL.  binning->n_t is the
 * recoil binning of every component.
 * Errors: SRW_EINVAL (bad sizes/values, an empty histogram, a concatenated
 * axis above 49152 columns), SRW_ENOMEM, SRW_ECUDA. */
srw_status srw_create_joint(const srw_binning* binning, const srw_source* sources, int n_sources,
                            const srw_joint_response* response, const srw_options* options, srw_handle* out);

/* Columns of the fold axis: *n_columns receives its length; source[c] and
 * bin[c] (host arrays of *n_columns ints, each may be NULL) receive the
 * component and true bin of column c.  For an srw_create handle the axis is
 * the true bins themselves (source 0). */
srw_status srw_joint_layout(srw_handle h, int* n_columns, int* source, int* bin);

/* Attach binned data (eqs. mu_total, logL).  Host pointers:
 *   counts: n_rec observed counts n_j >= 0 (need not be integers);
 *   bkg:    n_bkg x n_rec background templates in expected counts (summed);
 *           may be NULL when n_bkg == 0;
 *   mask:   n_rec live-bin mask M_j (0 drops the bin), or NULL for all bins.
 * Precomputes the theta-independent part of -2lnL in FP64 on the device.
 * A call that fails after it has begun replacing the data leaves the handle
 * without data: likelihood calls return SRW_ENODATA until a call succeeds. */
srw_status srw_set_data(srw_handle h, const double* counts, const double* bkg, int n_bkg,
                        const unsigned char* mask);

/* Spectra at one parameter point theta (5 floats, host or device per `where`).
 *   stage 0: S_i(theta), the recoil spectrum per true bin        (n_t floats)
 *   stage 1: W_i = w_i(theta) E_SM,i, the reweighted true spectrum (n_t floats)
 *   stage 2: sum_i R_ji W_i, the folded signal                   (n_rec floats)
 *   stage 3: mu_j = M_j (signal_j + background_j)                (n_rec floats)
 * Computed by the single-point kernels (FP32). */
srw_status srw_spectrum(srw_handle h, const float* theta, int stage, float* out, int where, void* stream);

/* -2 ln L (without pull terms) for P parameter points.
 *   theta: P x 5 float32; out: P float64.
 * P == 1 with SRW_FP32 runs the single-point path (weighted spectrum from
 * the coefficient spectra, HBM-streaming fold, fused Poisson reduction);
 * otherwise the batched path (one
 * persistent fold launch over all points with the Poisson reduction fused
 * into its epilogue) in the requested precision.  Each distinct
 * (path, precision, P, theta, out, stream) call signature is captured once
 * into a CUDA graph and replayed.
 * Returns SRW_EDOMAIN (host calls only) when a point's value is +inf.
 * Host calls return SRW_EINVAL for a non-finite theta (checked on the host
 * while the device computes) and then leave out untouched.  Page-locked
 * host buffers make the copies asynchronous; pageable ones work too. */
srw_status srw_loglik(srw_handle h, const float* theta, int P, double* out, int where,
                      srw_precision precision, void* stream);

/* The plain single-point FP32 path applied to P points one after another, as
 * the paper's pipeline does it (Sec. IV.B): per point the cross-section
 * integrals are recomputed over all (node, bin) pairs by the spectrum kernel,
 * then one HBM-streaming fold; launches in order, replayed from a captured
 * CUDA graph per call signature, like srw_loglik. */
srw_status srw_loglik_points(srw_handle h, const float* theta, int P, double* out, int where, void* stream);

/* Exact rank-8 evaluation of the same -2 ln L (the paper's pipeline has no
 * counterpart; it follows from its equations): the recoil spectrum is linear
 * in the eight coupling monomials c(theta) (Sec. II, eqs. g_tilde, xs_total),
 * so the fold of eq. matrix_reweight is
 *   mu(theta) = R W_ref + b + M (c(theta) - c_ref),  M = R shat^T  [n_rec][8],
 * with M computed once in FP64 at srw_create.  Per point: eight coefficients,
 * eight FMAs and one Poisson deviance per reconstructed bin (FP32), summed in
 * double-float; no fold over the true bins.  grad (P x 5 float64, may be NULL)
 * receives d(-2 ln L)/d theta from the same linearity:
 *   2 sum_b (d c_b / d theta_k) sum_j M_jb (1 - n_j / mu_j).
 * Values agree with the batched paths to rounding; `where`/`stream` as in
 * srw_loglik; SRW_EDOMAIN (host calls) when a value is +inf. */
srw_status srw_loglik_linear(srw_handle h, const float* theta, int P, double* out, double* grad, int where,
                             void* stream);

/* -2 ln L with the overall signal rate profiled (a nuisance of the fit, Sec.
 * IV.B): per point
 *   min over alpha >= 0 of  -2 ln L(mu = alpha mu_sig(theta) + b)  [+ ((alpha - 1)/sigma_alpha)^2]
 * (the pull term only when sigma_alpha > 0; sigma_alpha = 0 leaves alpha
 * free), mu_sig from the rank-8 form of srw_loglik_linear.  Eight Newton steps
 * on the convex objective from alpha = 1, then the value at alpha-hat.
 * alpha (P float64, may be NULL) receives alpha-hat.  `where`/`stream` as in
 * srw_loglik. */
srw_status srw_loglik_profiled(srw_handle h, const float* theta, int P, double sigma_alpha, double* out,
                               double* alpha, int where, void* stream);

/* Folded signal spectra for P points with the batched fold:
 *   out[p * n_rec + j] = sum_i R_ji W_i(theta_p)   (P x n_rec float32)
 * in the requested precision (eq. matrix_reweight for a batch of points; no
 * data needed).  This is the exact-path generator of training spectra for a
 * learned surrogate.  Host calls allocate a temporary device buffer. */
srw_status srw_spectrum_batch(srw_handle h, const float* theta, int P, float* out, int where,
                              srw_precision precision, void* stream);

/* Copy the eight FP64 coefficient spectra B[8][n_t] (host memory) such that
 * S(theta) = sum_b c_b(theta) B_b with
 *   c = { gLe^2, gRe^2, -gLe gRe, gLt^2, gRt^2, -gLt gRt, 1, mu_hat^2 }
 * (e = nu_e, t = nu_tau couplings after the NSI shift; index 6 is the full
 * nu_mu spectrum; index 7 the magnetic-moment spectrum for mu_hat = 1). */
srw_status srw_get_basis(srw_handle h, double* out);

/* Time the candidate tile configurations of the batched fold for P points
 * at `precision` and keep the fastest for this handle.  If `cache_path` is
 * not NULL the choice is also read from / appended to that text file.
 * `chosen` (may be NULL) receives the index of the chosen configuration. */
srw_status srw_autotune(srw_handle h, int P, srw_precision precision, const char* cache_path,
                        void* stream, int* chosen);

/* Tensor-core fold configuration `index` (0 .. n-1; SRW_EINVAL past the
 * last): rec tile width `tile` (128 or 256 reconstructed bins per work item),
 * `k_block` (true bins per pipeline stage) and `stages` (shared-memory
 * pipeline depth, for the split precisions).  These are srw_autotune's
 * candidates.  Every candidate accumulates each output element from the same
 * updates in the same order, so the folded spectra are bitwise equal across
 * candidates (-2 ln L differs at most by the order of the per-tile partial
 * sums); candidates differ in speed only.  Any pointer may be NULL. */
srw_status srw_fold_config(int index, int* tile, int* k_block, int* stages);
/* Use configuration `index` for `precision` on this handle (a tensor-core
 * precision; replaces the autotuned choice until the next srw_autotune). */
srw_status srw_set_fold_config(srw_handle h, srw_precision precision, int index);
/* The configuration this handle uses for `precision` (*index) and how many
 * candidates the last srw_autotune for it timed (*timed; 0 if none ran or the
 * choice came from the cache file).  Either pointer may be NULL. */
srw_status srw_get_fold_config(srw_handle h, srw_precision precision, int* index, int* timed);

/* Work of the batched tensor-core fold at `precision` with rec tiles of
 * `tile` bins (128 or 256; 0 = the handle's current configuration):
 * *executed_fraction receives the fraction of the (rec tile, block of 64 true
 * bins) pairs it executes.  Per rec tile the fold
 * runs only the range of true-bin blocks in which the split response has a
 * nonzero element; the skipped blocks hold zeros in both split operands, so
 * their products are exact zeros and skipping them changes no bit of the
 * result.  1 for SRW_FP32 (the SIMT fold runs every block). */
srw_status srw_fold_work(srw_handle h, srw_precision precision, int tile, double* executed_fraction);

/* Bytes of R the single-point fold (the GEMV of srw_loglik with P = 1 and
 * SRW_FP32, and srw_spectrum stages 2-3) streams per call: each row's nonzero
 * band [first nonzero column rounded down to 4 floats, a length rounded up to
 * 32 floats), found at srw_create; outside it every element of R is an exact
 * zero, so the GEMV skips it without changing its result (eq. visible_spectrum).
 * The rows are split over the GEMV's blocks so that each streams about the
 * same number of bytes. */
srw_status srw_gemv_work(srw_handle h, long long* bytes);

/* Sizes of a context. */
typedef struct {
  int n_t, n_rec, n_nodes, k_pad;
  int device, sm_count, tensor_path;   /* tensor_path: 1 if the tcgen05 fold can run */
  double lambda;                        /* E_SM = lambda * S_SM normalisation (0 if e_true_sm given) */
  size_t device_bytes;                  /* persistent device memory held by the context */
} srw_info_t;
srw_status srw_info(srw_handle h, srw_info_t* info);

/* Reference point of the folds.  Every fold is evaluated as
 *   mu(theta) = R W_ref + R (W(theta) - W_ref)
 * (the same quantity as R W(theta), eq. matrix_reweight), with R W_ref
 * computed once in FP64, so the rounding errors of the FP32 and BF16 folds
 * scale with |W(theta) - W_ref| instead of |W(theta)|.  The default
 * reference is the SM point theta = 0.  theta_ref (5 floats, host memory)
 * selects another point (e.g. the current best fit); NULL removes the
 * point: the folds then carry all of W(theta) in the chosen precision except
 * its theta-independent part (the nu_mu spectrum), which is folded once in
 * FP64 in every mode.
 * Synchronous; invalidates captured graphs.  If the reference fold fails
 * (SRW_ECUDA), the new point's coefficients are in place with the old fold:
 * repeat the call before evaluating. */
srw_status srw_set_reference(srw_handle h, const float* theta_ref);

/* Kernel timing.  With profiling enabled, srw_loglik launches its kernels
 * directly (no CUDA graph) and records CUDA events on the call's stream
 * immediately before and after the fold kernel alone (the GEMV of the
 * single-point path, the batched fold otherwise; not the scale pre-pass, the
 * weights kernel or the final reduction); srw_profile_read waits for the last
 * such launch and returns that kernel's device time in milliseconds.  With
 * profiling disabled the calls replay their captured graphs. */
srw_status srw_profile(srw_handle h, int enable);
srw_status srw_profile_read(srw_handle h, float* fold_ms);

/* Allocation-free single-point likelihood (the paper has no counterpart; it
 * serves callers that cannot allocate device memory: code running inside
 * another framework's memory manager, which owns every device allocation, or
 * code that must not call cudaMalloc/cudaFree because they can synchronise the
 * device).  No handle and no allocation: every argument is a device pointer on
 * the current device, owned by the caller; the call is stream-ordered on
 * `stream` and returns before the result is ready.
 *   R:      n_rec x ld float32 response, row-major, zero beyond the last true bin
 *   W:      ld float32 weighted true spectrum (e.g. from srw_spectrum stage 1)
 *   counts: n_rec observed counts; bkg: n_rec summed background or NULL;
 *   mask:   n_rec live-bin mask or NULL;  out: 1 double, -2 ln L (eq. logL)
 * of mu_j = M_j (sum_i R_ji W_i + bkg_j), folded in FP32 like the single-
 * point path with the reference point disabled.
 * Limits: 1 <= n_rec <= 65536, ld a positive multiple of 64, R and W 16-byte
 * aligned; larger sizes are rejected with SRW_EINVAL (message from
 * srw_noalloc_last_error).  The kernels' scratch is a fixed static device array
 * of about 8 KB shared by every call: calls that overlap on the GPU race on it,
 * so serialise them (one stream).  The first call on each device resolves that
 * array's device address and sets a kernel attribute; make that first call
 * before any stream capture. */
srw_status srw_loglik_point_noalloc(const float* R, int n_rec, int ld, const float* W, const double* counts,
                                    const double* bkg, const unsigned char* mask, double* out, void* stream);
const char* srw_noalloc_last_error(void);

/* ---------------------------------------------------------------------------
 * Grouped evaluation: several detector configurations (each an srw_handle with
 * its own binning, response, data and reference point) evaluated in ONE
 * persistent fold launch, so that configurations of very different sizes
 * share the GPU without one launch per configuration.  Each configuration's
 * -2 ln L is the same quantity srw_loglik gives for that handle (eq. logL);
 * the paper evaluates one configuration at a time, the grouping is a batching
 * of the same computation.
 */
typedef struct srw_group_ctx* srw_group;

/* Group n handles (n >= 1, all on one device, each with data set) with P[g]
 * points for handle g (P[g] >= 0, sum >= 1).  The handles are not owned and
 * must outlive the group; later srw_set_data / srw_set_reference calls on a
 * member are picked up by the next group call.  The group builds one work
 * schedule per precision on first use (see srw_group_autotune). */
srw_status srw_group_create(const srw_handle* handles, int n, const int* P, srw_group* out);

/* -2 ln L of every point of every configuration.
 *   theta: (sum_g P[g]) x 5 float32, configuration 0's points first, then
 *          configuration 1's, ...;  out: sum_g P[g] float64 in the same order.
 * SRW_BF16 / SRW_BF16X3 / SRW_FP16X3: one persistent tensor-core launch over all
 * configurations (work items = 128-point x bn-bin tiles, bn = 128 or 256 per
 * configuration, assigned to CTAs longest-first onto the least-loaded CTA),
 * then one reduction launch.  SRW_FP32: the SIMT fold of each configuration
 * in turn, then the same reduction.  `where` and `stream` as in srw_loglik;
 * host calls return SRW_EDOMAIN when a value is +inf. */
srw_status srw_group_loglik(srw_group g, const float* theta, double* out, int where, srw_precision precision,
                            void* stream);

/* Time the candidate schedules for `precision` and keep the fastest:
 *   0: every configuration with bn = 256;
 *   1: bn per configuration from a cost model of its padded tiles;
 *   2: every configuration with bn = 128 (shallower stages, more of them);
 *   3: bn per configuration by measurement: starting from the fastest of 0-2,
 *      the tile width of one configuration at a time (the 16 most expensive)
 *      is flipped and kept where the launch gets more than 1 % shorter.
 * `chosen` (may be NULL) receives the candidate index.  No-op for SRW_FP32. */
srw_status srw_group_autotune(srw_group g, srw_precision precision, void* stream, int* chosen);

/* Use candidate schedule `candidate` (0 .. 3 as above; 3 before an autotune
 * falls back to 1) for `precision` without timing (a fixed choice, or one read
 * back from srw_group_schedule). */
srw_status srw_group_set_schedule(srw_group g, srw_precision precision, int candidate);

/* The schedule in use for `precision` (built if needed): widest tile, the tile
 * width of each configuration (bn: n ints, may be NULL), work items, CTAs and
 * the candidate index. */
srw_status srw_group_schedule(srw_group g, srw_precision precision, int* bn_max, int* bn, int* n_items,
                              int* n_cta, int* candidate);

/* Device time of the last grouped fold launch (as srw_profile / srw_profile_read). */
srw_status srw_group_profile(srw_group g, int enable);
srw_status srw_group_profile_read(srw_group g, float* fold_ms);

const char* srw_group_last_error(srw_group g);
srw_status srw_group_destroy(srw_group g);

/* ---------------------------------------------------------------------------
 * Learned surrogate (the paper has no counterpart; it serves dense scans):
 * a GELU MLP theta -> log mu_j (expected counts per reconstructed bin of
 * handle h), widths 5 -> 256 -> 256 -> 256 -> n_rec, trained on spectra of
 * the exact path and used to pre-screen scans, with the exact path deciding.
 *   x = (theta - centre) / half_width;  h_k = gelu(W_k h_{k-1} + b_k)  (k = 1..3,
 *   gelu(z) = z Phi(z));  y = W_4 h_3 + b_4;  log mu_j = m_j + s_j y_j
 * with per-bin standardization (m_j, s_j) of the training targets (identity
 * until srw_surrogate_fit sets it).  All products run on the tcgen05 tensor
 * cores in BF16 with FP32 accumulation; Adam keeps FP32 master weights.
 * Weight arrays (host, FP32, row-major) are passed as 8 pointers
 * {W1 [256][5], b1 [256], W2 [256][256], b2, W3 [256][256], b3, W4 [n_rec][256], b4 [n_rec]}.
 * The handle must have data set and the tensor-core path; it must outlive s.
 */
typedef struct srw_surrogate_ctx* srw_surrogate;

srw_status srw_surrogate_create(srw_handle h, const float* centre, const float* half_width,
                                const float* const* weights, srw_surrogate* out);
/* Replace the weights (resets the Adam state) / read the FP32 master weights. */
srw_status srw_surrogate_set_weights(srw_surrogate s, const float* const* weights);
srw_status srw_surrogate_get_weights(srw_surrogate s, float* const* weights);
/* Network output y (before de-standardization) for P points: y [P][n_rec] (host). */
srw_status srw_surrogate_forward(srw_surrogate s, const float* theta, int P, float* y);
/* Mean squared error of y against targets [P][n_rec] (host) and its gradients
 * (8 host arrays shaped like the weights); no update. */
srw_status srw_surrogate_gradients(srw_surrogate s, const float* theta, const float* targets, int P,
                                   float* const* grads, double* loss);
/* One training step (forward, backward, Adam with beta1 0.9, beta2 0.999,
 * eps 1e-8, learning rate lr) on P points; loss = the step's mean squared error. */
srw_status srw_surrogate_train_step(srw_surrogate s, const float* theta, const float* targets, int P, float lr,
                                    double* loss);
/* Train on n points (host theta [n][5], e.g. uniform in the box): the exact
 * path computes the expected counts mu = R W(theta) + b (srw_spectrum_batch in
 * `precision`, plus the summed background), the targets are log mu
 * standardized per bin over the training set (which also sets m_j, s_j), and
 * `epochs` passes of Adam over batches of `batch` points (fixed order) run with
 * a cosine learning-rate decay from lr to lr_final.  epoch_loss (may be NULL)
 * receives the mean squared error of each epoch.  Needs n * ceil(n_rec/256) *
 * 1 KB of device memory for the targets (8.4 GB at n = 1e6, n_rec = 2048). */
typedef struct {
  int batch;           /* points per step: a positive multiple of 128 */
  int epochs;
  float lr, lr_final;
  int precision;       /* srw_precision of the exact spectra */
} srw_fit_opts;
srw_status srw_surrogate_fit(srw_surrogate s, const float* theta, long long n, const srw_fit_opts* opts,
                             float* epoch_loss);

/* Checkpoint / resume of training (the paper has no counterpart: its fits are
 * stateless; the surrogate's training is not).  srw_surrogate_save writes the
 * whole training state: FP32 master weights and biases, Adam's first and
 * second moments and step count, the per-bin standardization and the number
 * of completed epochs of the last fit.  The file is written as path + ".tmp"
 * and renamed over `path`, so an interrupted save leaves the previous
 * checkpoint intact; it carries a checksum.  srw_surrogate_load restores it
 * into a surrogate of the same network and parameter box (SRW_EINVAL
 * otherwise, or if the file is damaged); *epochs_done (may be NULL) receives
 * the completed epochs.
 * srw_surrogate_fit_resume runs epochs first_epoch .. stop_epoch - 1
 * (stop_epoch <= 0: to opts->epochs) of the fit that srw_surrogate_fit(opts)
 * would run on the same points: the same
 * targets and batches (fixed order, no random state), the learning-rate
 * schedule continued from step first_epoch x steps, Adam continued from the
 * loaded state; if checkpoint_path is not NULL a checkpoint is saved after
 * every epoch.  A fit interrupted after epoch k and resumed from its
 * checkpoint with first_epoch = k ends with the same weights as the
 * uninterrupted fit.  epoch_loss (may be NULL) has opts->epochs entries; the
 * resumed ones are written. */
srw_status srw_surrogate_save(srw_surrogate s, const char* path);
srw_status srw_surrogate_load(srw_surrogate s, const char* path, long long* epochs_done);
srw_status srw_surrogate_fit_resume(srw_surrogate s, const float* theta, long long n, const srw_fit_opts* opts,
                                    int first_epoch, int stop_epoch, const char* checkpoint_path, float* epoch_loss);

/* Surrogate -2 ln L (eq. logL with mu_j = exp(m_j + s_j y_j), the handle's data
 * and mask) for P points; `where` and `stream` as in srw_loglik. */
srw_status srw_surrogate_loglik(srw_surrogate s, const float* theta, int P, double* out, int where, void* stream);

/* Pre-screened scan over the Sobol points with sequence indices [first,
 * first + n_points) mapped to the box (Sobol 1967 with Joe & Kuo 2008
 * direction numbers, Gray-code order; point 0 is the box corner):
 *   1. held-out check: the exact path and the surrogate on the n_check points
 *      check_theta; the box is cut into cells_per_dim^5 cells; a cell is
 *      flagged when its largest |d(-2lnL)| exceeds tol or it holds no check
 *      point;
 *   2. the surrogate's -2 ln L of every scan point;
 *   3. exact re-evaluation (in `precision`) of the points whose surrogate value
 *      is among the lowest keep_frac, plus
 *        SRW_SCAN_FLAG_CELLS : every point of every flagged cell;
 *        SRW_SCAN_ERROR_BARS : afterwards, every other point whose surrogate
 *          value minus margin_factor x max(its cell's held-out |d|, tol) is at
 *          or below the best exact value found (a point that could still be
 *          the minimum within the cell's error bar; cells without a check
 *          point: all of their points);
 *   4. the exact minimum among the re-evaluated points.
 * With n_check = 0 no cell is flagged (SRW_SCAN_FLAG_CELLS) or every cell
 * counts as unchecked (SRW_SCAN_ERROR_BARS). */
typedef enum { SRW_SCAN_FLAG_CELLS = 0, SRW_SCAN_ERROR_BARS = 1 } srw_scan_rule;
typedef struct {
  long long first, n_points;
  double keep_frac;
  const float* check_theta;
  int n_check;
  double tol;
  int cells_per_dim;           /* 1..16 */
  int precision;
  int rule;                    /* srw_scan_rule */
  double margin_factor;        /* >= 1 (SRW_SCAN_ERROR_BARS) */
} srw_scan_opts;
typedef struct {
  double best_value;             /* exact -2 ln L minimum among the re-evaluated points */
  long long best_index;          /* its Sobol index */
  float best_theta[5];
  double surrogate_min;          /* smallest surrogate value of the scan */
  long long n_kept;              /* points with surrogate values at or below the keep_frac threshold */
  long long n_selected;          /* all re-evaluated points */
  long long n_rescued;           /* of which added by the error-bar pass (SRW_SCAN_ERROR_BARS) */
  int n_cells, n_flagged_cells;
  double check_max_abs_d;        /* largest |d(-2lnL)| on the check set */
  float ms_check, ms_surrogate, ms_select, ms_exact;  /* device time of each phase */
} srw_scan_result;
srw_status srw_surrogate_scan(srw_surrogate s, const srw_scan_opts* opts, srw_scan_result* res);

/* A resumable scan (the paper has no counterpart).  The points of `opts` are
 * cut into chunks of chunk_points consecutive Sobol indices; each chunk is
 * one srw_surrogate_scan with the same options (its own lowest keep_frac and
 * the same cell rule), and after each chunk its result is recorded in the
 * text file state_path (rewritten through a temporary file and a rename).  A
 * call first reads that file, skips the chunks it records, and runs at most
 * max_new_chunks further chunks (<= 0: all the rest); *complete (may be
 * NULL) is 1 once every chunk is done.  *res is the result over the completed
 * chunks: the smallest exact minimum (ties: smaller Sobol index), counts and
 * times summed.  The file records the scan's options (and a checksum of the
 * check points): a file of another scan gives SRW_EINVAL.  Each chunk keeps its
 * own lowest keep_frac, so the number of re-evaluated points can exceed the
 * single call's; the minimum is the same whenever the rule's error bars hold
 * (the true minimum's chunk re-evaluates it).  Device memory is bounded by
 * the chunk, not by n_points. */
srw_status srw_surrogate_scan_chunked(srw_surrogate s, const srw_scan_opts* opts, long long chunk_points,
                                      const char* state_path, int max_new_chunks, srw_scan_result* res,
                                      int* complete);

/* The same scan without the surrogate: the exact path on every point; the
 * minimum, its index and the device time.  `precision`: an srw_precision of
 * the batched fold, or SRW_RANK8 for the exact rank-8 evaluator
 * (srw_loglik_linear). */
#define SRW_RANK8 16
srw_status srw_surrogate_scan_exact(srw_surrogate s, long long first, long long n_points, int precision,
                                    double* best_value, long long* best_index, float* ms);

/* Points first .. first + count - 1 of the scan's Sobol sequence, mapped to the
 * box (host theta [count][5]). */
srw_status srw_surrogate_sobol(srw_surrogate s, long long first, int count, float* theta);
/* The per-bin standardization m_j, s_j of log mu (n_rec floats each, host). */
srw_status srw_surrogate_get_standardization(srw_surrogate s, float* mean, float* stdv);

const char* srw_surrogate_last_error(srw_surrogate s);
srw_status srw_surrogate_destroy(srw_surrogate s);

/* Failure-detection diagnostic (the paper has no counterpart): launches one
 * block on the current device whose thread waits, with the same bounded wait
 * every kernel of the library uses, on an mbarrier that nothing arrives on.
 * After about limit_us microseconds (1 .. 1e6) the wait gives up, the block
 * records a timeout and returns; the call then reports SRW_ETIMEOUT (SRW_OK
 * would mean the wait did not expire).  The context remains usable. */
srw_status srw_diag_wait_timeout(unsigned limit_us);

/* Host-side fault injection (the paper has no counterpart): makes the
 * library's own failure paths run on demand, for tests, without faulting,
 * trapping or hanging the GPU.  An armed fault fires once, at the (skip+1)-th
 * matching event after it was armed, and then disarms:
 *   SRW_FAULT_ALLOC   a device allocation of the library is not made and
 *                     reports out-of-memory (the call returns SRW_ENOMEM);
 *   SRW_FAULT_LAUNCH  a kernel-launch check reports a launch failure (the
 *                     call returns SRW_ECUDA; a CUDA graph being captured for
 *                     the call is discarded, never cached);
 *   SRW_FAULT_TIMEOUT a fold launch (single-point GEMV or tensor-core fold)
 *                     makes one wait wait on an mbarrier that nothing arrives
 *                     on, with a 1 ms limit; the wait gives up and the kernel
 *                     takes its abort path: the affected points' values are
 *                     NaN, host-pointer calls return SRW_ETIMEOUT, and a
 *                     graph captured with the fault is run once, not cached.
 * SRW_FAULT_NONE disarms.  The environment variable SRW_FAULT ("alloc",
 * "launch" or "timeout", optionally ":N" for skip = N) arms a fault once per
 * process, before the first library call that allocates or launches; an
 * explicit srw_fault_inject() overrides it.  After every injected failure the
 * handle stays usable: the next call computes normally.  Process-wide state
 * (all handles and threads). */
typedef enum { SRW_FAULT_NONE = 0, SRW_FAULT_ALLOC = 1, SRW_FAULT_LAUNCH = 2, SRW_FAULT_TIMEOUT = 3 } srw_fault_kind;
srw_status srw_fault_inject(int kind, long long skip);
/* *kind = the armed fault kind (SRW_FAULT_NONE once it has fired or if none
 * is armed). */
srw_status srw_fault_pending(int* kind);
/* Parse an SRW_FAULT specification ("kind" or "kind:N") without arming it:
 * SRW_EINVAL if it is not one; kind and skip may be NULL. */
srw_status srw_fault_parse(const char* spec, int* kind, long long* skip);

/* Device-side status of the handle's calls with `where` = SRW_DEVICE since the
 * last srw_check (or the last host-pointer call, which reports and clears its
 * own): synchronises `stream` (NULL: the handle's stream), reads and clears
 * the handle's device status word and returns SRW_ETIMEOUT if a bounded
 * device wait expired (the affected points' values are NaN), else
 * SRW_EDOMAIN if some value is +inf, else SRW_OK. */
srw_status srw_check(srw_handle h, void* stream);

const char* srw_last_error(srw_handle h);
const char* srw_status_string(srw_status s);
srw_status srw_destroy(srw_handle h);

#ifdef __cplusplus
}
#endif

#endif /* SRW_H_ */
