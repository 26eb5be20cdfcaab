"""GPU parity of the per-component joint response (srw_create_joint) against
the FP64 joint oracle (Sec. III.B-C, eqs. Rij, fNp_reweight, mu_total).

The GPU builds R_cat[j][(k, i)] = M_j N_k R^(k)_ij in FP64 and stores it in
FP32 (one rounding, 2^-24 relative per element), then runs the same folds as
a conditional handle over the concatenated (component, true bin) axis.  The
bars are those of the conditional parity tests:
* layout (which columns enter the axis) and the coefficient spectra: exact /
  1e-10 relative;
* FP32 spectra per bin: 1e-6 relative (the stored FP32 R_cat adds at most
  6e-8);
* -2 ln L: |d| <= 1e-4 (FP32) and 1e-3 (BF16 and FP16 splits) in the fit
  region, |d| <= tol + 2 B elsewhere with the measured per-bin budget
  B = 2 sum_j |1 - n_j/mu_j| |dmu_j|.  The fit region is taken by its
  likelihood: points within Delta(-2 ln L) <= 100 of the reference point.
  The tensor-core folds accumulate in FP32 with a small systematic bias
  (measured -1e-6 to -3e-6 of the folded deviation R (W - W_ref), from
  truncation in the accumulation), which moves -2 ln L by about
  2 beta Delta(-2 ln L): below 1e-3 inside that region.

Workloads: a small three-component set (7Be lines, pep, 13N; 600 true x 300
reconstructed bins, so the concatenated axis of 863 columns spans fourteen
K blocks with a ragged tail and the reconstructed bins three ragged row
tiles), and the full six-component solar set (4096 x 2048 bins, 1e7 Monte
Carlo events per component).
"""

import numpy as np
import pytest

import oracle as O
import workloads
from oracle.joint_oracle import JointOracleModel, normalised_spectrum
from workloads.solar import _source, continuum_nodes, pee_solar

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_BIN = 1e-6
TOL_LL = {"fp32": 1e-4, "bf16x3": 1e-3, "fp16x3": 1e-3}


@pytest.fixture(scope="module")
def srw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2607_00488_gb300 as pkg
    return pkg


def small_workload(events=None):
    t_edges = np.linspace(0.0, 2.0, 601)
    rec_edges = np.linspace(0.0, 2.0, 301)
    e, w = continuum_nodes(1.2, 200, 3.0e8)
    comps = [_source("be7", np.array([0.862, 0.384]), np.array([4.5e9, 0.5e9]), pee_solar),
             _source("pep", np.array([1.44]), np.array([1.4e8]), pee_solar),
             _source("n13", e, w, pee_solar)]
    f_hat = [normalised_spectrum(O.recoil_spectrum([c], t_edges, np.zeros(5))) for c in comps]
    wl = workloads.joint_workload("joint_small", t_edges, rec_edges, comps, f_hat, 1.0e5, 2_000_000, 30)
    wl["events"] = events
    return wl


class JointCase:
    def __init__(self, srw, wl, counts=None):
        self.wl = wl
        self.ref = JointOracleModel.from_workload(wl)
        if counts is None:  # pseudo-data from the oracle's SM expectation
            self.ref.set_data(np.zeros(len(wl["live"])), wl["bkg"])
            counts = workloads.poisson_counts(self.ref.mu(np.zeros(5)), 0)
        self.counts = counts
        self.ref.set_data(counts, wl["bkg"])
        self.lk = srw.Likelihood(wl, counts)


@pytest.fixture(scope="module")
def small(srw):
    c = JointCase(srw, small_workload())
    yield c
    c.lk.close()


@pytest.fixture(scope="module")
def solar(srw):
    wl = workloads.solar_joint_workload()
    c = JointCase(srw, wl, workloads.load_counts(wl["name"]))
    yield c
    c.lk.close()


def near_sm(n, seed):
    rng = np.random.default_rng(seed)
    th = np.zeros((n, 5), np.float32)
    th[:, :4] = rng.uniform(-0.02, 0.02, (n, 4))
    th[:, 4] = rng.uniform(0.0, 0.5, n)
    return th


def budget(case, th, mu_sig_gpu):
    mu = case.ref.mu(th.astype(np.float64))
    dmu = np.asarray(mu_sig_gpu, np.float64) - case.ref.mu_sig(th.astype(np.float64))
    on = mu > 0
    return 2.0 * np.sum(np.abs(1.0 - case.counts[on] / mu[on]) * np.abs(dmu[on]))


def rel_max(got, want, floor):
    got, want = np.asarray(got, np.float64), np.asarray(want, np.float64)
    big = np.abs(want) > floor
    return np.max(np.abs(got[big] - want[big]) / np.abs(want[big]))


# ---------------------------------------------------------------- axis and create-time tables
@pytest.mark.parametrize("name", ["small", "solar"])
def test_layout_is_the_bins_with_events(name, request):
    c = request.getfixturevalue(name)
    src, b = c.lk.layout()
    want_src, want_bin = [], []
    for k, h in enumerate(c.wl["hist"]):
        cols = np.nonzero(h.sum(axis=0) > 0)[0]
        want_src += [k] * cols.size
        want_bin += list(cols)
    assert np.array_equal(src, want_src) and np.array_equal(b, want_bin)
    assert c.lk.info()["n_t"] == len(want_src)


@pytest.mark.parametrize("name", ["small", "solar"])
def test_basis_is_the_component_coefficient_spectra(name, request):
    c = request.getfixturevalue(name)
    wl = c.wl
    src, b = c.lk.layout()
    got = c.lk.basis()
    for k, comp in enumerate(wl["components"]):
        want = O.coefficient_spectra([comp], wl["t_edges"], wl["t_min"], wl["sin2w"], wl["f_tau"])
        sel = src == k
        np.testing.assert_allclose(got[:, sel], want[:, b[sel]], rtol=1e-10, atol=1e-13 * np.abs(want).max())


# ---------------------------------------------------------------- spectra per bin
@pytest.mark.parametrize("name", ["small", "solar"])
def test_spectrum_stages(name, request):
    c = request.getfixturevalue(name)
    src, b = c.lk.layout()
    for t in np.concatenate([np.zeros((1, 5), np.float32), workloads.theta_box(2, 40)]):
        t64 = t.astype(np.float64)
        f = [c.ref.component_spectrum(k, t64) for k in range(len(c.wl["components"]))]
        s_want = np.array([f[k][i] for k, i in zip(src, b)])
        assert rel_max(c.lk.spectrum(t, 0), s_want, 1e-12 * s_want.max()) <= TOL_BIN
        w_want = np.array([f[k][i] / c.ref.f_sm[k][i] if c.ref.f_sm[k][i] > 0 else 1.0 for k, i in zip(src, b)])
        assert rel_max(c.lk.spectrum(t, 1), w_want, 0.0) <= TOL_BIN
        mu_sig = c.ref.mu_sig(t64)
        assert rel_max(c.lk.spectrum(t, 2), mu_sig, 1e-3 * mu_sig.max()) <= TOL_BIN
        mu = c.ref.mu(t64)
        assert rel_max(c.lk.spectrum(t, 3), mu, 1e-3 * mu.max()) <= TOL_BIN


@pytest.mark.parametrize("prec,tol", [("fp32", TOL_BIN), ("bf16x3", 2e-5), ("fp16x3", 5e-6)])
def test_batched_spectra_per_bin(srw, small, prec, tol):
    th = np.concatenate([np.zeros((1, 5), np.float32), workloads.theta_box(130, 41)])
    got = small.lk.spectrum_batch(th, srw.PRECISIONS[prec])
    for k in (0, 1, 64, 127, 128, 130):
        want = small.ref.mu_sig(th[k].astype(np.float64))
        assert rel_max(got[k], want, 1e-3 * want.max()) <= tol, k


# ---------------------------------------------------------------- -2 ln L
# Fit-region points: near the SM reference, scaled so that -2 ln L lies within
# 100 of its value at the reference (with the components' Monte Carlo shapes
# |eps| = 0.02 is already ~200 away on both sets).
FIT_SCALE = np.array([0.25, 0.25, 0.25, 0.25, 0.5], np.float32)


@pytest.mark.parametrize("name", ["small", "solar"])
def test_loglik_fit_region_all_paths(srw, name, request):
    c = request.getfixturevalue(name)
    th = np.concatenate([np.zeros((1, 5), np.float32), near_sm(7, 42) * FIT_SCALE])
    want = c.ref.neg2lnl_batch(th.astype(np.float64))
    assert np.max(want - want[0]) <= 100.0, want - want[0]
    single = np.array([c.lk.loglik(t[None, :], srw.SRW_FP32)[0] for t in th])
    got = {"single": single, "points": c.lk.loglik_points(th), "fp32": c.lk.loglik(th, srw.SRW_FP32),
           "bf16x3": c.lk.loglik(th, srw.SRW_BF16X3), "fp16x3": c.lk.loglik(th, srw.SRW_FP16X3)}
    print(name, "fit region max |d|:", {k: float(np.max(np.abs(v - want))) for k, v in got.items()},
          "max delta(-2lnL) %.1f" % np.max(want - want[0]))
    for k, v in got.items():
        tol = TOL_LL.get(k, TOL_LL["fp32"])
        assert np.max(np.abs(v - want)) <= tol, (k, v - want)


@pytest.mark.parametrize("name", ["small", "solar"])
def test_rank8_evaluator(srw, name, request):
    # mu = mu_ref + b + M (c - c_ref) with its constants in FP32: per-bin errors
    # of 2^-24 relative of mu_j, so |d| <= 1e-4 + 2 B with
    # B = 2 sum_j |1 - n_j / mu_j| 1.2e-7 mu_j (the conditional path's bound)
    c = request.getfixturevalue(name)
    th = np.concatenate([np.zeros((1, 5), np.float32), near_sm(5, 50), workloads.theta_box(3, 51)])
    got = c.lk.loglik_linear(th)
    for k, t in enumerate(th):
        t64 = t.astype(np.float64)
        mu = c.ref.mu(t64)
        on = mu > 0
        b = 2.0 * np.sum(np.abs(1.0 - c.counts[on] / mu[on]) * 1.2e-7 * mu[on])
        want = c.ref.neg2lnl(t64)
        assert abs(got[k] - want) <= TOL_LL["fp32"] + 2.0 * b, (k, got[k] - want, b)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "fp16x3"])
def test_loglik_within_measured_budget(srw, small, prec):
    th = np.concatenate([near_sm(4, 43), workloads.theta_box(9, 43)])
    p = srw.PRECISIONS[prec]
    got = small.lk.loglik(th, p)
    spectra = small.lk.spectrum_batch(th, p)
    for k in range(th.shape[0]):
        want = small.ref.neg2lnl(th[k].astype(np.float64))
        assert abs(got[k] - want) <= TOL_LL[prec] + 2.0 * budget(small, th[k], spectra[k]), k


def test_full_scan_sampled(srw, solar):
    # the batched launch at the scan size: 65,536 points in one call, sampled
    th = workloads.theta_box(65536, 3)
    th[:3] = near_sm(3, 44)
    dev = torch.device("cuda")
    out = torch.empty(65536, dtype=torch.float64, device=dev)
    solar.lk.loglik(torch.tensor(th, device=dev), srw.SRW_FP16X3, out=out)
    got = out.cpu().numpy()
    assert np.all(np.isfinite(got))
    for k in (0, 1, 2, 4097, 65535):
        want = solar.ref.neg2lnl(th[k].astype(np.float64))
        if k < 3:
            assert abs(got[k] - want) <= TOL_LL["fp16x3"], (k, got[k] - want)
        else:
            b = budget(solar, th[k], solar.lk.spectrum_batch(th[k:k + 1], srw.SRW_FP16X3)[0])
            assert abs(got[k] - want) <= TOL_LL["fp16x3"] + 2.0 * b, (k, got[k] - want, b)


def test_profiled_normalisation(srw, small):
    th = np.concatenate([np.zeros((1, 5), np.float32), near_sm(3, 45)])
    v, a = small.lk.loglik_profiled(th, 0.1)
    for k, t in enumerate(th):
        mu_sig = small.ref.mu_sig(t.astype(np.float64))
        want, a_want = O.profiled_neg2lnl(mu_sig, small.ref.bkg_sum, small.counts, 0.1)
        assert abs(v[k] - want) <= 1e-3 and abs(a[k] - a_want) <= 1e-5, (k, v[k] - want, a[k] - a_want)


def test_reference_point_moves(srw, small):
    # the reference moved to another fit-region point (as a fit moves it to
    # its current best estimate); the bars hold around it
    t_ref = np.array([0.004, -0.003, 0.002, 0.0, 0.2], np.float32)
    th = near_sm(4, 46) * FIT_SCALE + t_ref
    want = small.ref.neg2lnl_batch(th.astype(np.float64))
    assert np.max(np.abs(want - small.ref.neg2lnl(t_ref.astype(np.float64)))) <= 100.0
    try:
        small.lk.set_reference(t_ref)
        for p, tol in ((srw.SRW_FP32, 1e-4), (srw.SRW_FP16X3, 1e-3), (srw.SRW_BF16X3, 1e-3)):
            assert np.max(np.abs(small.lk.loglik(th, p) - want)) <= tol, p
    finally:
        small.lk.set_reference(np.zeros(5))


def test_given_event_numbers(srw):
    wl = small_workload(events=np.array([4.0e4, 5.0e3, 2.0e4]))
    c = JointCase(srw, wl)
    try:
        th = np.concatenate([np.zeros((1, 5), np.float32), near_sm(3, 47)])
        want = c.ref.neg2lnl_batch(th.astype(np.float64))
        assert np.max(np.abs(c.lk.loglik(th, srw.SRW_FP32) - want)) <= 1e-4
        assert c.lk.info()["lambda"] == 0.0
    finally:
        c.lk.close()


def test_grouped_with_a_conditional_configuration(srw, small):
    be7 = workloads.be7_line_workload()
    lk2 = srw.Likelihood(be7, workloads.load_counts(be7["name"]))
    try:
        th1, th2 = workloads.theta_box(200, 48), workloads.theta_box(37, 49)
        grp = srw.GroupedLikelihood([small.lk, lk2], [200, 37])
        try:
            for p in (srw.SRW_FP16X3, srw.SRW_BF16X3):
                grp.set_schedule(p, 0)  # 256-bin tiles everywhere, as the members' default
                got = grp.loglik(np.concatenate([th1, th2]), p)
                assert np.array_equal(got[:200], small.lk.loglik(th1, p)), p
                assert np.array_equal(got[200:], lk2.loglik(th2, p)), p
        finally:
            grp.close()
    finally:
        lk2.close()


def test_empty_component_histogram_is_rejected(srw):
    wl = small_workload()
    wl["hist"][1] = np.zeros_like(wl["hist"][1])
    with pytest.raises(srw.SrwError) as ei:
        srw.Likelihood(wl)
    assert ei.value.status == 1 and "no events" in str(ei.value)
