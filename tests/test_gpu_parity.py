"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Tolerances
* FP64 create-time coefficient spectra: 1e-10 relative.
* FP32 spectra (single-point kernels): per-bin relative error <= 1e-6.
* -2 ln L in the fit region (points near the reference point, where a fit
  or a confidence interval is decided): |d| <= 1e-4 for the FP32 paths and
  |d| <= 1e-3 for the BF16 hi+lo (3-product) path.
* -2 ln L everywhere: a fold whose per-bin results carry relative errors
  delta_j changes -2 ln L by about 2 sum_j (1 - n_j/mu_j) mu_j delta_j, so far
  from the data (mu - n large) the same per-bin precision gives a larger d.
  Every point must satisfy |d| <= tol + 2 * B with the measured budget
  B = 2 sum_j |1 - n_j/mu_j| |dmu_j| (dmu_j: the same path's per-bin error),
  i.e. the likelihood reduction adds no error of its own.
* BF16 single product: per-bin relative error <= 2 * 2^-8 (both operands are
  rounded to 8 significant bits).
* FP16 hi+lo split (SRW_FP16X3): each operand kept to ~2^-22 relative after
  its power-of-two scaling, so the fold error is set by the FP32 accumulation
  in tensor memory: 256 K-steps of 16 at 2^-24 each give ~1e-6 of the summed
  term magnitudes, which for box points (|W - W_ref| up to ~3 W) bounds the
  per-bin relative error by 5e-6.  -2 ln L: the same bars as the BF16 split.
"""

import numpy as np
import pytest

import oracle as O
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP32_BIN = 1e-6
TOL_FP32_LL = 1e-4
TOL_BF16X3_LL = 1e-3
TOL_FP16X3_LL = 1e-3
TOL_FP16X3_BIN = 5e-6
TOL_BF16_BIN = 2.0 * 2.0 ** -8


@pytest.fixture(scope="module")
def srw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2607_00488_gb300 as pkg
    return pkg


class Case:
    def __init__(self, srw, wl, with_data=True, mask=None, **kw):
        self.wl = wl
        self.counts = workloads.load_counts(wl["name"]) if with_data else None
        self.lk = srw.Likelihood(wl, self.counts, mask=mask, **kw)
        self.ref = O.OracleModel.from_workload(wl, **kw)
        if with_data:
            self.ref.set_data(self.counts, wl["bkg"], mask)


@pytest.fixture(scope="module")
def be7(srw):
    c = Case(srw, workloads.be7_line_workload())
    yield c
    c.lk.close()


@pytest.fixture(scope="module")
def solar(srw):
    c = Case(srw, workloads.solar_set_workload())
    yield c
    c.lk.close()


def near_sm(n, seed):
    """Points in the fit region around the SM reference: |eps| <= 0.02, mu_hat <= 0.5."""
    rng = np.random.default_rng(seed)
    th = np.zeros((n, 5), np.float32)
    th[:, :4] = rng.uniform(-0.02, 0.02, (n, 4))
    th[:, 4] = rng.uniform(0.0, 0.5, n)
    return th


def _rel_bins(got, want, floor):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    big = np.abs(want) > floor
    rel = np.abs(got[big] - want[big]) / np.abs(want[big])
    absd = np.abs(got[~big] - want[~big])
    return (rel.max() if rel.size else 0.0), (absd.max() if absd.size else 0.0)


def _budget(case, th, mu_sig_gpu, prec=None):
    """B = 2 sum_j |1 - n_j/mu_j| |dmu_j| from the measured per-bin errors;
    for the tensor-core precisions (FP32 epilogue) plus the bound of the
    epilogue's own FP32 evaluation of t_j = n_j ln(n_j/mu_j) + (mu_j - n_j):
    three roundings of 2^-24 on each part, doubled in -2 ln L."""
    mu = case.ref.mu(th.astype(np.float64))
    dmu = np.asarray(mu_sig_gpu, np.float64) - case.ref.mu_sig(th.astype(np.float64))
    n = case.counts
    on = mu > 0
    b = 2.0 * np.sum(np.abs(1.0 - n[on] / mu[on]) * np.abs(dmu[on]))
    if prec in ("bf16", "bf16x3", "fp16x3", 1, 2, 3):
        nlog = np.where(n[on] > 0, n[on] * np.abs(np.log(np.where(n[on] > 0, n[on], 1.0) / mu[on])), 0.0)
        b += 0.5 * 2.0 * 3.0 * 2.0 ** -24 * float(np.sum(nlog + np.abs(mu[on] - n[on])))  # halved: tests use 2 B
    return b


# ---------------------------------------------------------------- create-time basis
@pytest.mark.parametrize("name", ["be7", "solar"])
def test_coefficient_spectra_fp64(name, request):
    c = request.getfixturevalue(name)
    wl = c.wl
    want = O.coefficient_spectra(wl["sources"], wl["t_edges"], wl["t_min"], wl["sin2w"], wl["f_tau"])
    got = c.lk.basis()
    np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-13 * np.abs(want).max())


# ---------------------------------------------------------------- single-point spectra
def _thetas(n=3, seed=21):
    rng = np.random.default_rng(seed)
    th = [np.zeros(5, np.float32), np.array([0.1, -0.2, 0.05, 0.3, 2.0], np.float32)]
    for _ in range(n):
        th.append(np.concatenate([rng.uniform(-0.3, 0.3, 4), rng.uniform(0, 3, 1)]).astype(np.float32))
    return th


@pytest.mark.parametrize("name", ["be7", "solar"])
def test_spectrum_stage0_fp32(name, request):
    c = request.getfixturevalue(name)
    for th in _thetas():
        want = c.ref.spectrum(th.astype(np.float64))
        got = c.lk.spectrum(th, 0)
        rel, absd = _rel_bins(got, want, 1e-4 * np.abs(want).max())
        assert rel <= TOL_FP32_BIN, (th, rel)
        assert absd <= 1e-4 * TOL_FP32_BIN * np.abs(want).max()


@pytest.mark.parametrize("name", ["be7", "solar"])
def test_weighted_spectrum_stage1(name, request):
    c = request.getfixturevalue(name)
    for th in _thetas():
        want = c.ref.weighted_true(th.astype(np.float64))
        rel, _ = _rel_bins(c.lk.spectrum(th, 1), want, 1e-4 * np.abs(want).max())
        assert rel <= TOL_FP32_BIN, (th, rel)


def test_weights_identically_one_at_sm(be7):
    # W(theta = 0) is E_SM itself: S(0)/S_SM is exactly 1 on the device
    w0 = be7.lk.spectrum(np.zeros(5, np.float32), 1)
    rel, _ = _rel_bins(w0, be7.ref.e_sm, 1e-6 * be7.ref.e_sm.max())
    assert rel <= 1e-6
    np.testing.assert_array_equal(w0, be7.lk.spectrum(np.zeros(5, np.float32), 1))


@pytest.mark.parametrize("name", ["be7", "solar"])
def test_fold_stages(name, request):
    c = request.getfixturevalue(name)
    for th in _thetas(n=1):
        want = c.ref.mu_sig(th.astype(np.float64))
        rel, _ = _rel_bins(c.lk.spectrum(th, 2), want, 1e-3 * want.max())
        assert rel <= TOL_FP32_BIN, rel
        want_mu = c.ref.mu(th.astype(np.float64))
        rel, _ = _rel_bins(c.lk.spectrum(th, 3), want_mu, 1e-3 * want_mu.max())
        assert rel <= TOL_FP32_BIN, rel


# ---------------------------------------------------------------- likelihood, fit region
@pytest.mark.parametrize("name", ["be7", "solar"])
def test_loglik_fit_region_all_paths(srw, name, request):
    c = request.getfixturevalue(name)
    th = np.concatenate([np.zeros((1, 5), np.float32), near_sm(9, 3)])
    want = c.ref.neg2lnl_batch(th.astype(np.float64))
    single = np.array([c.lk.loglik(t[None, :], srw.SRW_FP32)[0] for t in th])
    points = c.lk.loglik_points(th)
    fp32 = c.lk.loglik(th, srw.SRW_FP32)
    x3 = c.lk.loglik(th, srw.SRW_BF16X3)
    h3 = c.lk.loglik(th, srw.SRW_FP16X3)
    print("fit region max |d|: fp32 %.2e bf16x3 %.2e fp16x3 %.2e" % (
        np.max(np.abs(fp32 - want)), np.max(np.abs(x3 - want)), np.max(np.abs(h3 - want))))
    assert np.max(np.abs(h3 - want)) <= TOL_FP16X3_LL, h3 - want
    assert np.max(np.abs(single - want)) <= TOL_FP32_LL, single - want
    assert np.max(np.abs(points - want)) <= TOL_FP32_LL, points - want
    assert np.max(np.abs(fp32 - want)) <= TOL_FP32_LL, fp32 - want
    assert np.max(np.abs(x3 - want)) <= TOL_BF16X3_LL, x3 - want


# ---------------------------------------------------------------- likelihood, everywhere
@pytest.mark.parametrize("name,prec,tol", [
    ("be7", "fp32", TOL_FP32_LL), ("be7", "bf16x3", TOL_BF16X3_LL),
    ("solar", "fp32", TOL_FP32_LL), ("solar", "bf16x3", TOL_BF16X3_LL),
    ("be7", "fp16x3", TOL_FP16X3_LL), ("solar", "fp16x3", TOL_FP16X3_LL),
])
def test_loglik_within_measured_budget(srw, name, prec, tol, request):
    c = request.getfixturevalue(name)
    th = np.concatenate([c.wl["theta"][:8], workloads.theta_box(5, 11)])
    p = srw.PRECISIONS[prec]
    got = c.lk.loglik(th, p)
    spectra = c.lk.spectrum_batch(th, p)
    for k in range(th.shape[0]):
        want = c.ref.neg2lnl(th[k].astype(np.float64))
        b = _budget(c, th[k], spectra[k], prec)
        assert abs(got[k] - want) <= tol + 2.0 * b, (k, got[k] - want, b)


def test_single_point_within_measured_budget(srw, solar):
    th = workloads.theta_box(4, 12)
    for t in th:
        got = solar.lk.loglik(t[None, :], srw.SRW_FP32)[0]
        want = solar.ref.neg2lnl(t.astype(np.float64))
        b = _budget(solar, t, solar.lk.spectrum(t, 2))
        assert abs(got - want) <= TOL_FP32_LL + 2.0 * b, (got - want, b)


# ---------------------------------------------------------------- batched spectra per bin
@pytest.mark.parametrize("prec,tol", [("fp32", TOL_FP32_BIN), ("bf16x3", 2e-5), ("bf16", TOL_BF16_BIN),
                                      ("fp16x3", TOL_FP16X3_BIN)])
def test_batched_spectra_per_bin(srw, solar, prec, tol):
    th = np.concatenate([np.zeros((1, 5), np.float32), workloads.theta_box(130, 13)])  # two point tiles, ragged
    got = solar.lk.spectrum_batch(th, srw.PRECISIONS[prec])
    for k in (0, 1, 64, 127, 128, 130):
        want = solar.ref.mu_sig(th[k].astype(np.float64))
        rel, _ = _rel_bins(got[k], want, 1e-3 * want.max())
        assert rel <= tol, (k, rel)


@pytest.mark.parametrize("prec,tol", [("bf16", TOL_BF16_BIN), ("fp16x3", TOL_FP16X3_BIN)])
def test_raw_fold_without_reference(srw, solar, prec, tol):
    # the reference point removed: all of W(theta) but its theta-independent
    # (nu_mu) part goes through the rounded operands (BF16: every product
    # rounded to 8 bits; FP16 split: scaled to the largest element of W, not
    # of a small deviation)
    th = workloads.theta_box(3, 14)
    try:
        solar.lk.set_reference(None)
        got = solar.lk.spectrum_batch(th, srw.PRECISIONS[prec])
    finally:
        solar.lk.set_reference(np.zeros(5))
    for k in range(3):
        want = solar.ref.mu_sig(th[k].astype(np.float64))
        rel, _ = _rel_bins(got[k], want, 1e-3 * want.max())
        assert rel <= tol, rel


def test_reference_point_moves(srw, be7):
    """A fit moves the fold's reference point to its current estimate; near
    it the split folds carry only the small deviation W(theta) - W_ref.  Data
    drawn at eps_L_ee = 0.1 (oracle expectation, Poisson, seed 9), reference
    point there, points in the fit region around it: the fit-region bars."""
    centre = np.array([0.1, 0.0, 0.0, 0.0, 0.0])
    m = O.OracleModel.from_workload(be7.wl)
    m.set_data(np.zeros(be7.wl["R"].shape[0]), be7.wl["bkg"])
    counts = workloads.poisson_counts(m.mu(centre), 9)
    m.set_data(counts, be7.wl["bkg"])
    th = near_sm(6, 5) + centre.astype(np.float32)
    want = m.neg2lnl_batch(th.astype(np.float64))
    with srw.Likelihood(be7.wl, counts) as lk:
        lk.set_reference(centre)
        x3 = lk.loglik(th, srw.SRW_BF16X3)
        h3 = lk.loglik(th, srw.SRW_FP16X3)
        fp32 = lk.loglik(th, srw.SRW_FP32)
    assert np.max(np.abs(x3 - want)) <= TOL_BF16X3_LL, x3 - want
    assert np.max(np.abs(h3 - want)) <= TOL_FP16X3_LL, h3 - want
    assert np.max(np.abs(fp32 - want)) <= TOL_FP32_LL, fp32 - want


def test_batched_agrees_with_single_point_path(srw, solar):
    th = np.concatenate([np.zeros((1, 5), np.float32), near_sm(63, 6)])
    single = solar.lk.loglik_points(th)
    batched = solar.lk.loglik(th, srw.SRW_FP32)
    assert np.max(np.abs(single - batched)) <= TOL_FP32_LL


@pytest.mark.parametrize("prec,tol", [("fp16x3", TOL_FP16X3_LL), ("bf16x3", TOL_BF16X3_LL)])
def test_full_scan_sampled(srw, solar, prec, tol):
    # the benchmark's launch: 65,536 points in one call, sampled against the oracle
    th = workloads.theta_box(65536, 3)
    th[:4] = near_sm(4, 8)
    dev = torch.device("cuda")
    out = torch.empty(65536, dtype=torch.float64, device=dev)
    p = srw.PRECISIONS[prec]
    solar.lk.loglik(torch.tensor(th, device=dev), p, out=out)
    got = out.cpu().numpy()
    assert np.all(np.isfinite(got))
    idx = [0, 1, 2, 3, 127, 65535]
    for k in idx:
        want = solar.ref.neg2lnl(th[k].astype(np.float64))
        if k < 4:
            assert abs(got[k] - want) <= tol
        else:
            b = _budget(solar, th[k], solar.lk.spectrum_batch(th[k:k + 1], p)[0], prec)
            assert abs(got[k] - want) <= tol + 2.0 * b


# ---------------------------------------------------------------- exact rank-8 evaluator
@pytest.mark.parametrize("name", ["be7", "solar"])
def test_linear_evaluator_matches_oracle(srw, name, request):
    # mu = mu_ref + b + M (c - c_ref) with M in FP32: per-bin errors of 2^-24
    # relative of mu_ref + b (carried as n - mu_ref - b and n + mu_ref + b) and of
    # sum_b |M_jb dc_b|; fit region: the FP32 bar; everywhere: |d| <= tol + 2 B
    # with B = 2 sum_j |1 - n_j / mu_j| (1.2e-7 mu_j + 1.2e-7 sum_b |M_jb dc_b|).
    c = request.getfixturevalue(name)
    wl = c.wl
    fit = np.concatenate([np.zeros((1, 5), np.float32), near_sm(7, 31)])
    box = workloads.theta_box(6, 32)
    th = np.concatenate([fit, box])
    got = c.lk.loglik_linear(th)
    B = O.coefficient_spectra(wl["sources"], wl["t_edges"], wl["t_min"], wl["sin2w"], wl["f_tau"])
    s_sm, e_sm = c.ref.s_sm, c.ref.e_sm
    shat = np.where(s_sm > 0, B * (e_sm / np.where(s_sm > 0, s_sm, 1.0)), 0.0)
    M = np.asarray(wl["R"], np.float64) @ shat.T  # [n_rec, 8]
    c0 = O.coupling_coefficients(np.zeros(5), wl["sin2w"])
    for k, t in enumerate(th):
        t64 = t.astype(np.float64)
        want = c.ref.neg2lnl(t64)
        if k < fit.shape[0]:
            assert abs(got[k] - want) <= TOL_FP32_LL, (k, got[k] - want)
        mu = c.ref.mu(t64)
        dc = O.coupling_coefficients(t64, wl["sin2w"]) - c0
        on = mu > 0
        eps = 1.2e-7 * mu + 1.2e-7 * np.abs(M * dc).sum(axis=1)
        budget = 2.0 * np.sum(np.abs(1.0 - c.counts[on] / mu[on]) * eps[on])
        assert abs(got[k] - want) <= TOL_FP32_LL + 2.0 * budget, (k, got[k] - want, budget)


def test_linear_evaluator_equals_the_folds(srw, solar):
    # two FP32 evaluations of the same quantity, each checked against the
    # oracle above; at 1e5 events each stays within ~2e-4 of it in the fit
    # region (largest seen: 1.7e-4), so their difference stays within 4e-4
    # there, and within a relative 1e-6 far from the data (per-bin errors
    # ~1e-7 times the residual sums)
    fit = near_sm(100, 33)
    box = workloads.theta_box(300, 34)
    for th, rel in ((fit, 0.0), (box, 1e-6)):
        lin = solar.lk.loglik_linear(th)
        simt = solar.lk.loglik(th, srw.SRW_FP32)
        tol = 4e-4 + rel * np.abs(simt)
        assert np.all(np.abs(lin - simt) <= tol), np.max(np.abs(lin - simt) / tol)


@pytest.mark.parametrize("name", ["be7", "solar"])
def test_linear_gradient_matches_finite_differences(srw, name, request):
    c = request.getfixturevalue(name)
    th = np.concatenate([near_sm(2, 35), workloads.theta_box(2, 36)]).astype(np.float64)
    _, grad = c.lk.loglik_linear(th.astype(np.float32), grad=True)
    h = 1e-5
    for k, t in enumerate(th):
        t = t.astype(np.float32).astype(np.float64)  # the point the GPU evaluated
        fd = np.zeros(5)
        for a in range(5):
            e = np.zeros(5)
            e[a] = h
            fd[a] = (c.ref.neg2lnl(t + e) - c.ref.neg2lnl(t - e)) / (2 * h)
        scale = np.max(np.abs(fd)) + 1.0
        np.testing.assert_allclose(grad[k], fd, rtol=2e-3, atol=2e-4 * scale)


# ---------------------------------------------------------------- profiled signal normalisation
@pytest.mark.parametrize("name", ["be7", "solar"])
def test_profiled_normalisation_matches_oracle(srw, name, request):
    # same FP32 evaluation as the rank-8 evaluator at alpha-hat: the fit-region
    # bar of two FP32 paths (4e-4) near the data, 1e-6 relative far from it;
    # alpha-hat to 1e-4 (the objective is flat in alpha at its minimum)
    c = request.getfixturevalue(name)
    th = np.concatenate([near_sm(3, 37), workloads.theta_box(2, 38)])
    for sigma in (0.0, 0.05):
        got, alpha = c.lk.loglik_profiled(th, sigma)
        for k, t in enumerate(th):
            want, a_want = O.profiled_neg2lnl(c.ref.mu_sig(t.astype(np.float64)), c.ref.bkg_sum, c.counts, sigma)
            assert abs(got[k] - want) <= 4e-4 + 1e-6 * abs(want), (sigma, k, got[k] - want)
            assert abs(alpha[k] - a_want) <= 1e-4 * max(1.0, a_want), (sigma, k, alpha[k], a_want)


def test_profiled_asimov_recovers_the_normalisation(srw, be7):
    from oracle.mlp_oracle import data_constant
    theta0 = np.array([0.02, -0.01, 0.0, 0.0, 0.3])
    counts = 1.3 * be7.ref.mu_sig(theta0) + be7.ref.bkg_sum  # Asimov data, oracle expectation
    with srw.Likelihood(be7.wl, counts) as lk:
        v, a = lk.loglik_profiled(theta0[None, :].astype(np.float32))
    assert a[0] == pytest.approx(1.3, rel=1e-5)
    assert v[0] == pytest.approx(data_constant(counts), abs=1e-3)


# ---------------------------------------------------------------- skipped zero blocks
def _split_nonzero(R, f16):
    """Host emulation of the response splits: which elements have a nonzero hi
    or lo part (FP16: rows scaled by 2^(14 - e), e the binary exponent of the
    row maximum; BF16: unscaled)."""
    from workloads.mlp import round_to_bf16
    R = np.asarray(R, np.float32)
    if f16:
        m = np.abs(R).max(axis=1)
        e = np.frexp(m)[1]
        x = R * np.ldexp(np.float32(1.0), 14 - e)[:, None].astype(np.float32)
        hi = x.astype(np.float16)
        lo = (x - hi.astype(np.float32)).astype(np.float16)
    else:
        hi = round_to_bf16(R)
        lo = round_to_bf16(R - hi)
    return (hi != 0) | (lo != 0)


def _block_fraction(nz, bn, bk=64):
    n_rec, n_t = nz.shape
    n_kb = -(-n_t // bk)
    used = 0
    for r0 in range(0, n_rec, bn):
        cols = np.nonzero(nz[r0:r0 + bn].any(axis=0))[0]
        used += (cols.max() // bk - cols.min() // bk + 1) if cols.size else 1
    return used / (-(-n_rec // bn) * n_kb)


@pytest.mark.parametrize("prec,f16", [("fp16x3", True), ("bf16x3", False)])
@pytest.mark.parametrize("bn", [128, 256])
def test_skipped_blocks_are_the_zero_blocks(srw, solar, prec, f16, bn):
    # the (rec tile, K block) pairs the tensor-core fold executes are exactly
    # the ranges that hold nonzero split elements (index work: exact)
    got = solar.lk.fold_work(srw.PRECISIONS[prec], bn)
    want = _block_fraction(_split_nonzero(solar.wl["R"], f16), bn)
    assert got == pytest.approx(want, abs=1e-12), (got, want)
    assert got < 0.7  # the banded response leaves most blocks empty


# ---------------------------------------------------------------- the benchmark's parity points
def test_bench_fit_region_points_all_paths(srw, solar):
    """The benchmark's own fit-region sample (8 points, seed 99): the bars of
    the metric hold there for every path.  Point 7 lies Delta(-2 ln L) ~ 220
    from the data, where systematic per-bin errors of the fold reach -2 ln L
    most strongly."""
    th = workloads.fit_region_points(8)
    want = solar.ref.neg2lnl_batch(th.astype(np.float64))
    single = np.array([solar.lk.loglik(t[None, :], srw.SRW_FP32)[0] for t in th])
    got = {"single": single, "fp32": solar.lk.loglik(th, srw.SRW_FP32),
           "bf16x3": solar.lk.loglik(th, srw.SRW_BF16X3), "fp16x3": solar.lk.loglik(th, srw.SRW_FP16X3),
           "linear": solar.lk.loglik_linear(th)}
    d = {k: float(np.max(np.abs(v - want))) for k, v in got.items()}
    print("bench fit-region max |d|:", d)
    for k in ("single", "fp32", "linear"):
        assert d[k] <= TOL_FP32_LL, (k, d)
    assert d["bf16x3"] <= TOL_BF16X3_LL, d
    assert d["fp16x3"] <= TOL_FP16X3_LL, d


@pytest.mark.parametrize("prec,tol", [("fp32", TOL_FP32_LL), ("bf16x3", TOL_BF16X3_LL), ("fp16x3", TOL_FP16X3_LL)])
def test_bench_box_points_within_budget(srw, solar, prec, tol):
    """The benchmark's box sample (12 evenly spaced points of the 65,536-point
    batch): far from the data the absolute bar does not apply; every point
    meets |d| <= tol + 2 B with the measured per-bin budget B."""
    th = workloads.box_sample(65536, 12, 3)
    p = srw.PRECISIONS[prec]
    got = solar.lk.loglik(th, p)
    spectra = solar.lk.spectrum_batch(th, p)
    for k in range(th.shape[0]):
        want = solar.ref.neg2lnl(th[k].astype(np.float64))
        b = _budget(solar, th[k], spectra[k], prec)
        assert abs(got[k] - want) <= tol + 2.0 * b, (k, got[k] - want, b)


# ---------------------------------------------------------------- fold configurations
def test_fold_candidates_are_bitwise_equal(srw, solar):
    """Every autotuner candidate (tile width, K block, pipeline depth)
    accumulates every output element from the same updates in the same order
    (the K direction is fixed per 256 rows; blocks one candidate runs and
    another skips add exact zeros): the folded spectra are bitwise equal,
    -2 ln L equal up to the order of the per-tile partial sums."""
    th = np.concatenate([np.zeros((1, 5), np.float32), workloads.theta_box(200, 15)])
    cfgs = srw.srw_fold_configs()
    assert len(cfgs) >= 2
    for prec in (srw.SRW_BF16, srw.SRW_BF16X3, srw.SRW_FP16X3):
        ref = None
        for i, tile, k_block, stages in cfgs:
            solar.lk.set_fold_config(prec, i)
            got = (solar.lk.spectrum_batch(th, prec), solar.lk.loglik(th, prec))
            if ref is None:
                ref = got
                continue
            np.testing.assert_array_equal(got[0], ref[0], err_msg="candidate %d" % i)
            np.testing.assert_allclose(got[1], ref[1], rtol=1e-12, atol=1e-9, err_msg="candidate %d" % i)
        solar.lk.set_fold_config(prec, 0)


def _band_bytes(R, ld):
    """Host recomputation of the GEMV's streamed columns: per row the first
    nonzero column rounded down to 4 floats, the length rounded up to 32 floats
    and kept inside the padded row; an all-zero row keeps 32."""
    total = 0
    for row in np.asarray(R, np.float32):
        nz = np.nonzero(row)[0]
        if nz.size == 0:
            total += 32
            continue
        lo = nz[0] // 4 * 4
        total += min(ld, -(-(nz[-1] + 1 - lo) // 32) * 32)
    return 4 * total


@pytest.mark.parametrize("name", ["be7", "solar"])
def test_gemv_streams_the_nonzero_bands(srw, name, request):
    c = request.getfixturevalue(name)
    ld = c.lk.info()["k_pad"]
    assert c.lk.gemv_work() == _band_bytes(c.wl["R"], ld)
    assert c.lk.gemv_work() < 4 * c.wl["R"].size  # the banded response leaves part of every row empty
