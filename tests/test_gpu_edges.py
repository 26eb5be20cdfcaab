"""Edge cases of the CUDA path against the oracle: ragged sizes, a single
point, masked and empty bins, a supplied baseline spectrum, midpoint binning,
the domain error, and device-pointer calls on a torch stream."""

import numpy as np
import pytest

import oracle as O
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def srw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2607_00488_gb300 as pkg
    return pkg


def small_workload(n_t=37, n_rec=29, seed=0):
    """Ragged sizes: no dimension a multiple of a tile."""
    rng = np.random.default_rng(seed)
    t_edges = np.concatenate([[0.0], np.sort(rng.uniform(0.0, 1.4, n_t - 1)), [1.4]])
    rec_edges = np.linspace(0.0, 1.4, n_rec + 1)
    r = workloads.solar.response_matrix(t_edges, rec_edges, res=0.06)
    src = [{"e": np.array([0.862]), "w": np.array([0.9]), "pee": np.array([0.55])},
           {"e": np.array([1.44, 0.3, 0.7]), "w": np.array([0.3, 1.2, 0.5]), "pee": np.array([0.5, 0.56, 0.54])}]
    bkg = rng.uniform(0.0, 30.0, (2, n_rec))
    wl = {"name": "ragged", "t_edges": t_edges, "rec_edges": rec_edges, "sources": src, "R": r, "bkg": bkg,
          "exposure": 5.0e3, "t_min": 1e-3, "sin2w": 0.23121, "f_tau": 0.5}
    return wl


def _oracle(wl, counts, mask=None, **kw):
    m = O.OracleModel.from_workload(wl, **kw)
    m.set_data(counts, wl["bkg"], mask)
    return m


def _asimov(wl, **kw):
    m = O.OracleModel.from_workload(wl, **kw)
    m.set_data(np.zeros(wl["R"].shape[0]), wl["bkg"])
    return workloads.poisson_counts(m.mu(np.zeros(5)), 3)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "fp16x3"])
def test_ragged_sizes_and_single_point(srw, prec):
    wl = small_workload()
    counts = _asimov(wl)
    ref = _oracle(wl, counts)
    th = np.concatenate([np.zeros((1, 5), np.float32), workloads.theta_box(130, 2, eps_max=0.01, mu_max=0.3)])
    with srw.Likelihood(wl, counts) as lk:
        got = lk.loglik(th, srw.PRECISIONS[prec])
        one = lk.loglik(th[5:6], srw.PRECISIONS[prec])
    want = ref.neg2lnl_batch(th.astype(np.float64))
    tol = 1e-4 if prec == "fp32" else 1e-3
    assert np.max(np.abs(got - want)) <= tol
    assert abs(one[0] - want[5]) <= tol


def test_mask_and_empty_bins(srw):
    wl = small_workload(seed=1)
    counts = _asimov(wl)
    counts[::4] = 0.0                      # bins with no events
    mask = np.ones(wl["R"].shape[0], np.uint8)
    mask[3:9] = 0                          # dead bins
    ref = _oracle(wl, counts, mask)
    th = np.concatenate([np.zeros((1, 5), np.float32), workloads.theta_box(7, 3, eps_max=0.02, mu_max=0.5)])
    with srw.Likelihood(wl, counts, mask=mask) as lk:
        for prec, tol in (("fp32", 1e-4), ("bf16x3", 1e-3), ("fp16x3", 1e-3)):
            got = lk.loglik(th, srw.PRECISIONS[prec])
            np.testing.assert_allclose(got, ref.neg2lnl_batch(th.astype(np.float64)), rtol=0, atol=tol)
        single = lk.loglik(th[2:3], srw.SRW_FP32)
        assert abs(single[0] - ref.neg2lnl(th[2].astype(np.float64))) <= 1e-4


def test_supplied_baseline_spectrum(srw):
    wl = small_workload(seed=2)
    base = O.OracleModel.from_workload(wl).e_sm * np.random.default_rng(4).uniform(0.9, 1.1, len(wl["t_edges"]) - 1)
    counts = _asimov(wl, e_true_sm=base)
    ref = _oracle(wl, counts, e_true_sm=base)
    th = workloads.theta_box(6, 5, eps_max=0.05, mu_max=1.0)
    with srw.Likelihood(wl, counts, e_true_sm=base) as lk:
        np.testing.assert_allclose(lk.spectrum(th[0], 1), ref.weighted_true(th[0].astype(np.float64)), rtol=1e-6)
        got = lk.loglik(th, srw.SRW_FP32)
    np.testing.assert_allclose(got, ref.neg2lnl_batch(th.astype(np.float64)), rtol=0, atol=1e-4)


def test_midpoint_binning(srw):
    wl = small_workload(seed=3)
    counts = _asimov(wl, midpoint=True)
    ref = _oracle(wl, counts, midpoint=True)
    th = workloads.theta_box(5, 6, eps_max=0.05, mu_max=1.0)
    with srw.Likelihood(wl, counts, midpoint=True) as lk:
        s = lk.spectrum(th[1], 0)
        want = ref.spectrum(th[1].astype(np.float64))
        big = want > 1e-4 * want.max()
        assert np.max(np.abs(s[big] / want[big] - 1)) <= 1e-6
        np.testing.assert_allclose(lk.basis(), O.coefficient_spectra(wl["sources"], wl["t_edges"], wl["t_min"],
                                                                     midpoint=True), rtol=1e-10,
                                   atol=1e-13 * np.abs(want).max())
        got = lk.loglik(th, srw.SRW_FP32)
    np.testing.assert_allclose(got, ref.neg2lnl_batch(th.astype(np.float64)), rtol=0, atol=1e-4)


def test_domain_error_gives_inf(srw):
    wl = small_workload(seed=5)
    wl["R"][7, :] = 0.0                   # a reconstructed bin nothing can reach
    wl["bkg"][:, 7] = 0.0
    counts = _asimov(wl)
    counts[7] = 3.0                        # ...but it holds events
    th = np.zeros((2, 5), np.float32)
    with srw.Likelihood(wl, counts) as lk:
        for prec in ("fp32", "bf16x3", "fp16x3"):
            assert np.all(np.isinf(lk.loglik(th, srw.PRECISIONS[prec])))
        assert np.isinf(lk.loglik(th[:1], srw.SRW_FP32)[0])
    assert O.neg2lnl(O.OracleModel.from_workload(wl).mu_sig(np.zeros(5)) + wl["bkg"].sum(0), counts) == np.inf


def test_device_pointers_on_torch_stream(srw):
    wl = workloads.be7_line_workload()
    counts = workloads.load_counts(wl["name"])
    th = np.concatenate([np.zeros((1, 5), np.float32), wl["theta"]])
    ref = _oracle(wl, counts)
    want = ref.neg2lnl_batch(th.astype(np.float64))
    s = torch.cuda.Stream()
    with srw.Likelihood(wl, counts) as lk, torch.cuda.stream(s):
        dth = torch.tensor(th, device="cuda")
        out = torch.empty(th.shape[0], dtype=torch.float64, device="cuda")
        lk.loglik(dth, srw.SRW_FP32, out=out, stream=s)
        lk.loglik(dth, srw.SRW_FP32, out=out, stream=s)  # replays the captured graph
        s.synchronize()
        got = out.cpu().numpy()
    mu = np.array([ref.mu(t.astype(np.float64)) for t in th])
    # far grid points: bounded by the rounding of the FP32 fold (see test_gpu_parity)
    bound = 1e-4 + 2 * 2.0 ** -22 * np.abs(mu - counts).sum(axis=1)
    assert np.all(np.abs(got - want) <= bound)


def test_bounded_wait_reports_timeout_and_context_survives(srw):
    # a wait on an mbarrier that nothing arrives on gives up after its limit
    import time
    t0 = time.perf_counter()
    st = srw.lib().srw_diag_wait_timeout(2000)  # 2 ms
    dt = time.perf_counter() - t0
    assert st == 6  # SRW_ETIMEOUT
    assert dt < 5.0
    # the context is still usable: a normal evaluation afterwards
    wl = workloads.be7_line_workload()
    with srw.Likelihood(wl, workloads.load_counts(wl["name"])) as lk:
        v = lk.loglik(np.zeros((2, 5), np.float32), srw.SRW_BF16X3)
    assert np.all(np.isfinite(v))


def test_single_point_bands_longer_than_a_stage(srw):
    """The banded single-point GEMV on rows whose nonzero bands range from a few
    hundred floats to more than one 4096-float ring stage (a band longer than a
    stage is cut into stage-sized segments, short bands share a stage): values
    equal the FP64 oracle's, and the bytes streamed are exactly the bands."""
    rng = np.random.default_rng(11)
    n_t, n_rec = 8001, 301
    t_edges = np.linspace(0.0, 1.4, n_t + 1)
    rec_edges = np.linspace(0.0, 1.4, n_rec + 1)
    wl = small_workload(seed=6)
    wl.update({"name": "long_bands", "t_edges": t_edges, "rec_edges": rec_edges,
               "R": workloads.solar.response_matrix(t_edges, rec_edges, res=0.06),
               "bkg": rng.uniform(0.0, 30.0, (2, n_rec))})
    lens = []
    for row in wl["R"]:
        nz = np.nonzero(row)[0]
        lens.append(nz[-1] + 1 - nz[0] if len(nz) else 0)
    assert max(lens) > 4096 and min(lens) < 2048  # bands cut across stages and bands that share one
    counts = _asimov(wl)
    ref = _oracle(wl, counts)
    th = np.concatenate([np.zeros((1, 5), np.float32), workloads.theta_box(3, 7, eps_max=0.05, mu_max=1.0)])
    with srw.Likelihood(wl, counts) as lk:
        ld = lk.info()["k_pad"]
        band = 0
        for row in wl["R"]:
            nz = np.nonzero(row)[0]
            lo = nz[0] // 4 * 4 if len(nz) else 0
            ln = min((nz[-1] + 1 - lo + 31) // 32 * 32, ld) if len(nz) else 32
            band += 4 * ln
        assert lk.gemv_work() == band
        for k in range(th.shape[0]):
            got = lk.loglik(th[k:k + 1], srw.SRW_FP32)[0]
            assert abs(got - ref.neg2lnl(th[k].astype(np.float64))) <= 1e-4, k


def test_non_finite_theta_fails_and_leaves_out_untouched(srw):
    """Host-buffer calls check theta for finiteness while the device works: a
    NaN or inf fails the call with SRW_EINVAL before anything is written to the
    caller's result buffer, and the handle stays usable."""
    wl = small_workload(seed=8)
    counts = _asimov(wl)
    ref = _oracle(wl, counts)
    th = workloads.theta_box(6, 9, eps_max=0.05, mu_max=1.0)
    with srw.Likelihood(wl, counts) as lk:
        for bad in (np.nan, np.inf):
            for prec in ("fp32", "bf16x3", "fp16x3"):
                for n in (1, th.shape[0]):
                    t = th[:n].copy()
                    t[n - 1, 2] = bad
                    out = np.full(n, 123.0)
                    with pytest.raises(srw.SrwError) as e:
                        lk.loglik(t, srw.PRECISIONS[prec], out=out)
                    assert e.value.status == srw.SRW_EINVAL
                    assert np.all(out == 123.0)
        got = lk.loglik(th, srw.SRW_FP32)
    np.testing.assert_allclose(got, ref.neg2lnl_batch(th.astype(np.float64)), rtol=0, atol=1e-4)


def test_single_point_many_rows_per_block(srw):
    """62,000 reconstructed bins of 4096 true bins: each GEMV block owns about
    420 rows next to a full 96 KB copy ring, so the per-row partial sums must
    stay compact in shared memory. The single-point call works and agrees with
    the batched FP32 fold (SIMT, another kernel) on the same points."""
    rng = np.random.default_rng(12)
    n_t, n_rec = 4096, 62000
    t_edges = np.linspace(0.0, 1.4, n_t + 1)
    rec_edges = np.linspace(0.0, 1.4, n_rec + 1)
    wl = small_workload(seed=9)
    wl.update({"name": "many_rows", "t_edges": t_edges, "rec_edges": rec_edges,
               "R": workloads.solar.response_matrix(t_edges, rec_edges, res=0.06),
               "bkg": rng.uniform(0.0, 0.5, (2, n_rec))})
    counts = workloads.poisson_counts(np.full(n_rec, 2.0), 13)
    th = np.concatenate([np.zeros((1, 5), np.float32), workloads.theta_box(2, 14, eps_max=0.05, mu_max=1.0)])
    with srw.Likelihood(wl, counts) as lk:
        batched = lk.loglik(th, srw.SRW_FP32)
        for k in range(th.shape[0]):
            single = lk.loglik(th[k:k + 1], srw.SRW_FP32)[0]
            assert np.isfinite(single)
            # two FP32 paths far from these flat pseudo-data: equal to ~1e-7 relative
            assert abs(single - batched[k]) <= 1e-3 + 1e-6 * abs(batched[k]), (k, single, batched[k])
