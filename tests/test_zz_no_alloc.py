"""The allocation-free single-point entry point.

Some callers cannot allocate device memory themselves (code running inside
another framework's memory manager, which owns every device allocation, or
code that must not call cudaMalloc/cudaFree because those calls can
synchronise the device).  srw_loglik_point_noalloc serves them: the caller
passes every input and the output as device memory, and the kernels' scratch
is a fixed static device array inside the library.  These tests call it
through the C ABI and check it

* against the existing single-point entry point that performs the same
  arithmetic (srw_loglik_points: the weighted spectrum from the cross-section
  integrals, then the fold, with the reference point disabled so that both
  fold W directly), twice in a row, since consecutive calls share the
  scratch array; with and without a mask;
* against the FP64 oracle's fold and -2 ln L on the 2048-bin solar set and
  on a response whose rows span more than one 4096-float chunk (ld = 4160);
* on a stream other than the default one;
* and that a fold whose device wait times out (host-side fault injection)
  leaves NaN in out, never a finite wrong value.
"""

import numpy as np
import pytest

import oracle as O
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP32_LL = 1e-4


@pytest.fixture(scope="module")
def srw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2607_00488_gb300 as pkg
    return pkg


def _device_R(wl, ld, dev):
    n_rec, n_t = wl["R"].shape
    R = torch.zeros((n_rec, ld), dtype=torch.float32, device=dev)
    R[:, :n_t] = torch.from_numpy(wl["R"]).to(dev)
    return R


def _oracle_value(R, W, counts, bkg, mask=None):
    """-2 ln L of the FP64 oracle for the same FP32 inputs (fold, expectation, Poisson)."""
    mu = O.expected_counts(O.fold(np.asarray(R, np.float64), np.asarray(W, np.float64)), bkg, mask)
    return O.neg2lnl(mu, counts, mask)


def _noalloc(srw, R, W, c, b, mask=None, stream=None):
    out = torch.full((1,), float("nan"), dtype=torch.float64, device=R.device)
    srw.srw_loglik_point_noalloc(R, W, c, out, bkg=b, mask=mask, stream=stream)
    if stream is not None:
        stream.synchronize()
    torch.cuda.synchronize()
    return out.item()


@pytest.mark.parametrize("masked", [False, True])
def test_no_alloc_entry_point_matches_loglik(srw, masked):
    wl = workloads.be7_line_workload()
    counts = workloads.load_counts(wl["name"])
    dev = torch.device("cuda")
    mask = None
    if masked:
        mask = np.ones(wl["R"].shape[0], np.uint8)
        mask[:9] = 0
        mask[60:64] = 0
    with srw.Likelihood(wl, counts, mask=mask) as lk:
        lk.set_reference(None)
        ld = lk.info()["k_pad"]
        R = _device_R(wl, ld, dev)
        c = torch.from_numpy(counts).to(dev)
        b = torch.from_numpy(wl["bkg"].sum(axis=0)).to(dev)
        m = torch.from_numpy(mask).to(dev) if masked else None
        thetas = [np.zeros(5, np.float32), np.array([0.01, -0.015, 0.005, 0.0, 0.3], np.float32)]
        for th in thetas:
            W = torch.zeros(ld, dtype=torch.float32, device=dev)
            lk.spectrum(torch.from_numpy(th).to(dev), 1, out=W)
            want = lk.loglik_points(th[None, :])[0]
            ref = _oracle_value(wl["R"], W.cpu().numpy()[: wl["R"].shape[1]], counts, wl["bkg"].sum(axis=0), mask)
            for _ in range(2):
                got = _noalloc(srw, R, W, c, b, m)
                assert abs(got - want) <= TOL_FP32_LL, (got, want)
                assert abs(got - ref) <= TOL_FP32_LL, (got, ref)


def test_no_alloc_solar_set_against_the_oracle(srw):
    """The 2048-bin solar set, the size the scratch limits and the fold's
    shared memory are set for, on a non-default stream."""
    wl = workloads.solar_set_workload()
    counts = workloads.load_counts(wl["name"])
    dev = torch.device("cuda")
    ref = O.OracleModel.from_workload(wl)
    n_rec, n_t = wl["R"].shape
    ld = (n_t + 63) // 64 * 64
    R = _device_R(wl, ld, dev)
    c = torch.from_numpy(counts).to(dev)
    bsum = wl["bkg"].sum(axis=0)
    b = torch.from_numpy(bsum).to(dev)
    stream = torch.cuda.Stream()
    for th in (np.zeros(5), np.array([0.01, -0.01, 0.0, 0.005, 0.4])):
        w = np.zeros(ld, np.float32)
        w[:n_t] = ref.weighted_true(th)
        W = torch.from_numpy(w).to(dev)
        want = _oracle_value(wl["R"], w[:n_t], counts, bsum)
        for _ in range(2):
            got = _noalloc(srw, R, W, c, b, stream=stream)
            assert abs(got - want) <= TOL_FP32_LL, (got, want)


def test_no_alloc_rows_longer_than_one_chunk(srw):
    """ld = 4160: each row spans two of the fold's 4096-float chunks, the
    second one ragged (64 floats)."""
    rng = np.random.default_rng(7)
    n_rec, ld = 512, 4160
    # banded response with a long one-sided tail, rows normalised to 0.9
    i = np.arange(ld)[None, :]
    j = np.arange(n_rec)[:, None] * (ld / n_rec)
    r = np.exp(-0.5 * ((i - j) / 40.0) ** 2) + 1e-3 * np.exp(-np.abs(i - j) / 300.0) * (i > j)
    r *= rng.uniform(0.99, 1.01, r.shape)
    r = (0.9 * r / r.sum(axis=0, keepdims=True)).astype(np.float32)
    w = rng.uniform(50.0, 150.0, ld).astype(np.float32)
    mu = r.astype(np.float64) @ w.astype(np.float64)
    bkg = np.full(n_rec, 5.0)
    counts = workloads.poisson_counts(mu + bkg, 8)
    mask = (rng.uniform(size=n_rec) > 0.05).astype(np.uint8)
    dev = torch.device("cuda")
    R, W = torch.from_numpy(r).to(dev), torch.from_numpy(w).to(dev)
    c, b, m = (torch.from_numpy(x).to(dev) for x in (counts, bkg, mask))
    for msk, mt in ((None, None), (mask, m)):
        want = _oracle_value(r, w, counts, bkg, msk)
        for _ in range(2):
            got = _noalloc(srw, R, W, c, b, mt)
            assert abs(got - want) <= TOL_FP32_LL, (got, want)


def test_no_alloc_timeout_gives_nan(srw):
    """A device wait of the fold that expires (forced by host-side fault
    injection: it waits on an mbarrier nothing arrives on, for 1 ms) makes the
    value NaN; the next call computes normally."""
    wl = workloads.be7_line_workload()
    counts = workloads.load_counts(wl["name"])
    dev = torch.device("cuda")
    ref = O.OracleModel.from_workload(wl)
    n_rec, n_t = wl["R"].shape
    ld = (n_t + 63) // 64 * 64
    R = _device_R(wl, ld, dev)
    w = np.zeros(ld, np.float32)
    w[:n_t] = ref.weighted_true(np.zeros(5))
    W = torch.from_numpy(w).to(dev)
    c = torch.from_numpy(counts).to(dev)
    bsum = wl["bkg"].sum(axis=0)
    b = torch.from_numpy(bsum).to(dev)
    srw.srw_fault_inject("timeout")
    try:
        assert np.isnan(_noalloc(srw, R, W, c, b))
    finally:
        srw.srw_fault_inject("none")
    want = _oracle_value(wl["R"], w[:n_t], counts, bsum)
    assert abs(_noalloc(srw, R, W, c, b) - want) <= TOL_FP32_LL


def test_no_alloc_rejects_oversized_input(srw):
    dev = torch.device("cuda")
    R = torch.zeros((70000, 64), dtype=torch.float32, device=dev)  # beyond the 65536-bin limit
    W = torch.zeros(64, dtype=torch.float32, device=dev)
    c = torch.zeros(70000, dtype=torch.float64, device=dev)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(srw.SrwError) as ei:
        srw.srw_loglik_point_noalloc(R, W, c, out)
    assert ei.value.status == 1
