"""Failure paths on the GPU, made to run by host-side fault injection.

Nothing here faults, traps or hangs the GPU.  An injected allocation or
launch failure is reported by the host code without the allocation or with
the launch's status replaced; an injected timeout makes one wait of a fold
wait on an mbarrier that nothing arrives on, with a 1 ms limit, after which
the kernel takes its ordinary abort path.  Each test checks the status the
call returns, the values it leaves (NaN for points a timed-out fold could not
finish) and that the next call on the same handle computes the oracle's
value again.
"""

import numpy as np
import pytest

import oracle as O
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ENOMEM, ECUDA, ETIMEOUT = 2, 3, 6


@pytest.fixture(scope="module")
def srw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2607_00488_gb300 as pkg
    pkg.srw_fault_inject("none")
    yield pkg
    pkg.srw_fault_inject("none")


@pytest.fixture(scope="module")
def case(srw):
    wl = workloads.be7_line_workload()
    counts = workloads.load_counts(wl["name"])
    ref = O.OracleModel.from_workload(wl)
    ref.set_data(counts, wl["bkg"])
    lk = srw.Likelihood(wl, counts)
    th = workloads.theta_box(300, 11, eps_max=0.02, mu_max=0.5)
    want = ref.neg2lnl_batch(th.astype(np.float64))
    yield wl, counts, lk, th, want
    lk.close()


def _ok(lk, th, want, prec):
    got = lk.loglik(th, prec)
    assert np.max(np.abs(got - want)) <= (1e-4 if prec == 0 else 1e-3)


def test_allocation_failure_in_create(srw, case):
    wl, counts, _, th, want = case
    srw.srw_fault_inject("alloc", 5)
    with pytest.raises(srw.SrwError) as ei:
        srw.Likelihood(wl, counts)
    assert ei.value.status == ENOMEM
    assert srw.srw_fault_pending() == 0
    with srw.Likelihood(wl, counts) as lk:  # nothing left behind: a new handle works
        _ok(lk, th[:20], want[:20], srw.SRW_FP16X3)


def test_allocation_failure_in_a_call_leaves_the_handle_usable(srw, case):
    _, _, lk, th, want = case
    big = np.concatenate([th] * 40)  # grows the staging buffers: the call allocates
    srw.srw_fault_inject("alloc")
    with pytest.raises(srw.SrwError) as ei:
        lk.loglik(big, srw.SRW_FP16X3)
    assert ei.value.status == ENOMEM
    got = lk.loglik(big, srw.SRW_FP16X3)
    assert np.max(np.abs(got - np.concatenate([want] * 40))) <= 1e-3


def test_set_data_after_a_failed_first_set_data(srw, case):
    # the first srw_set_data of a handle allocates its data buffers; when the
    # second of them fails, the next srw_set_data allocates the rest
    wl, counts, _, th, want = case
    with srw.Likelihood(wl) as lk:
        srw.srw_fault_inject("alloc", 1)
        with pytest.raises(srw.SrwError) as ei:
            srw.srw_set_data(lk.handle, counts, wl["bkg"])
        assert ei.value.status == ENOMEM
        with pytest.raises(srw.SrwError) as ei:
            lk.loglik(th[:4], srw.SRW_FP32)
        assert ei.value.status == 4  # SRW_ENODATA: no data yet
        srw.srw_set_data(lk.handle, counts, wl["bkg"])
        _ok(lk, th[:20], want[:20], srw.SRW_FP32)
        _ok(lk, th[:20], want[:20], srw.SRW_FP16X3)


def test_a_failed_growth_then_a_call_that_fits_the_old_size(srw, case):
    # the failed call freed the old staging buffers before its allocation
    # failed: a later call that fits the old capacity must allocate again
    _, _, lk, th, want = case
    lk.loglik(np.concatenate([th] * 2), srw.SRW_FP16X3)  # some capacity exists
    srw.srw_fault_inject("alloc")
    with pytest.raises(srw.SrwError) as ei:
        lk.loglik(np.concatenate([th] * 200), srw.SRW_FP16X3)  # grows the staging buffers
    assert ei.value.status == ENOMEM
    _ok(lk, th[:20], want[:20], srw.SRW_FP16X3)
    _ok(lk, th[:1], want[:1], srw.SRW_FP32)


@pytest.mark.parametrize("prec", [0, 2, 3])
def test_launch_failure_is_reported_and_not_cached(srw, case, prec):
    _, _, lk, th, want = case
    n = 64 + prec  # a call signature without a cached graph
    srw.srw_fault_inject("launch")
    with pytest.raises(srw.SrwError) as ei:
        lk.loglik(th[:n], prec)
    assert ei.value.status == ECUDA
    _ok(lk, th[:n], want[:n], prec)  # the discarded capture is not replayed


@pytest.mark.parametrize("prec", [0, 2, 3])
def test_timeout_host_call_reports_etimeout(srw, case, prec):
    _, _, lk, th, want = case
    n = 1 if prec == 0 else 200 + prec  # FP32: the single-point GEMV
    srw.srw_fault_inject("timeout")
    with pytest.raises(srw.SrwError) as ei:
        lk.loglik(th[:n], prec)
    assert ei.value.status == ETIMEOUT
    assert srw.srw_fault_pending() == 0
    _ok(lk, th[:n], want[:n], prec)  # the graph of the faulted call was not cached


@pytest.mark.parametrize("prec", [0, 3])
def test_timeout_device_call_gives_nan_then_check_reports_it(srw, case, prec):
    _, _, lk, th, want = case
    n = 1 if prec == 0 else 260
    dev = torch.device("cuda")
    t = torch.from_numpy(th[:n]).to(dev)
    out = torch.zeros(n, dtype=torch.float64, device=dev)
    srw.srw_fault_inject("timeout")
    lk.loglik(t, prec, out=out)  # asynchronous: no status yet
    got = out.cpu().numpy()
    bad = np.isnan(got)
    assert bad.any()  # the points of the items the aborted block held
    assert np.max(np.abs(got[~bad] - want[:n][~bad]), initial=0.0) <= (1e-4 if prec == 0 else 1e-3)
    with pytest.raises(srw.SrwError) as ei:
        lk.check()
    assert ei.value.status == ETIMEOUT
    lk.check()  # read and cleared
    lk.loglik(t, prec, out=out)
    got = out.cpu().numpy()
    assert np.max(np.abs(got - want[:n])) <= (1e-4 if prec == 0 else 1e-3)
    lk.check()


def test_timeout_in_a_grouped_launch(srw, case):
    wl, counts, lk, th, want = case
    with srw.Likelihood(wl, counts) as lk2:
        grp = srw.GroupedLikelihood([lk, lk2], [150, 90])
        tt = np.concatenate([th[:150], th[:90]])
        ww = np.concatenate([want[:150], want[:90]])
        srw.srw_fault_inject("timeout")
        with pytest.raises(srw.SrwError) as ei:
            grp.loglik(tt, srw.SRW_FP16X3)
        assert ei.value.status == ETIMEOUT
        got = grp.loglik(tt, srw.SRW_FP16X3)
        assert np.max(np.abs(got - ww)) <= 1e-3
        grp.close()


def test_surrogate_calls_fail_cleanly_on_allocation_faults(srw, case):
    # an allocation that fails part-way through a call's own buffers returns
    # the status, frees what the call had allocated, and the next call gives
    # the same values
    from workloads.mlp import BOX_CENTRE, BOX_HALF, init_weights
    _, _, lk, _, _ = case
    with srw.Surrogate(lk, init_weights(128, seed=3), BOX_CENTRE, BOX_HALF) as sg:
        th = sg.sobol(0, 1000)
        want = sg.loglik(th)
        for skip in (0, 1):  # the first or the second of the call's two buffers
            srw.srw_fault_inject("alloc", skip)
            with pytest.raises(srw.SrwError) as ei:
                sg.loglik(th)
            assert ei.value.status in (ENOMEM, ECUDA)
            assert srw.srw_fault_pending() == 0
        np.testing.assert_array_equal(sg.loglik(th), want)
        ref = sg.scan_exact(4096)
        for skip in (0, 2):  # the first or the third of the scan's four buffers
            srw.srw_fault_inject("alloc", skip)
            with pytest.raises(srw.SrwError):
                sg.scan_exact(4096)
            assert srw.srw_fault_pending() == 0
        again = sg.scan_exact(4096)
        assert again["best_value"] == ref["best_value"] and again["best_index"] == ref["best_index"]
