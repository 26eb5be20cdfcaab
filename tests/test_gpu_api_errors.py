"""Argument errors of the C entry points, called through ctypes below the
Python binding's own checks: each bad argument returns its documented
status (SRW_EINVAL, SRW_ENODATA) before any device work, and the handle
stays usable afterwards (a valid call then matches the oracle)."""

import ctypes

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


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def test_entry_points_reject_bad_arguments(srw, be7_workload):
    from paper_2607_00488_gb300 import srw as B
    L = B.lib()
    wl = be7_workload
    th = np.zeros((2, 5), np.float32)
    out = np.zeros(2, np.float64)
    spec = np.zeros(wl["R"].shape[1], np.float32)
    with srw.Likelihood(wl) as lk:  # no data yet
        h = lk.handle
        assert L.srw_loglik(h, _p(th), 2, _p(out), B.SRW_HOST, B.SRW_FP32, None) == B.SRW_ENODATA
        assert L.srw_spectrum(h, _p(th), 3, _p(spec), B.SRW_HOST, None) == B.SRW_ENODATA
        counts = workloads.load_counts(wl["name"])
        B.srw_set_data(h, counts, wl["bkg"])
        cases = [
            ("NULL handle", L.srw_loglik(None, _p(th), 2, _p(out), B.SRW_HOST, B.SRW_FP32, None)),
            ("NULL theta", L.srw_loglik(h, None, 2, _p(out), B.SRW_HOST, B.SRW_FP32, None)),
            ("NULL out", L.srw_loglik(h, _p(th), 2, None, B.SRW_HOST, B.SRW_FP32, None)),
            ("P = 0", L.srw_loglik(h, _p(th), 0, _p(out), B.SRW_HOST, B.SRW_FP32, None)),
            ("P < 0", L.srw_loglik(h, _p(th), -3, _p(out), B.SRW_HOST, B.SRW_FP32, None)),
            ("precision", L.srw_loglik(h, _p(th), 2, _p(out), B.SRW_HOST, 7, None)),
            ("where", L.srw_loglik(h, _p(th), 2, _p(out), 5, B.SRW_FP32, None)),
            ("points where", L.srw_loglik_points(h, _p(th), 2, _p(out), 5, None)),
            ("spectrum stage", L.srw_spectrum(h, _p(th), 4, _p(spec), B.SRW_HOST, None)),
            ("spectrum where", L.srw_spectrum(h, _p(th), 1, _p(spec), 5, None)),
            ("batch where", L.srw_spectrum_batch(h, _p(th), 2, _p(spec), 5, B.SRW_FP32, None)),
            ("batch P", L.srw_spectrum_batch(h, _p(th), 0, _p(spec), B.SRW_HOST, B.SRW_FP32, None)),
            ("linear where", L.srw_loglik_linear(h, _p(th), 2, _p(out), None, 5, None)),
        ]
        for name, st in cases:
            assert st == B.SRW_EINVAL, name
        assert np.all(out == 0.0)  # nothing was written by the rejected calls
        # the handle still works: a valid call against the oracle
        ref = O.OracleModel.from_workload(wl)
        ref.set_data(counts, wl["bkg"])
        th[1] = [0.02, -0.01, 0.0, 0.0, 0.5]
        got = lk.loglik(th, srw.SRW_FP32)
        want = ref.neg2lnl_batch(th.astype(np.float64))
        assert np.max(np.abs(got - want)) <= 1e-4
