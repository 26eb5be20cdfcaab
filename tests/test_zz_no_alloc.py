"""The allocation-free single-point entry point.

Some callers cannot allocate device memory themselves (code running inside
another framework's memory manager, which owns every device allocation, or
code that must not call cudaMalloc/cudaFree because those calls can
synchronise the device).  srw_loglik_point_noalloc serves them: the caller
passes every input and the output as device memory, and the kernels' scratch
is a fixed static device array inside the library.  This test calls it through
the C ABI and checks it against the existing single-point entry point that
performs the same arithmetic (srw_loglik_points: the weighted spectrum from
the cross-section integrals, then the fold, with the reference point disabled
so that both fold W directly), twice in a row, since consecutive calls share
the scratch array.
"""

import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP32_LL = 1e-4


def test_no_alloc_entry_point_matches_loglik():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2607_00488_gb300 as srw

    wl = workloads.be7_line_workload()
    counts = workloads.load_counts(wl["name"])
    dev = torch.device("cuda")
    with srw.Likelihood(wl, counts) as lk:
        lk.set_reference(None)
        n_rec, n_t = wl["R"].shape
        ld = lk.info()["k_pad"]
        R = torch.zeros((n_rec, ld), dtype=torch.float32, device=dev)
        R[:, :n_t] = torch.from_numpy(wl["R"]).to(dev)
        c = torch.from_numpy(counts).to(dev)
        b = torch.from_numpy(wl["bkg"].sum(axis=0)).to(dev)
        thetas = [np.zeros(5, np.float32), np.array([0.01, -0.015, 0.005, 0.0, 0.3], np.float32)]
        for th in thetas:
            W = torch.zeros(ld, dtype=torch.float32, device=dev)
            lk.spectrum(torch.from_numpy(th).to(dev), 1, out=W)
            want = lk.loglik_points(th[None, :])[0]
            for _ in range(2):
                out = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
                srw.srw_loglik_point_noalloc(R, W, c, out, bkg=b)
                torch.cuda.synchronize()
                got = out.item()
                assert abs(got - want) <= TOL_FP32_LL, (got, want)


def test_no_alloc_rejects_oversized_input():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_00488_gb300 as srw
    dev = torch.device("cuda")
    R = torch.zeros((70000, 64), dtype=torch.float32, device=dev)  # beyond the 65536-bin limit
    W = torch.zeros(64, dtype=torch.float32, device=dev)
    c = torch.zeros(70000, dtype=torch.float64, device=dev)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(srw.SrwError) as ei:
        srw.srw_loglik_point_noalloc(R, W, c, out)
    assert ei.value.status == 1
