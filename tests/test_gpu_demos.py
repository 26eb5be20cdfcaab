"""End-to-end Asimov injection and recovery on the GPU path against the oracle.

Data: the oracle's expected counts at the injected point (eps^L_ee = 0.05,
mu_nu = 3e-11 mu_B on the 7Be line).  The GPU scans of eps^L_ee and mu_nu must
have their minimum at the injected grid point (-2 ln L there equal to the
data constant, Gibbs' inequality) and 90 % CL interval edges equal to the
oracle's scan of the same grid to 1e-3 of the grid range.
"""

import os

import numpy as np
import pytest

import oracle as O
import workloads
from oracle.mlp_oracle import data_constant

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


def _injected():
    """The paper's injection values (tests/golden/asimov_sec6b.txt)."""
    vals = {}
    for line in open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "asimov_sec6b.txt")):
        f = line.split()
        if f and not f[0].startswith("#"):
            vals[f[0]] = float(f[1])
    return vals


def test_asimov_injection_recovery(srw):
    from paper_2607_00488_gb300 import demos
    wl = workloads.be7_line_workload()
    inj = _injected()
    theta_inj = np.array([inj["eps_L_ee"], 0.0, 0.0, 0.0, inj["mu_nu_1e-11_muB"]])
    ref = O.OracleModel.from_workload(wl)
    ref.set_data(np.zeros(wl["R"].shape[0]), wl["bkg"])
    counts = ref.mu(theta_inj)  # Asimov data from the oracle
    ref.set_data(counts, wl["bkg"])
    scans = [(0, np.linspace(0.0, 0.1, 201)), (4, np.linspace(0.0, 6.0, 241))]
    for evaluate in ("fp16x3", "linear"):
        got = demos.asimov_study(wl, theta_inj, scans, evaluate=evaluate, counts=counts)
        for (axis, grid), r in zip(scans, got):
            th = np.tile(theta_inj.astype(np.float32), (len(grid), 1))
            th[:, axis] = grid.astype(np.float32)  # the points the GPU evaluates
            want = demos.interval(grid, [ref.neg2lnl(t.astype(np.float64)) for t in th])
            span = grid[-1] - grid[0]
            assert r["argmin"] == pytest.approx(theta_inj[axis]), (evaluate, axis, r)
            assert r["min"] == pytest.approx(data_constant(counts), abs=1e-3), (evaluate, axis, r)
            for edge in ("lo", "hi"):
                assert (r[edge] is None) == (want[edge] is None), (evaluate, axis, edge)
                if want[edge] is not None:
                    assert abs(r[edge] - want[edge]) <= 1e-3 * span, (evaluate, axis, edge, r[edge], want[edge])
