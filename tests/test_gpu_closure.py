"""The paper's closure test (Sec. VI.A, Figs. closure and closure_conv) run
through the library.

The worked example of test_closure.py: a 7Be line, N_p photoelectron bins
with 500 photoelectrons/MeV, a quenched light yield and Gaussian
photoelectron statistics, ROI 50 < N_p < 400.  Here the reweighted prediction
comes from the CUDA path: srw_create in midpoint mode (eq. fT at the bin
centre, the paper's evaluation) with the SM-weighted response matrix
R[N_p][T bin] (what an SM Monte Carlo sample gives; built on the host from
the oracle's quadrature, as test_closure.py does) and the integrated SM
recoil histogram as the supplied baseline E_true^SM (eq. matrix_reweight).
srw_spectrum stage 2 then returns eq. fNp_reweight's folded signal.  It is
compared with the oracle's direct continuum fold at n_T = 25, 50, 100 and
2000 recoil bins: the n_T^-2 slope, the printed 25-bin deviations (to a
factor of two: the quenching law is not given in the paper) and the 2000-bin
limits (integral < 1e-6, every ROI bin < 1e-5), and it must agree with the
oracle's own reweighted prediction.
"""

import math

import numpy as np
import pytest

import oracle as O
import test_closure as C

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


def _closure_inputs(n_t, tmax):
    """Recoil edges, SM-weighted response [N_p bin][T bin] and the integrated
    SM recoil histogram for n_t uniform bins on [0, T_max]."""
    edges = np.linspace(0.0, tmax, n_t + 1)
    e_sm = O.recoil_spectrum(C.SRC, edges, np.zeros(5), C.T_MIN)
    resp = np.zeros((n_t, C.NP_EDGES.size - 1))
    for i in range(n_t):
        a, b = max(edges[i], C.T_MIN), edges[i + 1]
        if b <= a or e_sm[i] == 0.0:
            continue
        num = C._integrate(lambda t: C._p_np_given_t(t) * C._dsigma(t, np.zeros(5))[:, None], a, b,
                           max(2, 4000 // n_t))
        resp[i] = num / e_sm[i]
    return edges, np.maximum(resp.T, 0.0), e_sm


def _gpu_reweighted(srw, theta, n_t, tmax):
    edges, R, e_sm = _closure_inputs(n_t, tmax)
    wl = {"t_edges": edges, "R": R.astype(np.float32), "sources": C.SRC, "exposure": 1.0, "t_min": C.T_MIN,
          "sin2w": 0.23121, "f_tau": 0.5}
    with srw.Likelihood(wl, midpoint=True, e_true_sm=e_sm) as lk:
        return np.asarray(lk.spectrum(np.asarray(theta, np.float32), 2), np.float64)


@pytest.mark.parametrize("case,theta,dev25", C.CASES, ids=[c[0] for c in C.CASES])
def test_closure_on_the_gpu_path(srw, case, theta, dev25):
    tmax = float(O.t_max(C.E_LINE))
    direct = C._direct(theta, tmax)
    roi = direct[C.ROI].sum()
    devs = {}
    for n_t in (25, 50, 100, 2000):
        mu = _gpu_reweighted(srw, theta, n_t, tmax)
        cpu = C._reweighted(theta, n_t, tmax)
        # the library's reweighted fold equals the oracle's (FP32 R and spectra)
        np.testing.assert_allclose(mu[C.ROI], cpu[C.ROI], rtol=2e-6)
        devs[n_t] = (abs(mu[C.ROI].sum() - roi) / roi, np.max(np.abs(mu[C.ROI] / direct[C.ROI] - 1.0)))
    print(case, {k: ("%.2e" % v[0], "%.2e" % v[1]) for k, v in devs.items()})
    slope = math.log(devs[25][0] / devs[100][0]) / math.log(4.0)
    assert slope == pytest.approx(C.LIMITS["slope"], rel=0.05)
    assert dev25 / 2.0 < devs[25][0] < dev25 * 2.0
    assert devs[2000][0] < C.LIMITS["integral_2000"]
    assert devs[2000][1] < C.LIMITS["bin_2000"]
