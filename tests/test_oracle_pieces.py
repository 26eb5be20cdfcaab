"""Direct pins of the oracle's building blocks that the other oracle tests
reach only through the spectrum: the per-bin antiderivatives (Sec. II, eqs.
sm_cross_section, xs_mm, integrated over a recoil bin), the exposure
normalisation of the SM baseline spectrum and the expected counts (eq.
mu_total).  Each is checked against something other than its own formula:
numerical derivatives, Gauss-Legendre quadrature, and the defining
properties.
"""

import numpy as np
import pytest

import oracle as O


def _points(seed=11, n=40):
    rng = np.random.default_rng(seed)
    e = rng.uniform(0.2, 16.0, n)
    t = rng.uniform(0.05, 0.95, n) * O.t_max(e)
    gl = rng.uniform(-1.0, 1.0, n)
    gr = rng.uniform(-1.0, 1.0, n)
    return e, t, gl, gr


def test_weak_antiderivative_differentiates_to_the_cross_section():
    e, t, gl, gr = _points()
    h = 1e-5 * t
    num = (O.weak_antiderivative(e, t + h, gl, gr) - O.weak_antiderivative(e, t - h, gl, gr)) / (2.0 * h)
    assert np.allclose(num, O.dsigma_weak(e, t, gl, gr), rtol=1e-8, atol=1e-10)


def test_mm_antiderivative_differentiates_to_the_cross_section():
    e, t, _, _ = _points(12)
    mu = 2.3
    h = 1e-6 * t
    num = (O.mm_antiderivative(e, t + h, mu) - O.mm_antiderivative(e, t - h, mu)) / (2.0 * h)
    assert np.allclose(num, O.dsigma_mm(e, t, mu), rtol=1e-7)


@pytest.mark.parametrize("e", [0.384, 0.862, 1.44, 9.0])
def test_antiderivative_differences_are_the_bin_integrals(e):
    # 32-point Gauss-Legendre on 64 sub-intervals of [a, b] (substitution
    # u = ln T for the 1/T term), against F(b) - F(a)
    x, wq = np.polynomial.legendre.leggauss(32)
    a, b = 1e-3, float(O.t_max(e))
    edges = np.linspace(a, b, 65)
    gl, gr, mu = 0.7, -0.3, 1.7
    weak = mm = 0.0
    for lo, hi in zip(edges[:-1], edges[1:]):
        t = 0.5 * (hi - lo) * x + 0.5 * (hi + lo)
        weak += 0.5 * (hi - lo) * np.sum(wq * O.dsigma_weak(e, t, gl, gr))
    ue = np.linspace(np.log(a), np.log(b), 65)
    for lo, hi in zip(ue[:-1], ue[1:]):
        u = 0.5 * (hi - lo) * x + 0.5 * (hi + lo)
        t = np.exp(u)
        mm += 0.5 * (hi - lo) * np.sum(wq * O.dsigma_mm(e, t, mu) * t)
    assert O.weak_antiderivative(e, b, gl, gr) - O.weak_antiderivative(e, a, gl, gr) == pytest.approx(weak, rel=1e-12)
    assert O.mm_antiderivative(e, b, mu) - O.mm_antiderivative(e, a, mu) == pytest.approx(mm, rel=1e-12)


def test_baseline_spectrum_carries_the_exposure():
    rng = np.random.default_rng(5)
    r = rng.uniform(0.0, 1.0, (7, 11)) * (rng.uniform(size=(7, 11)) < 0.6)
    s_sm = rng.uniform(0.0, 3.0, 11)
    e_sm = O.baseline_true_spectrum(s_sm, r, 12345.0)
    # the folded baseline holds the exposure, and E_SM is a multiple of S_SM
    assert np.sum(r @ e_sm) == pytest.approx(12345.0, rel=1e-13)
    ratio = e_sm[s_sm > 0] / s_sm[s_sm > 0]
    assert np.allclose(ratio, ratio[0], rtol=1e-14)


def test_expected_counts_drop_masked_bins():
    mu_sig = np.array([1.0, 2.0, 3.0, 4.0])
    bkg = np.array([0.5, 0.25, 0.0, 1.0])
    assert np.array_equal(O.expected_counts(mu_sig, bkg), [1.5, 2.25, 3.0, 5.0])
    assert np.array_equal(O.expected_counts(mu_sig, bkg, np.array([1, 0, 1, 0], np.uint8)), [1.5, 0.0, 3.0, 0.0])
