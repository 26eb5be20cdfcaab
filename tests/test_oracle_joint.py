"""Pins of the joint-response oracle (Sec. III.B-C, eqs. Rij, fNp_reweight, mu_total).

Each test ties the oracle to something other than its own formulas: the
paper's statements about the construction (global normalisation to s^(k), the
SM recovered by construction, the conditional kernel recovered by dividing by
f_hat^SM), the already-pinned conditional oracle, and invariances that a
plausible slip (mask applied along the wrong axis, per-column instead of
global normalisation, a dropped prefactor, a transposed histogram) breaks.
"""

import numpy as np
import pytest

import oracle as O
from oracle.joint_oracle import (JointOracleModel, default_events, joint_response, normalised_spectrum,
                                 predicted_distribution, reweighting_function)
from workloads.joint import live_time, scale_factor, mc_histogram
from workloads.solar import _source, continuum_nodes, pee_solar, response_matrix

T_EDGES = np.linspace(0.0, 2.0, 129)
REC_EDGES = np.linspace(0.0, 2.0, 65)


def small_components():
    e, w = continuum_nodes(1.2, 50, 3.0e8)
    return [_source("be7", np.array([0.862, 0.384]), np.array([4.5e9, 0.5e9]), pee_solar),
            _source("pep", np.array([1.44]), np.array([1.4e8]), pee_solar),
            _source("n13", e, w, pee_solar)]


def spectra(comps, theta):
    return [O.recoil_spectrum([c], T_EDGES, np.asarray(theta, dtype=float)) for c in comps]


def test_joint_response_normalised_globally_to_the_scale():
    rng = np.random.default_rng(0)
    hist = rng.poisson(5.0, size=(7, 11)).astype(float)
    mask = rng.uniform(0.5, 1.0, size=7)
    r = joint_response(hist, mask, 0.37)
    assert r.sum() == pytest.approx(0.37, rel=1e-14)
    # a global, not per-true-bin, normalisation: the column sums keep the
    # histogram's (live-corrected) proportions
    col = (hist / mask[:, None]).sum(axis=0)
    np.testing.assert_allclose(r.sum(axis=0) / r.sum(axis=0)[0], col / col[0], rtol=1e-13)
    # invariant under the overall MC statistics and an overall live-time factor
    np.testing.assert_allclose(joint_response(3.0 * hist, mask, 0.37), r, rtol=1e-14)
    np.testing.assert_allclose(joint_response(hist, 0.5 * mask, 0.37), r, rtol=1e-14)


def test_live_time_correction_undoes_thinning():
    # expected histogram thinned by the live fraction of its reconstructed bin:
    # dividing by the same mask restores the unthinned shape exactly
    rng = np.random.default_rng(1)
    g = rng.uniform(0.0, 1.0, size=(9, 5))
    live = np.linspace(0.8, 1.0, 9)
    np.testing.assert_allclose(joint_response(g * live[:, None], live, 1.0), g / g.sum(), rtol=1e-13)
    # the mask acts on reconstructed bins (rows): a mask along true bins would not undo it
    assert not np.allclose(joint_response(g * live[:, None], np.ones(9), 1.0), g / g.sum(), rtol=1e-6)


def test_sm_recovered_by_construction():
    # eq. fNp_reweight at the SM: sum_i R_ij (for any joint response, also
    # where the SM spectrum vanishes in some bins)
    comps = small_components()
    f_sm = spectra(comps, np.zeros(5))
    rng = np.random.default_rng(2)
    for f in f_sm:
        r = rng.uniform(0.0, 1.0, size=(64, 128))
        np.testing.assert_allclose(predicted_distribution(r, f, f), r.sum(axis=1), rtol=1e-12)
    assert np.any(f_sm[0] == 0.0)  # the 7Be lines end well below 2 MeV


def test_reweighting_function_is_relative_to_the_normalised_sm():
    comps = small_components()
    f_sm = spectra(comps, np.zeros(5))[2]
    f_th = spectra(comps, [0.1, -0.05, 0.02, 0.0, 1.5])[2]
    r = reweighting_function(f_th, f_sm)
    live = f_sm > 0
    np.testing.assert_allclose(r[live], f_th[live] / f_sm[live] * f_sm.sum(), rtol=1e-12)
    assert np.all(r[~live] == f_sm.sum())
    assert normalised_spectrum(f_sm).sum() == pytest.approx(1.0, rel=1e-14)


def test_joint_reduces_to_the_conditional_response():
    # Noise-free SM histograms built from a conditional response R_c (live-time
    # thinned): the joint chain must give exactly the conditional oracle's
    # prediction mu_j = sum_i R_c,ji w_i E_SM,i, which is pinned separately.
    comps = small_components()
    r_c = response_matrix(T_EDGES, REC_EDGES, res=0.05, kq=0.01, tail_frac=1e-3).astype(np.float64)
    live = live_time(REC_EDGES)
    f_sm = spectra(comps, np.zeros(5))
    hist, scale = [], []
    for f in f_sm:
        exact = 1.0e6 * normalised_spectrum(f)[None, :] * r_c  # expected SM events [j, i]
        hist.append(exact * live[:, None])
        scale.append(exact.sum() / 1.0e6)
    joint = JointOracleModel(T_EDGES, comps, hist, [live] * 3, scale, live=None, exposure=1.0e5)
    cond = O.OracleModel(T_EDGES, comps, r_c, 1.0e5)
    for theta in ([0, 0, 0, 0, 0], [0.2, -0.1, 0.05, 0.1, 0.0], [-0.3, 0.3, -0.2, 0.25, 2.5]):
        np.testing.assert_allclose(joint.mu_sig(theta), cond.mu_sig(theta), rtol=1e-11, atol=1e-9)


def test_rates_follow_the_integrated_spectrum():
    # With rate_k(theta) proportional to the component's integrated spectrum
    # the prefactor of eq. fNp_reweight cancels: MT rate_k f^(k) = N_k sum_i R_ij f_i(theta)/f_i(SM)
    comps = small_components()
    rng = np.random.default_rng(3)
    hist = [rng.poisson(20.0, size=(64, 128)).astype(float) for _ in comps]
    mask = [np.ones(64)] * 3
    m = JointOracleModel(T_EDGES, comps, hist, mask, [0.9, 0.8, 0.7], exposure=5.0e4)
    theta = [0.15, 0.1, -0.2, 0.05, 2.0]
    f_th = spectra(comps, theta)
    for k in range(3):
        f_sm = m.f_sm[k]
        w = np.where(f_sm > 0, f_th[k] / np.where(f_sm > 0, f_sm, 1.0), 1.0)
        r = hist[k] / hist[k].sum() * [0.9, 0.8, 0.7][k]
        np.testing.assert_allclose(m.component_mu(k, theta), m.events[k] * (r @ w), rtol=1e-12)
    # and the SM signal adds up to the exposure
    assert m.mu_sig(np.zeros(5)).sum() == pytest.approx(5.0e4, rel=1e-13)


def test_given_events_and_common_mask():
    comps = small_components()
    rng = np.random.default_rng(4)
    hist = [rng.poisson(20.0, size=(64, 128)).astype(float) for _ in comps]
    live = np.linspace(0.5, 1.0, 64)
    ev = np.array([1.0e4, 2.0e3, 5.0e2])
    s = np.array([0.9, 0.8, 0.7])
    m = JointOracleModel(T_EDGES, comps, hist, [np.ones(64)] * 3, s, live=live, events=ev)
    sm = m.mu_sig(np.zeros(5))
    want = live * sum(ev[k] * (hist[k] / hist[k].sum() * s[k]).sum(axis=1) for k in range(3))
    np.testing.assert_allclose(sm, want, rtol=1e-12)
    assert default_events(m.f_sm, m.r_joint, live, 1.0).shape == (3,)


def test_sampled_histograms_follow_the_sm():
    # the synthetic Monte Carlo: counts conserved up to thinning and losses,
    # the scale factor is the live-corrected detected fraction
    comps = small_components()
    r_c = response_matrix(T_EDGES, REC_EDGES, res=0.05, kq=0.01, tail_frac=1e-3)
    live = live_time(REC_EDGES)
    f_hat = normalised_spectrum(spectra(comps, np.zeros(5))[2])
    h = mc_histogram(f_hat, r_c, live, 200000, 7)
    assert h.shape == (64, 128) and np.all(h >= 0) and np.all(h == np.round(h))
    assert np.all(h[:, f_hat == 0] == 0)
    s = scale_factor(h, live, 200000)
    eff = (r_c.astype(np.float64) * f_hat[None, :]).sum()
    assert s == pytest.approx(eff, abs=5e-3)
