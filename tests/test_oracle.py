"""Pins of the FP64 oracle against values fixed by physics and mathematics.

Each test pins part of the oracle to something other than itself: textbook
cross sections and constants, the kinematic endpoint, the structure of the
cross section at the endpoint, brute-force quadrature, exact identities of the
fold, and brute-force Poisson probabilities.  A dropped term, a wrong sign, a
swapped flavour or a transposed response breaks at least one of them.
"""

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

HBARC2 = (197.3269804e-13) ** 2   # (hbar c)^2 in MeV^2 cm^2 (CODATA 2018)
R_E_CM = 2.8179403262e-13         # classical electron radius [cm] (CODATA 2018)


def _single(e, pee=1.0, w=1.0):
    return [{"e": np.array([e], dtype=float), "w": np.array([w], dtype=float), "pee": np.array([pee], dtype=float)}]


# ---------------------------------------------------------------- constants
def test_sigma0_matches_vogel_engel():
    # Vogel & Engel, PRD 39 (1989) 3378: sigma_0 = 2 G_F^2 m_e^2 / pi = 88.06e-46 cm^2
    assert O.sigma0() * O.M_E * HBARC2 == pytest.approx(88.06e-46, rel=2e-4)


def test_mm_prefactor_is_pi_re_squared():
    # pi alpha^2 / m_e^2 = pi r_e^2 (classical electron radius)
    pref_cm2 = O.mm_kappa() * O.sigma0() / O.MU_NU_UNIT ** 2 * HBARC2
    assert pref_cm2 == pytest.approx(math.pi * R_E_CM ** 2, rel=1e-8)
    assert O.mm_kappa() == pytest.approx(1.4476e-3, rel=2e-4)


@pytest.mark.parametrize("flavor,pee,f_tau,sigma_per_mev", [
    ("nu_e", 1.0, 0.5, 9.49e-45),    # textbook high-energy nu_e e cross section / E
    ("nu_mu", 0.0, 0.0, 1.58e-45),   # textbook nu_mu e cross section / E
])
def test_high_energy_total_cross_section(flavor, pee, f_tau, sigma_per_mev):
    e = 1000.0
    edges = np.linspace(0.0, 1000.0, 101)
    s = O.recoil_spectrum(_single(e, pee), edges, np.zeros(5), t_min=1e-9, f_tau=f_tau)
    sigma_cm2 = s.sum() * O.sigma0() * HBARC2
    # tree level; the textbook numbers include small radiative corrections
    assert sigma_cm2 / e == pytest.approx(sigma_per_mev, rel=3e-2)


def test_high_energy_limit_gl2_plus_gr2_over_3():
    g = O.sm_couplings(0.23121)["e"]
    for e in (1e3, 1e4):
        edges = np.linspace(0.0, e, 11)
        s = O.recoil_spectrum(_single(e), edges, np.zeros(5), t_min=1e-12).sum()
        assert s / e == pytest.approx(g[0] ** 2 + g[1] ** 2 / 3.0, rel=2 * O.M_E / e)


# ---------------------------------------------------------------- kinematics
@pytest.mark.parametrize("e,tmax", [(0.862, 0.66492), (0.384, 0.23058), (1.44, 1.22296), (16.0, 15.7485)])
def test_kinematic_endpoint(e, tmax):
    assert float(O.t_max(e)) == pytest.approx(tmax, abs=6e-5)


def test_be7_compton_edge_bins(be7_workload):
    wl = be7_workload
    s = O.recoil_spectrum(wl["sources"], wl["t_edges"], np.zeros(5), wl["t_min"])
    edge = 0.66492
    k = int(edge * 256)  # bin holding the edge
    assert k == 170
    assert np.all(s[:k] > 0)
    assert 0 < s[k] < s[k - 1]
    assert np.all(s[k + 1:] == 0.0)


def test_weak_cross_section_is_perfect_square_at_endpoint():
    # At T = T_max, m_e T / E^2 = 2 (1 - T/E), so the quadratic form in
    # (g_L, g_R) collapses to (g_L - (1 - T/E) g_R)^2: this fixes the sign
    # of the interference term and its m_e factor.
    rng = np.random.default_rng(7)
    for _ in range(50):
        e = rng.uniform(0.1, 20.0)
        gl, gr = rng.normal(size=2)
        t = float(O.t_max(e))
        expect = (gl - (1.0 - t / e) * gr) ** 2
        assert O.dsigma_weak(e, t, gl, gr) == pytest.approx(expect, rel=1e-10, abs=1e-13)
        # strictly positive below the endpoint for generic couplings
        assert O.dsigma_weak(e, 0.9 * t, gl, gr) > 0


def test_pure_helicity_shapes():
    e = 2.0
    t = np.linspace(0.0, float(O.t_max(e)), 7)
    assert np.allclose(O.dsigma_weak(e, t, 1.0, 0.0), 1.0)
    assert np.allclose(O.dsigma_weak(e, t, 0.0, 1.0), (1.0 - t / e) ** 2)


# ---------------------------------------------------------------- bin integrals
def _gauss_legendre(f, a, b, n_sub=64, order=32):
    x, w = np.polynomial.legendre.leggauss(order)
    edges = np.linspace(a, b, n_sub + 1)
    tot = 0.0
    for lo, hi in zip(edges[:-1], edges[1:]):
        xm, xr = 0.5 * (hi + lo), 0.5 * (hi - lo)
        tot += xr * np.sum(w * f(xm + xr * x))
    return tot


def test_bin_integrals_match_quadrature():
    rng = np.random.default_rng(11)
    sources = [
        {"e": np.array([0.862, 0.5]), "w": np.array([1.0, 0.3]), "pee": np.array([0.55, 0.6])},
        {"e": np.array([1.44, 0.25]), "w": np.array([0.2, 2.0]), "pee": np.array([0.5, 0.57])},
    ]
    edges = np.sort(np.concatenate([[0.0, 1.3], rng.uniform(0.0, 1.3, 14)]))
    t_min, f_tau = 2e-3, 0.3
    for theta in (np.zeros(5), np.array([0.1, -0.2, 0.3, 0.05, 2.5]), np.array([-0.4, 0.4, -0.1, 0.2, 0.0])):
        s = O.recoil_spectrum(sources, edges, theta, t_min=t_min, f_tau=f_tau)
        g = O.nsi_couplings(theta, 0.23121)
        for i in range(len(edges) - 1):
            tot = 0.0
            for src in sources:
                for e, w, pee in zip(src["e"], src["w"], src["pee"]):
                    a, b = max(edges[i], t_min), min(edges[i + 1], float(O.t_max(e)))
                    if b <= a:
                        continue
                    pe, pm, pt = O.flavor_probabilities(pee, f_tau)

                    def f(t):
                        return (pe * O.dsigma_weak(e, t, *g["e"]) + pm * O.dsigma_weak(e, t, *g["mu"])
                                + pt * O.dsigma_weak(e, t, *g["tau"]) + O.dsigma_mm(e, t, theta[4]))
                    tot += w * _gauss_legendre(f, a, b)
            assert s[i] == pytest.approx(tot, rel=1e-12, abs=1e-15)


def test_midpoint_mode_is_eq_fT():
    src = _single(0.862, 0.55, 2.0)
    edges = np.linspace(0.0, 1.0, 9)
    th = np.array([0.1, 0.2, -0.1, 0.05, 1.5])
    s = O.recoil_spectrum(src, edges, th, t_min=1e-3, midpoint=True)
    g = O.nsi_couplings(th, 0.23121)
    pe, pm, pt = O.flavor_probabilities(0.55, 0.5)
    for i in range(8):
        tc = 0.5 * (edges[i] + edges[i + 1])
        if tc >= float(O.t_max(0.862)):
            assert s[i] == 0.0
            continue
        ds = (pe * O.dsigma_weak(0.862, tc, *g["e"]) + pm * O.dsigma_weak(0.862, tc, *g["mu"])
              + pt * O.dsigma_weak(0.862, tc, *g["tau"]) + O.dsigma_mm(0.862, tc, th[4]))
        assert s[i] == pytest.approx(2.0 * ds * 0.125, rel=1e-14)


# ---------------------------------------------------------------- flavour routing
def test_flavor_routing():
    edges = np.linspace(0.0, 1.2, 13)
    gsm = O.sm_couplings(0.23121)
    # pure nu_tau with eps_tautau shifts == pure nu_e with the same total couplings
    el, er = 0.13, -0.07
    tau = O.recoil_spectrum(_single(1.44, pee=0.0), edges, np.array([0, 0, el, er, 0.0]), f_tau=1.0)
    gl_t, gr_t = gsm["tau"][0] + el, gsm["tau"][1] + er
    as_e = O.recoil_spectrum(_single(1.44, pee=1.0), edges,
                             np.array([gl_t - gsm["e"][0], gr_t - gsm["e"][1], 0, 0, 0.0]))
    np.testing.assert_allclose(tau, as_e, rtol=1e-13)
    # pure nu_mu ignores every NSI parameter
    mu0 = O.recoil_spectrum(_single(1.44, pee=0.0), edges, np.zeros(5), f_tau=0.0)
    mu1 = O.recoil_spectrum(_single(1.44, pee=0.0), edges, np.array([0.3, -0.2, 0.25, 0.1, 0.0]), f_tau=0.0)
    np.testing.assert_array_equal(mu0, mu1)


# ---------------------------------------------------------------- weights
def test_weights_identically_one_at_sm(be7_workload, solar_workload):
    for wl in (be7_workload, solar_workload):
        m = O.OracleModel.from_workload(wl)
        w = O.reweight_factor(m.spectrum(np.zeros(5)), m.s_sm)
        assert np.all(w == 1.0)


def test_coupling_sign_flip_invariance(be7_workload):
    wl = be7_workload
    g = O.sm_couplings(wl["sin2w"])["e"]
    flip = np.array([-2 * g[0], -2 * g[1], 0.0, 0.0, 0.0])
    s0 = O.recoil_spectrum(wl["sources"], wl["t_edges"], np.zeros(5), wl["t_min"])
    s1 = O.recoil_spectrum(wl["sources"], wl["t_edges"], flip, wl["t_min"])
    np.testing.assert_allclose(s1, s0, rtol=1e-13)


def test_spectrum_is_linear_in_coupling_monomials(solar_workload):
    wl = solar_workload
    b = O.coefficient_spectra(wl["sources"], wl["t_edges"], wl["t_min"], wl["sin2w"], wl["f_tau"])
    rng = np.random.default_rng(3)
    for _ in range(3):
        th = np.concatenate([rng.uniform(-0.3, 0.3, 4), rng.uniform(0, 3, 1)])
        s = O.recoil_spectrum(wl["sources"], wl["t_edges"], th, wl["t_min"], wl["sin2w"], wl["f_tau"])
        np.testing.assert_allclose(O.coupling_coefficients(th, wl["sin2w"]) @ b, s, rtol=1e-12, atol=1e-15 * s.max())


def test_midpoint_spectrum_is_linear_in_coupling_monomials(solar_workload):
    # the same decomposition holds bin by bin in the midpoint mode (eq. fT literally)
    wl = solar_workload
    edges = wl["t_edges"][::8]  # 512 bins: every source still spans many of them
    b = O.coefficient_spectra(wl["sources"], edges, wl["t_min"], wl["sin2w"], wl["f_tau"], midpoint=True)
    rng = np.random.default_rng(4)
    for _ in range(3):
        th = np.concatenate([rng.uniform(-0.3, 0.3, 4), rng.uniform(0, 3, 1)])
        s = O.recoil_spectrum(wl["sources"], edges, th, wl["t_min"], wl["sin2w"], wl["f_tau"], midpoint=True)
        np.testing.assert_allclose(O.coupling_coefficients(th, wl["sin2w"]) @ b, s, rtol=1e-12, atol=1e-15 * s.max())


def test_magnetic_moment_only_adds(be7_workload):
    wl = be7_workload
    s0 = O.recoil_spectrum(wl["sources"], wl["t_edges"], np.zeros(5), wl["t_min"])
    s1 = O.recoil_spectrum(wl["sources"], wl["t_edges"], np.array([0, 0, 0, 0, 2.0]), wl["t_min"])
    d = s1 - s0
    assert np.all(d[s0 > 0] > 0)
    # the 1/T enhancement: the added rate falls with T
    nz = d[s0 > 0]
    assert np.all(np.diff(nz[:150]) < 0)


# ---------------------------------------------------------------- fold
def test_identity_response():
    rng = np.random.default_rng(5)
    w = rng.uniform(0, 3, 17)
    np.testing.assert_array_equal(O.fold(np.eye(17), w), w)


def test_one_hot_picks_column_and_counts_are_conserved(be7_workload):
    r = be7_workload["R"].astype(np.float64)
    e = np.zeros(r.shape[1])
    e[37] = 1.0
    np.testing.assert_array_equal(O.fold(r, e), r[:, 37])
    w = np.random.default_rng(1).uniform(0, 1, r.shape[1])
    assert O.fold(r, w).sum() == pytest.approx(float(O.efficiency(r) @ w), rel=1e-13)


def test_exposure_normalisation(be7_workload):
    m = O.OracleModel.from_workload(be7_workload)
    assert m.mu_sig(np.zeros(5)).sum() == pytest.approx(be7_workload["exposure"], rel=1e-13)


# ---------------------------------------------------------------- likelihood
def _brute_neg2lnl(mu, n):
    tot = 0.0
    for m, k in zip(mu, n):
        k = int(k)
        # -2 ln( m^k e^-m / k! ) with the factorial exact
        tot += -2.0 * (k * math.log(m) - m - math.log(Fraction(math.factorial(k))))
    return tot


def test_poisson_against_brute_force():
    rng = np.random.default_rng(9)
    mu = rng.uniform(0.1, 30.0, 40)
    n = rng.poisson(mu).astype(float)
    assert O.neg2lnl(mu, n) == pytest.approx(_brute_neg2lnl(mu, n), rel=1e-12)


def test_poisson_against_scipy():
    from scipy.stats import poisson
    rng = np.random.default_rng(10)
    mu = rng.uniform(100.0, 5000.0, 64)
    n = rng.poisson(mu).astype(float)
    assert O.neg2lnl(mu, n) == pytest.approx(-2.0 * poisson.logpmf(n, mu).sum(), rel=1e-12)


def test_poisson_special_cases():
    assert O.neg2lnl([2.5], [0.0]) == pytest.approx(5.0)
    assert O.neg2lnl([0.0], [0.0]) == 0.0
    assert O.neg2lnl([0.0], [3.0]) == math.inf
    assert O.neg2lnl([-1.0], [0.0]) == math.inf
    assert O.neg2lnl([1.0, 7.0], [2.0, 9.0], mask=[0, 1]) == pytest.approx(O.neg2lnl([7.0], [9.0]))


def test_asimov_minimum_in_mu():
    # d/dmu of -2lnL vanishes at mu = n: scaling mu away from n raises it
    n = np.array([10.0, 50.0, 7.0, 120.0])
    base = O.neg2lnl(n, n)
    for s in (0.97, 1.03):
        assert O.neg2lnl(n * s, n) > base


def test_stored_counts_are_poisson_of_sm(be7_workload):
    import workloads
    n = workloads.load_counts(be7_workload["name"])
    m = O.OracleModel.from_workload(be7_workload)
    m.set_data(n, be7_workload["bkg"])
    nu = m.mu(np.zeros(5))
    assert n.shape == nu.shape
    # Pearson chi2 per bin of order 1
    chi2 = np.sum((n - nu) ** 2 / nu) / n.size
    assert 0.7 < chi2 < 1.3
