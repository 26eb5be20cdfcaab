"""FP64 CPU oracle for the spectrum-reweighting likelihood.

TEST INFRASTRUCTURE.  This module is the plain, slow, obviously-correct
reference the CUDA library is checked against.  Only the test-suite, the
smoke check and the CPU-baseline leg of the benchmark may import it; the
library never does, and it shares no code with the library.

Everything is float64 numpy written straight from the paper's definitions
(arXiv 2607.00488, "GPU-accelerated spectrum reweighting for new-physics
searches in solar neutrino-electron scattering"):

* chiral couplings                       Sec. II.A (tree level)
* SM differential cross section          Sec. II.A, eq. sm_cross_section
* oscillated flavour fluxes              Sec. II.A (phi_k^alpha = P_ek^alpha phi_k)
* NSI coupling shifts                    Sec. II.B, eqs. g_tilde, xs_nsi
* magnetic-moment cross section          Sec. II.C, eq. xs_mm
* incoherent sum                         Sec. II.C, eq. xs_total
* recoil spectrum per bin                Sec. III.A, eq. fT (and its exact
                                         bin-integrated form, see below)
* reweighting factor                     Sec. III.A, eqs. fT_norm, reweight_factor
* response fold                          Sec. II.D eq. visible_spectrum; Sec. I eq. matrix_reweight
* expected counts                        Sec. III.C, eq. mu_total
* Poisson -2 ln L                        Sec. III.C, eq. logL

Readings where the paper is silent (each is also recorded in the design notes):
* Cross sections are in units of sigma0 = 2 G_F^2 m_e / pi (the absolute
  scale cancels in the weights); mu_hat = mu_nu / (1e-11 mu_B).
* T is clipped to the kinematic endpoint T_max(E) = 2E^2/(m_e + 2E) and
  to T >= t_min (the analysis threshold that regulates the 1/T term,
  Sec. II.C) for the SM and MM terms alike.
* Default ("integrated") mode: S_i = integral over the recoil bin of
  sum_alpha P_alpha dsigma_alpha/dT + dsigma_MM/dT, summed over nodes with
  weight w_n = phi(E_n) dE.  "midpoint" mode is eq. fT literally: the
  cross section at the bin centre times the bin width, counted iff
  t_min <= T_c < T_max(E).
* The nu_mu / nu_tau split of 1 - P_ee is (1 - f_tau, f_tau).
* Weight w_i = S_i(theta)/S_i(SM), and w_i = 1 where S_i(SM) = 0.
* The SM true-recoil baseline E_SM is lambda * S_SM with lambda fixed so
  that sum_j (R E_SM)_j = exposure, unless a baseline is supplied.
* mu_j = M_j [ sum_i R_ji w_i E_SM,i + sum_b bkg_bj ]; -2lnL sums the
  masked-in bins; 0 ln 0 = 0; mu_j <= 0 with n_j > 0 (or mu_j < 0) gives +inf.
"""

from __future__ import annotations

import math

import numpy as np

# Physical constants (CODATA 2018)
M_E = 0.51099895000          # electron mass [MeV]
ALPHA = 1.0 / 137.035999084  # fine-structure constant
G_F = 1.1663787e-11          # Fermi constant [MeV^-2]
MU_NU_UNIT = 1.0e-11         # theta[4] is mu_nu in units of 1e-11 Bohr magnetons


# --------------------------------------------------------------------------
# kinematics and couplings
# --------------------------------------------------------------------------
def t_max(e):
    """Kinematic endpoint of the electron recoil, T_max = 2E^2/(m_e + 2E)."""
    e = np.asarray(e, dtype=np.float64)
    return 2.0 * e * e / (M_E + 2.0 * e)


def sm_couplings(sin2w):
    """Tree-level chiral couplings (Sec. II.A): (g_L, g_R) per flavour."""
    s = float(sin2w)
    return {"e": (0.5 + s, s), "mu": (-0.5 + s, s), "tau": (-0.5 + s, s)}


def nsi_couplings(theta, sin2w):
    """Flavour-diagonal NSI shifts g -> g + eps (Sec. II.B, eq. g_tilde).

    theta = (eps_L_ee, eps_R_ee, eps_L_tautau, eps_R_tautau, mu_hat); the
    nu_mu couplings are not shifted."""
    g = sm_couplings(sin2w)
    el_ee, er_ee, el_tt, er_tt = (float(x) for x in theta[:4])
    return {
        "e": (g["e"][0] + el_ee, g["e"][1] + er_ee),
        "mu": g["mu"],
        "tau": (g["tau"][0] + el_tt, g["tau"][1] + er_tt),
    }


def sigma0():
    """2 G_F^2 m_e / pi, the prefactor of eq. sm_cross_section [MeV^-3]."""
    return 2.0 * G_F * G_F * M_E / math.pi


def mm_kappa():
    """pi alpha^2 / m_e^2 (eq. xs_mm) in units of sigma0, for mu_nu = 1e-11 mu_B [MeV]."""
    return (math.pi * ALPHA * ALPHA / (M_E * M_E)) / sigma0() * MU_NU_UNIT ** 2


def flavor_probabilities(pee, f_tau):
    """(P_e, P_mu, P_tau) = (P_ee, (1-P_ee)(1-f_tau), (1-P_ee) f_tau)."""
    pee = np.asarray(pee, dtype=np.float64)
    return pee, (1.0 - pee) * (1.0 - f_tau), (1.0 - pee) * f_tau


# --------------------------------------------------------------------------
# cross sections (units of sigma0)
# --------------------------------------------------------------------------
def dsigma_weak(e, t, gl, gr):
    """eq. sm_cross_section / sigma0 (with NSI-shifted couplings, eq. xs_nsi)."""
    return gl * gl + gr * gr * (1.0 - t / e) ** 2 - gl * gr * M_E * t / (e * e)


def dsigma_mm(e, t, mu_hat):
    """eq. xs_mm / sigma0: kappa mu_hat^2 (1/T - 1/E)."""
    return mm_kappa() * mu_hat * mu_hat * (1.0 / t - 1.0 / e)


def weak_antiderivative(e, t, gl, gr):
    """F(T) with dF/dT = dsigma_weak(E, T)."""
    return gl * gl * t - gr * gr * (e / 3.0) * (1.0 - t / e) ** 3 - gl * gr * M_E * t * t / (2.0 * e * e)


def mm_antiderivative(e, t, mu_hat):
    """G(T) with dG/dT = dsigma_mm(E, T) (T > 0)."""
    return mm_kappa() * mu_hat * mu_hat * (np.log(t) - t / e)


# --------------------------------------------------------------------------
# recoil spectrum (eq. fT summed over components k and flavours alpha)
# --------------------------------------------------------------------------
def _pair_values(e, w, pee, lo, hi, t_min, g, mu_hat, f_tau, midpoint):
    e = e[:, None]
    pe, pm, pt = (p[:, None] for p in flavor_probabilities(pee, f_tau))
    tm = t_max(e)
    if midpoint:
        tc = 0.5 * (lo + hi)[None, :]
        ok = (tc >= t_min) & (tc < tm)
        tcs = np.where(ok, tc, 1.0)
        val = (pe * dsigma_weak(e, tcs, *g["e"]) + pm * dsigma_weak(e, tcs, *g["mu"])
               + pt * dsigma_weak(e, tcs, *g["tau"]) + dsigma_mm(e, tcs, mu_hat)) * (hi - lo)[None, :]
    else:
        a = np.maximum(lo, t_min)[None, :] + 0.0 * e
        b = np.minimum(hi[None, :], tm)
        ok = b > a
        a = np.where(ok, a, 1.0)
        b = np.where(ok, b, 1.0)
        val = (pe * (weak_antiderivative(e, b, *g["e"]) - weak_antiderivative(e, a, *g["e"]))
               + pm * (weak_antiderivative(e, b, *g["mu"]) - weak_antiderivative(e, a, *g["mu"]))
               + pt * (weak_antiderivative(e, b, *g["tau"]) - weak_antiderivative(e, a, *g["tau"]))
               + (mm_antiderivative(e, b, mu_hat) - mm_antiderivative(e, a, mu_hat)))
    return (w[:, None] * np.where(ok, val, 0.0)).sum(axis=0)


def recoil_spectrum(sources, t_edges, theta, t_min=1e-3, sin2w=0.23121, f_tau=0.5,
                    midpoint=False, chunk=256):
    """S_i(theta): recoil-bin spectrum summed over all sources and flavours.

    sources: iterable of dicts with float64 arrays ``e`` (MeV), ``w``
    (phi(E) dE per node) and ``pee``.  Returns float64 [n_t]."""
    t_edges = np.asarray(t_edges, dtype=np.float64)
    lo, hi = t_edges[:-1], t_edges[1:]
    g = nsi_couplings(theta, sin2w)
    mu_hat = float(theta[4])
    s = np.zeros(lo.shape[0], dtype=np.float64)
    for src in sources:
        e = np.asarray(src["e"], dtype=np.float64)
        w = np.asarray(src["w"], dtype=np.float64)
        pee = np.asarray(src["pee"], dtype=np.float64)
        for k0 in range(0, e.shape[0], chunk):
            sl = slice(k0, k0 + chunk)
            # bins starting at or above the largest endpoint in the chunk get nothing
            nb = int(np.searchsorted(lo, float(t_max(e[sl]).max()), side="left"))
            if nb == 0:
                continue
            s[:nb] += _pair_values(e[sl], w[sl], pee[sl], lo[:nb], hi[:nb], t_min, g, mu_hat, f_tau, midpoint)
    return s


def coupling_coefficients(theta, sin2w=0.23121):
    """Monomials c_b(theta) that multiply the coefficient spectra below:
    [gLe^2, gRe^2, -gLe gRe, gLt^2, gRt^2, -gLt gRt, 1, mu_hat^2]."""
    g = nsi_couplings(theta, sin2w)
    (gle, gre), (glt, grt) = g["e"], g["tau"]
    mu = float(theta[4])
    return np.array([gle * gle, gre * gre, -gle * gre, glt * glt, grt * grt, -glt * grt, 1.0, mu * mu])


def _term_integrals(e, a, b):
    """Integrals over [a, b] of the four T-shapes of the cross section:
    1, (1 - T/E)^2, m_e T / E^2 and 1/T - 1/E (antiderivative differences)."""
    i_one = b - a
    i_rr = (e / 3.0) * ((1.0 - a / e) ** 3 - (1.0 - b / e) ** 3)
    i_lr = M_E * (b * b - a * a) / (2.0 * e * e)
    i_mm = np.log(b) - np.log(a) - (b - a) / e
    return i_one, i_rr, i_lr, i_mm


def _term_midpoint(e, tc, width):
    return (width + 0.0 * e, width * (1.0 - tc / e) ** 2, width * M_E * tc / (e * e),
            width * (1.0 / tc - 1.0 / e))


def coefficient_spectra(sources, t_edges, t_min=1e-3, sin2w=0.23121, f_tau=0.5, midpoint=False,
                        chunk=256):
    """The recoil spectrum is a polynomial in the couplings and mu_hat^2;
    return its eight coefficient spectra [8, n_t] in the order of
    ``coupling_coefficients``: for nu_e the P_e-weighted bin integrals of
    1, (1-T/E)^2 and m_e T/E^2; the same three for nu_tau; the complete
    (unshifted) nu_mu spectrum; and the magnetic-moment spectrum for
    mu_nu = 1e-11 mu_B.  S(theta) = sum_b c_b(theta) B_b."""
    t_edges = np.asarray(t_edges, dtype=np.float64)
    lo, hi = t_edges[:-1], t_edges[1:]
    gm_l, gm_r = sm_couplings(sin2w)["mu"]
    kappa = mm_kappa()
    out = np.zeros((8, lo.shape[0]))
    for src in sources:
        e_all = np.asarray(src["e"], dtype=np.float64)
        w_all = np.asarray(src["w"], dtype=np.float64)
        pee_all = np.asarray(src["pee"], dtype=np.float64)
        for k0 in range(0, e_all.shape[0], chunk):
            sl = slice(k0, k0 + chunk)
            nb = int(np.searchsorted(lo, float(t_max(e_all[sl]).max()), side="left"))
            if nb == 0:
                continue
            e, w = e_all[sl][:, None], w_all[sl][:, None]
            pe, pm, pt = (p[:, None] for p in flavor_probabilities(pee_all[sl], f_tau))
            l, h = lo[:nb], hi[:nb]
            tm = t_max(e)
            if midpoint:
                tc = 0.5 * (l + h)[None, :]
                ok = (tc >= t_min) & (tc < tm)
                terms = _term_midpoint(e, np.where(ok, tc, 1.0), (h - l)[None, :])
            else:
                a = np.maximum(l, t_min)[None, :] + 0.0 * e
                b = np.minimum(h[None, :], tm)
                ok = b > a
                terms = _term_integrals(e, np.where(ok, a, 1.0), np.where(ok, b, 1.0))
            one, rr, lr, mm = (np.where(ok, t, 0.0) for t in terms)
            o = out[:, :nb]
            o[0] += (w * pe * one).sum(axis=0)
            o[1] += (w * pe * rr).sum(axis=0)
            o[2] += (w * pe * lr).sum(axis=0)
            o[3] += (w * pt * one).sum(axis=0)
            o[4] += (w * pt * rr).sum(axis=0)
            o[5] += (w * pt * lr).sum(axis=0)
            o[6] += (w * pm * (gm_l * gm_l * one + gm_r * gm_r * rr - gm_l * gm_r * lr)).sum(axis=0)
            o[7] += (w * kappa * mm).sum(axis=0)
    return out


# --------------------------------------------------------------------------
# reweighting, fold, expectation, likelihood
# --------------------------------------------------------------------------
def reweight_factor(s_theta, s_sm):
    """w_i = S_i(theta) / S_i(SM) (eqs. fT_norm, reweight_factor; the
    normalisation of f_hat cancels against E_SM), 1 where S_i(SM) = 0."""
    s_theta = np.asarray(s_theta, dtype=np.float64)
    s_sm = np.asarray(s_sm, dtype=np.float64)
    safe = np.where(s_sm != 0.0, s_sm, 1.0)
    return np.where(s_sm != 0.0, s_theta / safe, 1.0)


def efficiency(r):
    """eff_i = sum_j R_ji (Sec. II.D: column sums of the conditional response)."""
    return np.asarray(r, dtype=np.float64).sum(axis=0)


def baseline_true_spectrum(s_sm, r, exposure):
    """E_SM = lambda S_SM with sum_j (R E_SM)_j = exposure."""
    s_sm = np.asarray(s_sm, dtype=np.float64)
    lam = exposure / float(np.dot(efficiency(r), s_sm))
    return lam * s_sm


def fold(r, w_true):
    """Visible spectrum sum_i R_ji W_i (eq. visible_spectrum / matrix_reweight)."""
    return np.asarray(r, dtype=np.float64) @ np.asarray(w_true, dtype=np.float64)


def expected_counts(mu_sig, bkg_sum, mask=None):
    """mu_j = M_j (signal_j + background_j) (eq. mu_total)."""
    mu = np.asarray(mu_sig, dtype=np.float64) + np.asarray(bkg_sum, dtype=np.float64)
    if mask is not None:
        mu = mu * (np.asarray(mask) != 0)
    return mu


def neg2lnl(mu, n, mask=None):
    """-2 ln L = 2 sum_j [mu_j - n_j ln mu_j + ln Gamma(n_j + 1)] (eq. logL,
    without the Gaussian pull terms, which the caller adds)."""
    mu = np.asarray(mu, dtype=np.float64)
    n = np.asarray(n, dtype=np.float64)
    use = np.ones(mu.shape, dtype=bool) if mask is None else (np.asarray(mask) != 0)
    total = 0.0
    for j in np.nonzero(use)[0]:
        m, k = float(mu[j]), float(n[j])
        if m < 0.0 or (m == 0.0 and k > 0.0):
            return math.inf
        nlog = k * math.log(m) if k > 0.0 else 0.0
        total += m - nlog + math.lgamma(k + 1.0)
    return 2.0 * total


class OracleModel:
    """The full per-theta chain on one detector configuration, in float64."""

    def __init__(self, t_edges, sources, r, exposure, t_min=1e-3, sin2w=0.23121, f_tau=0.5,
                 midpoint=False, e_true_sm=None):
        self.t_edges = np.asarray(t_edges, dtype=np.float64)
        self.sources = sources
        self.r = np.asarray(r, dtype=np.float64)
        self.exposure = float(exposure)
        self.t_min, self.sin2w, self.f_tau, self.midpoint = float(t_min), float(sin2w), float(f_tau), bool(midpoint)
        self.s_sm = self.spectrum(np.zeros(5))
        if e_true_sm is None:
            self.e_sm = baseline_true_spectrum(self.s_sm, self.r, self.exposure)
        else:
            self.e_sm = np.asarray(e_true_sm, dtype=np.float64)
        self.counts = None
        self.bkg_sum = np.zeros(self.r.shape[0])
        self.mask = None

    @classmethod
    def from_workload(cls, wl, **kw):
        return cls(wl["t_edges"], wl["sources"], wl["R"], wl["exposure"], wl["t_min"], wl["sin2w"],
                   wl["f_tau"], **kw)

    def spectrum(self, theta):
        return recoil_spectrum(self.sources, self.t_edges, np.asarray(theta, dtype=np.float64), self.t_min,
                               self.sin2w, self.f_tau, self.midpoint)

    def weighted_true(self, theta):
        """W_i = w_i(theta) E_SM,i, the reweighted true-recoil spectrum."""
        return reweight_factor(self.spectrum(theta), self.s_sm) * self.e_sm

    def mu_sig(self, theta):
        return fold(self.r, self.weighted_true(theta))

    def set_data(self, counts, bkg=None, mask=None):
        self.counts = np.asarray(counts, dtype=np.float64)
        if bkg is not None:
            self.bkg_sum = np.asarray(bkg, dtype=np.float64).reshape(-1, self.r.shape[0]).sum(axis=0)
        self.mask = None if mask is None else np.asarray(mask)

    def mu(self, theta):
        return expected_counts(self.mu_sig(theta), self.bkg_sum, self.mask)

    def neg2lnl(self, theta):
        return neg2lnl(self.mu(theta), self.counts, self.mask)

    def neg2lnl_batch(self, thetas):
        return np.array([self.neg2lnl(t) for t in np.asarray(thetas, dtype=np.float64)])


# ---------------------------------------------------------------------------
# Profiled signal normalisation (a nuisance parameter of the fit, Sec. IV.B)
# ---------------------------------------------------------------------------
def profiled_neg2lnl(mu_sig, bkg, counts, sigma_alpha=0.0, mask=None):
    """min over alpha >= 0 of -2 ln L(alpha mu_sig + bkg) + ((alpha - 1)/sigma)^2
    (the pull term only when sigma_alpha > 0): the signal rate scaled by a free
    or Gaussian-constrained normalisation.  The minimum is found with a bounded
    scalar minimiser in float64 and returned with alpha-hat."""
    from scipy.optimize import minimize_scalar
    mu_sig = np.asarray(mu_sig, dtype=np.float64)
    bkg = np.asarray(bkg, dtype=np.float64)

    def f(a):
        v = neg2lnl(a * mu_sig + bkg, counts, mask)
        if sigma_alpha > 0.0:
            v += ((a - 1.0) / sigma_alpha) ** 2
        return v

    # bracket: the objective is convex in alpha; search [0, a_hi]
    a_hi = 2.0
    while f(2.0 * a_hi) < f(a_hi) and a_hi < 1e6:
        a_hi *= 2.0
    r = minimize_scalar(f, bounds=(0.0, 2.0 * a_hi), method="bounded", options={"xatol": 1e-12, "maxiter": 500})
    a = float(r.x)
    return f(a), a
