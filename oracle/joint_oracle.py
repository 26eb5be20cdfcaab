"""FP64 oracle of the per-source joint response (Sec. III.B-C).

TEST INFRASTRUCTURE.  Like the rest of ``oracle/``, only the test-suite, the
smoke check and the benchmark's CPU-baseline legs may import it; the library
never does, and the two share no code.

What it computes, in the paper's order:

* eq. Rij          R^(k)_ij = (N^(k)_ij / M^(k)_j) / sum_{i'j'} (N^(k)_i'j' / M^(k)_j') * s^(k),
                   from the SM Monte Carlo histogram N^(k) of component k
                   (true recoil bin i, reconstructed bin j), its live-time
                   correction mask M^(k) and its scale factor s^(k);
* eq. fT_norm      f_hat^SM(T_i) = f_T^SM(T_i) / sum_l f_T^SM(T_l);
* eq. reweight_factor  r^(k)(T_i) = f_T^(k)(T_i; theta) / f_hat^SM,(k)(T_i);
* eq. fNp_reweight f^(k)(j; theta) = sum_i R^(k)_ij r^(k)(T_i) / sum_l f_T^(k)(T_l; theta);
* eq. mu_total     mu_j = MT M_j sum_k rate_k(theta) f^(k)(j; theta) (+ backgrounds,
                   whose 1-D templates enter directly).

Readings where the paper is silent:

* Histograms are stored like the conditional response, [n_rec, n_t]
  (reconstructed bin j is the row, true bin i the column).
* The rate of a signal component follows its integrated cross section
  (Sec. III.C): rate_k(theta) = rate_k(SM) sum_l f_T^(k)(T_l; theta) /
  sum_l f_T^(k)(T_l; SM), the sum running over the recoil bins of the
  analysis.  MT rate_k(SM) is the component's SM event count N_k (given, or
  lambda F_k with F_k = sum_l f_T^(k)(T_l; SM) and lambda fixing the total SM
  signal to the exposure).
* Where f_hat^SM vanishes the reweighting is taken relative to the SM
  (r = sum_l f_T^SM(T_l), weight one), as on the conditional path.
"""

from __future__ import annotations

import numpy as np

from .srw_oracle import neg2lnl, recoil_spectrum


def joint_response(hist, mask, scale):
    """Eq. Rij for one component: the live-time-corrected histogram,
    normalised to a global sum of one, times the scale factor s^(k)."""
    hist = np.asarray(hist, dtype=np.float64)
    mask = np.asarray(mask, dtype=np.float64)
    corrected = hist / mask[:, None]
    return corrected / corrected.sum() * float(scale)


def normalised_spectrum(f):
    """Eq. fT_norm: the spectrum divided by its sum over the recoil bins."""
    f = np.asarray(f, dtype=np.float64)
    return f / f.sum()


def reweighting_function(f_theta, f_sm):
    """Eq. reweight_factor: r_i = f_T(T_i; theta) / f_hat^SM(T_i); the SM
    normalisation sum_l f_T^SM(T_l) where f_hat^SM(T_i) = 0."""
    f_theta = np.asarray(f_theta, dtype=np.float64)
    f_hat = normalised_spectrum(f_sm)
    safe = np.where(f_hat != 0.0, f_hat, 1.0)
    return np.where(f_hat != 0.0, f_theta / safe, float(np.sum(f_sm)))


def predicted_distribution(r_joint, f_theta, f_sm):
    """Eq. fNp_reweight: the joint response contracted with the reweighting
    function over the true index, divided by the integral of f_T(theta)."""
    r = reweighting_function(f_theta, f_sm)
    return np.asarray(r_joint, dtype=np.float64) @ r / float(np.sum(f_theta))


def default_events(f_sm, r_joint, live, exposure):
    """N_k = lambda F_k, F_k = sum_l f_T^(k)(T_l; SM), lambda such that the
    total SM signal sum_j M_j sum_k N_k f^(k)(j; SM) equals the exposure
    (f^(k)(j; SM) = sum_i R^(k)_ij)."""
    F = np.array([float(np.sum(f)) for f in f_sm])
    per_event = np.array([float(np.dot(live, np.asarray(r, dtype=np.float64).sum(axis=1))) for r in r_joint])
    lam = float(exposure) / float(np.dot(F, per_event))
    return lam * F


class JointOracleModel:
    """mu(theta) and -2 ln L with one joint response per signal component.

    components: one source dict (``e``, ``w``, ``pee``) per component k;
    hist[k]: [n_rec, n_t] SM Monte Carlo histogram; mask[k]: [n_rec]
    live-time correction M^(k); scale[k]: s^(k); live: [n_rec] common mask M_j
    of eq. mu_total; events: N_k = MT rate_k(SM), or None for the exposure
    normalisation above."""

    def __init__(self, t_edges, components, hist, mask, scale, live=None, events=None, exposure=None,
                 t_min=1e-3, sin2w=0.23121, f_tau=0.5, midpoint=False):
        self.t_edges = np.asarray(t_edges, dtype=np.float64)
        self.components = list(components)
        self.t_min, self.sin2w, self.f_tau, self.midpoint = float(t_min), float(sin2w), float(f_tau), bool(midpoint)
        n_rec = np.asarray(hist[0]).shape[0]
        self.live = np.ones(n_rec) if live is None else np.asarray(live, dtype=np.float64)
        self.r_joint = [joint_response(h, m, s) for h, m, s in zip(hist, mask, scale)]
        self.f_sm = [self.component_spectrum(k, np.zeros(5)) for k in range(len(self.components))]
        if events is None:
            self.events = default_events(self.f_sm, self.r_joint, self.live, exposure)
        else:
            self.events = np.asarray(events, dtype=np.float64)
        self.counts = None
        self.bkg_sum = np.zeros(n_rec)
        self.mask = None

    @classmethod
    def from_workload(cls, wl, **kw):
        return cls(wl["t_edges"], wl["components"], wl["hist"], wl["mc_mask"], wl["scale"], wl["live"],
                   wl.get("events"), wl["exposure"], wl["t_min"], wl["sin2w"], wl["f_tau"], **kw)

    def component_spectrum(self, k, theta):
        return recoil_spectrum([self.components[k]], self.t_edges, np.asarray(theta, dtype=np.float64),
                               self.t_min, self.sin2w, self.f_tau, self.midpoint)

    def rate_times_exposure(self, k, f_theta):
        """MT rate_k(theta): N_k scaled by the component's integrated spectrum."""
        return self.events[k] * float(np.sum(f_theta)) / float(np.sum(self.f_sm[k]))

    def component_mu(self, k, theta):
        """MT rate_k(theta) f^(k)(j; theta), before the common mask."""
        f = self.component_spectrum(k, theta)
        return self.rate_times_exposure(k, f) * predicted_distribution(self.r_joint[k], f, self.f_sm[k])

    def mu_sig(self, theta):
        return self.live * sum(self.component_mu(k, theta) for k in range(len(self.components)))

    def set_data(self, counts, bkg=None, mask=None):
        self.counts = np.asarray(counts, dtype=np.float64)
        if bkg is not None:
            self.bkg_sum = np.asarray(bkg, dtype=np.float64).reshape(-1, self.live.shape[0]).sum(axis=0)
        self.mask = None if mask is None else np.asarray(mask)

    def mu(self, theta):
        mu = self.mu_sig(theta) + self.bkg_sum
        if self.mask is not None:
            mu = mu * (self.mask != 0)
        return mu

    def neg2lnl(self, theta):
        return neg2lnl(self.mu(theta), self.counts, self.mask)

    def neg2lnl_batch(self, thetas):
        return np.array([self.neg2lnl(t) for t in np.asarray(thetas, dtype=np.float64)])
