"""Synthetic solar-neutrino workloads (inputs only, no method arithmetic).

Every generator is deterministic given its seed.  Units: energies in MeV; the
magnetic moment enters theta as mu_hat = mu_nu / (1e-11 mu_B).

theta layout (one row per parameter point, float32):
    [eps_L_ee, eps_R_ee, eps_L_tautau, eps_R_tautau, mu_hat]

Workloads (shapes of the solar analyses of Sec. II-III of the paper):
  * ``be7_line_workload``   - one 7Be line (0.862 MeV), 256 recoil bins on
    [0, 1] MeV, 128 reconstructed bins, Gaussian 5%/sqrt(E) response with
    light-yield quenching and +-1 % multiplicative noise, 1e5 signal events
    plus a flat 10 % background; 16 theta on a 4x4 (eps_L_ee, eps_R_ee) grid.
  * ``solar_set_workload``  - pp / 7Be (two lines) / pep / 13N / 15O / 8B,
    2000 energy nodes per continuum (8003 nodes), 4096 recoil bins on
    [0, 16] MeV, 2048 reconstructed bins, response with a 0.1 % exponential
    low tail, eight background templates.
  * ``batched_scan_workload`` - the solar set with P theta drawn uniformly in
    the box |eps| <= 0.3, mu_hat in [0, 3].
  * ``uneven_groups_workload`` - 64 detector configurations with uneven
    binnings, exposures, resolutions and theta counts.
"""

from __future__ import annotations

import math
import os

import numpy as np
from scipy.special import erf

THETA_NAMES = ("eps_L_ee", "eps_R_ee", "eps_L_tautau", "eps_R_tautau", "mu_hat")

M_E_INPUT = 0.51099895  # MeV; only used to shape beta-like background templates

DEFAULT_T_MIN = 1e-3
DEFAULT_SIN2W = 0.23121
DEFAULT_F_TAU = 0.5

_DATA_DIR = os.path.join(os.path.dirname(__file__), "data")


# --------------------------------------------------------------------------
# sources
# --------------------------------------------------------------------------
def pee_solar(e):
    """Survival probability model: 0.55 up to 1 MeV, linear in ln E down to
    0.30 at 5 MeV, 0.30 above."""
    e = np.asarray(e, dtype=np.float64)
    x = (np.log(np.clip(e, 1.0, 5.0)) - 0.0) / math.log(5.0)
    return 0.55 + (0.30 - 0.55) * x


def continuum_nodes(q, n_e, rate):
    """Midpoint energy nodes E_n=(n+1/2)Q/N_E with beta-like weights
    E^2 (Q-E)^2 dE, normalised to sum 1 and scaled by ``rate``."""
    de = q / n_e
    e = (np.arange(n_e, dtype=np.float64) + 0.5) * de
    shape = e * e * (q - e) ** 2
    w = shape * de
    w = w / w.sum() * rate
    return e, w


def _source(name, e, w, pee_fn):
    e = np.ascontiguousarray(e, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    return {"name": name, "e": e, "w": w, "pee": np.ascontiguousarray(pee_fn(e), dtype=np.float64)}


def be7_sources():
    return [_source("be7_862", np.array([0.862]), np.array([1.0]), lambda e: np.full_like(e, 0.55))]


def solar_sources(n_e=2000):
    """pp, 7Be (0.862 MeV 90 %, 0.384 MeV 10 %), pep, 13N, 15O, 8B with
    SSM-order relative rates (arbitrary units; the exposure fixes the scale)."""
    out = []
    for name, q, rate in (("pp", 0.420, 6.0e10),):
        e, w = continuum_nodes(q, n_e, rate)
        out.append(_source(name, e, w, pee_solar))
    out.append(_source("be7_862", np.array([0.862]), np.array([0.9 * 5.0e9]), pee_solar))
    out.append(_source("be7_384", np.array([0.384]), np.array([0.1 * 5.0e9]), pee_solar))
    out.append(_source("pep", np.array([1.44]), np.array([1.4e8]), pee_solar))
    for name, q, rate in (("n13", 1.20, 3.0e8), ("o15", 1.73, 2.0e8), ("b8", 16.0, 5.0e6)):
        e, w = continuum_nodes(q, n_e, rate)
        out.append(_source(name, e, w, pee_solar))
    return out


# --------------------------------------------------------------------------
# response matrix R[j, i] = P(reconstructed bin j | recoil bin i)
# --------------------------------------------------------------------------
def visible_energy(t, kq=0.01):
    """Quenched light yield: E_vis = T / (1 + kq / T)."""
    t = np.asarray(t, dtype=np.float64)
    return t * t / (t + kq)


def response_matrix(t_edges, rec_edges, res=0.05, kq=0.01, tail_frac=0.0, noise=0.0, seed=0):
    """Conditional response as float32 [n_rec, n_t].

    Column i is the bin-integrated Gaussian N(E_vis(T_c), sigma^2) with
    sigma = res*sqrt(E_vis/MeV) MeV at the recoil-bin centre T_c, optionally
    mixed with a one-sided exponential low tail (fraction ``tail_frac``,
    length 2 sigma) and multiplied element-wise by U[1-noise, 1+noise].
    Mass falling outside the reconstructed range is lost, so column sums are
    the (energy-dependent) efficiency."""
    t_edges = np.asarray(t_edges, dtype=np.float64)
    x = np.asarray(rec_edges, dtype=np.float64)[:, None]
    tc = 0.5 * (t_edges[1:] + t_edges[:-1])
    m = visible_energy(tc, kq)[None, :]
    sig = np.maximum(res * np.sqrt(m), 1e-9)
    cdf = 0.5 * (1.0 + erf((x - m) / (math.sqrt(2.0) * sig)))
    r = np.diff(cdf, axis=0)
    if tail_frac > 0.0:
        lam = 2.0 * sig
        # CDF of the density exp((x-m)/lam)/lam on x < m
        tcdf = np.where(x < m, np.exp((np.minimum(x, m) - m) / lam), 1.0)
        r = (1.0 - tail_frac) * r + tail_frac * np.diff(tcdf, axis=0)
    if noise > 0.0:
        rng = np.random.default_rng(seed)
        r = r * rng.uniform(1.0 - noise, 1.0 + noise, size=r.shape)
    return np.ascontiguousarray(r, dtype=np.float32)


# --------------------------------------------------------------------------
# background templates (expected counts per reconstructed bin)
# --------------------------------------------------------------------------
def _bin_average(fn, edges, sub=8):
    edges = np.asarray(edges, dtype=np.float64)
    lo, hi = edges[:-1], edges[1:]
    u = (np.arange(sub) + 0.5) / sub
    xs = lo[:, None] + (hi - lo)[:, None] * u[None, :]
    return fn(xs).mean(axis=1) * (hi - lo)


def _beta_shape(q, offset=0.0):
    def fn(x):
        k = x - offset
        ok = (k > 0) & (k < q)
        kk = np.where(ok, k, 0.0)
        val = np.sqrt(kk * kk + 2 * kk * M_E_INPUT) * (kk + M_E_INPUT) * (q - kk) ** 2
        return np.where(ok, val, 0.0)
    return fn


def _gauss_shape(mu, sig):
    return lambda x: np.exp(-0.5 * ((x - mu) / sig) ** 2)


def _template(fn, edges, total):
    v = _bin_average(fn, edges)
    s = v.sum()
    return v * (total / s) if s > 0 else v


def solar_backgrounds(rec_edges):
    """Eight background templates: 210Po-like peak, 85Kr- and 210Bi-like beta
    shapes, 11C-like continuum (1.02-1.98 MeV), flat, exponential falling,
    14C-like beta, second (208Tl-like) peak."""
    lo, hi = float(rec_edges[0]), float(rec_edges[-1])
    specs = [
        ("po210", _gauss_shape(0.40, 0.03), 2.0e4),
        ("kr85", _beta_shape(0.687), 5.0e3),
        ("bi210", _beta_shape(1.16), 1.0e4),
        ("c11", _beta_shape(0.96, offset=1.02), 4.0e3),
        ("flat", lambda x: np.ones_like(x), 2.0e3),
        ("expo", lambda x: np.exp(-(x - lo) / 0.8), 3.0e3),
        ("c14", _beta_shape(0.156), 5.0e4),
        ("tl208", _gauss_shape(2.61, 0.08), 5.0e2),
    ]
    del hi
    names = [s[0] for s in specs]
    bkg = np.stack([_template(fn, rec_edges, tot) for _, fn, tot in specs])
    return names, np.ascontiguousarray(bkg, dtype=np.float64)


# --------------------------------------------------------------------------
# parameter points
# --------------------------------------------------------------------------
def theta_box(p, seed, eps_max=0.3, mu_max=3.0):
    """P points uniform in |eps| <= eps_max (four couplings), mu_hat in [0, mu_max]."""
    rng = np.random.default_rng(seed)
    th = np.empty((p, 5), dtype=np.float64)
    th[:, :4] = rng.uniform(-eps_max, eps_max, size=(p, 4))
    th[:, 4] = rng.uniform(0.0, mu_max, size=p)
    return np.ascontiguousarray(th, dtype=np.float32)


def fit_region_points(n, seed=99, eps_max=0.02, mu_max=0.5):
    """Points near the SM (|eps| <= eps_max, mu_hat <= mu_max): where a fit or a
    confidence interval on 1e5-event data is decided.  Seed 99, n = 8 are the
    benchmark's parity points."""
    rng = np.random.default_rng(seed)
    th = np.zeros((n, 5), np.float32)
    th[:, :4] = rng.uniform(-eps_max, eps_max, (n, 4))
    th[:, 4] = rng.uniform(0.0, mu_max, n)
    return th


def box_sample(p, n, seed):
    """n evenly spaced points of the P-point box batch theta_box(P, seed) (the
    benchmark's box parity sample: P = 65536, n = 12, seed 3)."""
    return theta_box(p, seed)[np.linspace(0, p - 1, n).astype(int)]


def theta_grid_be7():
    g = np.linspace(-0.5, 0.5, 4)
    th = np.zeros((16, 5), dtype=np.float32)
    k = 0
    for a in g:
        for b in g:
            th[k, 0], th[k, 1] = a, b
            k += 1
    return th


def poisson_counts(nu, seed):
    """Poisson pseudo-data with mean ``nu`` (float64 counts)."""
    rng = np.random.default_rng(seed)
    return rng.poisson(np.asarray(nu, dtype=np.float64)).astype(np.float64)


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
def _common(name, t_edges, rec_edges, sources, r, bkg_names, bkg, exposure, theta):
    return {
        "name": name,
        "t_edges": np.ascontiguousarray(t_edges, dtype=np.float64),
        "rec_edges": np.ascontiguousarray(rec_edges, dtype=np.float64),
        "sources": sources,
        "R": r,
        "bkg_names": bkg_names,
        "bkg": bkg,
        "exposure": float(exposure),
        "t_min": DEFAULT_T_MIN,
        "sin2w": DEFAULT_SIN2W,
        "f_tau": DEFAULT_F_TAU,
        "theta": theta,
        "data_seed": 0,
    }


def be7_line_workload():
    """One 7Be line, 256 x 128 bins on [0, 1] MeV, 1e5 events + 10 % flat bkg."""
    t_edges = np.linspace(0.0, 1.0, 257)
    rec_edges = np.linspace(0.0, 1.0, 129)
    r = response_matrix(t_edges, rec_edges, res=0.05, kq=0.01, noise=0.01, seed=0)
    bkg = np.full((1, 128), 1.0e4 / 128.0)
    return _common("be7_line_256", t_edges, rec_edges, be7_sources(), r, ["flat"], bkg, 1.0e5, theta_grid_be7())


def solar_set_workload(theta_seed=1, n_theta=1):
    """Full synthetic solar set: 8003 nodes, 4096 x 2048 bins on [0, 16] MeV."""
    t_edges = np.linspace(0.0, 16.0, 4097)
    rec_edges = np.linspace(0.0, 16.0, 2049)
    r = response_matrix(t_edges, rec_edges, res=0.05, kq=0.01, tail_frac=1e-3)
    names, bkg = solar_backgrounds(rec_edges)
    return _common("solar_set_4096", t_edges, rec_edges, solar_sources(), r, names, bkg, 1.0e5,
                   theta_box(n_theta, theta_seed))


def batched_scan_workload(p=65536, theta_seed=3):
    """The solar set with P theta points uniform in the 5-D box."""
    wl = solar_set_workload()
    wl["name"] = "solar_scan_%d" % p
    wl["theta"] = theta_box(p, theta_seed)
    return wl


def uneven_groups_workload(n_groups=64, seed=4, scale=1.0):
    """Uneven detector configurations sharing the solar sources.

    Per group: N_T ~ U{512..8192}, N_rec ~ U{256..4096}, exposure log-uniform
    in [1e4, 1e7], resolution U[3 %, 8 %]/sqrt(E), P ~ U{256..4096}, a flat
    10 % background.  ``scale`` < 1 shrinks all sizes (for quick tests)."""
    rng = np.random.default_rng(seed)
    src = solar_sources()
    groups = []
    for g in range(n_groups):
        n_t = int(rng.integers(512, 8193))
        n_rec = int(rng.integers(256, 4097))
        expo = float(10.0 ** rng.uniform(4.0, 7.0))
        res = float(rng.uniform(0.03, 0.08))
        p = int(rng.integers(256, 4097))
        if scale != 1.0:
            n_t = max(8, int(n_t * scale))
            n_rec = max(8, int(n_rec * scale))
            p = max(1, int(p * scale))
        groups.append({"n_t": n_t, "n_rec": n_rec, "exposure": expo, "res": res, "p": p,
                       "theta_seed": 1000 + g})
    return {"name": "uneven_%d" % n_groups, "sources": src, "groups": groups, "seed": seed}


def uneven_group_inputs(groups_wl, g):
    """Materialise group ``g`` of ``uneven_groups_workload`` as a workload dict."""
    spec = groups_wl["groups"][g]
    t_edges = np.linspace(0.0, 16.0, spec["n_t"] + 1)
    rec_edges = np.linspace(0.0, 16.0, spec["n_rec"] + 1)
    r = response_matrix(t_edges, rec_edges, res=spec["res"], kq=0.01, tail_frac=1e-3)
    bkg = np.full((1, spec["n_rec"]), 0.1 * spec["exposure"] / spec["n_rec"])
    return _common("uneven_g%02d" % g, t_edges, rec_edges, groups_wl["sources"], r, ["flat"], bkg,
                   spec["exposure"], theta_box(spec["p"], spec["theta_seed"]))


WORKLOADS = {
    "be7_line_256": be7_line_workload,
    "solar_set_4096": solar_set_workload,
}


def counts_path(name):
    return os.path.join(_DATA_DIR, name + "_counts.txt")


def group_counts_path(name):
    return os.path.join(_DATA_DIR, name + "_counts.txt.gz")


def load_group_counts(groups_wl):
    """Stored pseudo-data of every configuration of a grouped workload (one
    array per configuration, written by the oracle's data script)."""
    flat = np.loadtxt(group_counts_path(groups_wl["name"]), dtype=np.float64).reshape(-1)
    sizes = [g["n_rec"] for g in groups_wl["groups"]]
    if flat.size != sum(sizes):
        raise ValueError("stored grouped counts do not match the workload")
    return np.split(flat, np.cumsum(sizes)[:-1])


def load_counts(name):
    """Stored pseudo-data counts for a workload (written once by the oracle's
    data script from the SM expectation, Poisson seed 0)."""
    return np.loadtxt(counts_path(name), dtype=np.float64).reshape(-1)
