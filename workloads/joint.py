"""Synthetic per-component Monte Carlo histograms for the joint response
(inputs only, no method arithmetic).

The paper builds one two-dimensional histogram N^(k)_ij per solar component k
from a detector simulation of SM events (true recoil bin i, reconstructed
bin j), with a bin-dependent live-time correction M_j and a scale factor s^(k)
(Sec. III.B).  The stand-in here samples such a simulation:

1. n_mc events per component; their true recoil bins are drawn from the
   component's normalised SM recoil spectrum (an input: the FP64 oracle
   writes it once to ``data/<name>_sm_spectra.txt.gz``, or a caller passes it);
2. each event's reconstructed bin is drawn from the conditional response
   column of its true bin (the smeared visible energy of the solar set), the
   rest of the column (1 - efficiency) being lost outside the window;
3. an event in reconstructed bin j is kept with the live-time fraction
   live_j (binomial thinning), so that N_ij / M_j with M_j = live_j undoes it;
4. s^(k) is the live-corrected fraction of the n_mc events inside the window
   (what the component's one-dimensional PDF integrates to there).

Histograms are float64 [n_rec, n_t] (reconstructed bin is the row), like the
conditional response.
"""

from __future__ import annotations

import os

import numpy as np

from .solar import (
    DEFAULT_F_TAU,
    DEFAULT_SIN2W,
    DEFAULT_T_MIN,
    _DATA_DIR,
    _source,
    pee_solar,
    response_matrix,
    solar_backgrounds,
    solar_sources,
    theta_box,
)


def solar_components(n_e=2000):
    """The solar set grouped into its physical components: pp, 7Be (both
    lines), pep, 13N, 15O, 8B."""
    src = {s["name"]: s for s in solar_sources(n_e)}
    be7 = _source("be7", np.concatenate([src["be7_862"]["e"], src["be7_384"]["e"]]),
                  np.concatenate([src["be7_862"]["w"], src["be7_384"]["w"]]), pee_solar)
    return [src["pp"], be7, src["pep"], src["n13"], src["o15"], src["b8"]]


def live_time(rec_edges, floor=0.9, e_on=0.15, width=0.02):
    """Bin-dependent live-time fraction: `floor` at low visible energy rising
    smoothly to 1 above e_on (a low-energy selection with reduced live time)."""
    rec_edges = np.asarray(rec_edges, dtype=np.float64)
    c = 0.5 * (rec_edges[1:] + rec_edges[:-1])
    return floor + (1.0 - floor) / (1.0 + np.exp(-(c - e_on) / width))


def mc_histogram(f_hat, r_cond, live, n_mc, seed):
    """One component's SM Monte Carlo histogram N[j, i] (steps 1-3 above)."""
    rng = np.random.default_rng(seed)
    f_hat = np.asarray(f_hat, dtype=np.float64)
    p_true = np.clip(f_hat, 0.0, None)
    p_true = p_true / p_true.sum()
    n_true = rng.multinomial(int(n_mc), p_true)
    r = np.asarray(r_cond, dtype=np.float64).T  # [n_t, n_rec]
    eff = r.sum(axis=1)
    over = eff > 1.0
    r[over] /= eff[over, None]
    lost = np.clip(1.0 - r.sum(axis=1), 0.0, None)
    pv = np.concatenate([r, lost[:, None]], axis=1)
    pv /= pv.sum(axis=1, keepdims=True)
    hist = rng.multinomial(n_true, pv)[:, :-1].T  # [n_rec, n_t]
    kept = rng.binomial(hist, np.asarray(live, dtype=np.float64)[:, None])
    return np.ascontiguousarray(kept, dtype=np.float64)


def scale_factor(hist, live, n_mc):
    """s^(k): live-corrected fraction of the simulated events in the window."""
    return float((np.asarray(hist) / np.asarray(live)[:, None]).sum() / float(n_mc))


def sm_spectra_path(name):
    return os.path.join(_DATA_DIR, name + "_sm_spectra.txt.gz")


def load_sm_spectra(name, n_components):
    """Stored normalised SM recoil spectra of the components (oracle output)."""
    flat = np.loadtxt(sm_spectra_path(name), dtype=np.float64)
    return flat.reshape(n_components, -1)


def joint_workload(name, t_edges, rec_edges, components, f_hat, exposure, n_mc, seed, res=0.05, tail_frac=1e-3,
                   bkg=None, bkg_names=None, theta=None):
    """Assemble a joint-response workload from normalised SM spectra f_hat[k]."""
    r_cond = response_matrix(t_edges, rec_edges, res=res, kq=0.01, tail_frac=tail_frac)
    live = live_time(rec_edges)
    hist, scale = [], []
    for k in range(len(components)):
        h = mc_histogram(f_hat[k], r_cond, live, n_mc, seed + k)
        hist.append(h)
        scale.append(scale_factor(h, live, n_mc))
    n_rec = len(rec_edges) - 1
    if bkg is None:
        bkg = np.full((1, n_rec), 0.1 * exposure / n_rec)
        bkg_names = ["flat"]
    return {
        "name": name,
        "t_edges": np.ascontiguousarray(t_edges, dtype=np.float64),
        "rec_edges": np.ascontiguousarray(rec_edges, dtype=np.float64),
        "components": components,
        "hist": hist,
        "mc_mask": [live.copy() for _ in components],
        "scale": np.array(scale),
        "live": live,
        "events": None,
        "exposure": float(exposure),
        "n_mc": int(n_mc),
        "bkg": np.ascontiguousarray(bkg, dtype=np.float64),
        "bkg_names": bkg_names,
        "t_min": DEFAULT_T_MIN,
        "sin2w": DEFAULT_SIN2W,
        "f_tau": DEFAULT_F_TAU,
        "theta": theta,
        "data_seed": 0,
    }


def solar_joint_grid():
    return np.linspace(0.0, 16.0, 4097), np.linspace(0.0, 16.0, 2049)


def solar_joint_workload(n_mc=10_000_000, seed=20, p=1, theta_seed=3, f_hat=None):
    """The solar set with one joint response per component: 4096 true x 2048
    reconstructed bins on [0, 16] MeV, six components, n_mc SM events each,
    eight background templates, 1e5 signal events."""
    t_edges, rec_edges = solar_joint_grid()
    comps = solar_components()
    if f_hat is None:
        f_hat = load_sm_spectra("solar_joint_4096", len(comps))
    names, bkg = solar_backgrounds(rec_edges)
    return joint_workload("solar_joint_4096", t_edges, rec_edges, comps, f_hat, 1.0e5, n_mc, seed, bkg=bkg,
                          bkg_names=names, theta=theta_box(p, theta_seed))
