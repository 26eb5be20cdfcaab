"""End-to-end demonstrations on the GPU path: Asimov injection and recovery.

Asimov data are the expected counts at an injected point (no fluctuation), so
-2 ln L is smallest exactly there; scanning one parameter with the others held
at their injected values recovers it, and the points where -2 ln L rises by
2.706 above its minimum bound the 90 % confidence interval for one parameter
(Wilks' theorem; the paper's sensitivity study, Sec. VI, scans epsilon^L_ee and
mu_nu this way).  The expected counts come from the library itself
(srw_spectrum stage 3: the folded signal plus the background templates).

    python -m paper_2607_00488_gb300.demos          # solar set: eps^L_ee and mu_nu
"""

from __future__ import annotations

import json
import sys

import numpy as np

from . import srw as _srw

DCHI2_90 = 2.705543454095404  # chi^2 (1 dof) quantile at 0.90


def asimov_counts(lk, theta_inj):
    """Expected counts at theta_inj (eq. mu_total): srw_spectrum stage 3 of the
    library, the folded signal plus the summed background templates of the
    handle's data set."""
    return lk.spectrum(np.asarray(theta_inj, np.float32), 3).astype(np.float64)


def interval(grid, values, level=DCHI2_90):
    """Minimum of a 1-D scan and the crossings of min + level (linear interpolation
    between grid points; None where the scan does not cross inside the grid)."""
    grid = np.asarray(grid, dtype=np.float64)
    v = np.asarray(values, dtype=np.float64)
    k = int(np.argmin(v))
    target = v[k] + level
    lo = hi = None
    for i in range(k, 0, -1):
        if v[i - 1] >= target:
            lo = grid[i - 1] + (target - v[i - 1]) / (v[i] - v[i - 1]) * (grid[i] - grid[i - 1])
            break
    for i in range(k, len(v) - 1):
        if v[i + 1] >= target:
            hi = grid[i] + (target - v[i]) / (v[i + 1] - v[i]) * (grid[i + 1] - grid[i])
            break
    return {"argmin": float(grid[k]), "min": float(v[k]), "lo": lo, "hi": hi}


def scan_axis(lk, theta_inj, axis, grid, evaluate="fp16x3"):
    """-2 ln L along one parameter axis, the others held at theta_inj.
    evaluate: a precision name of the batched fold ("fp16x3", "bf16x3", "fp32")
    or "linear" (the exact rank-8 evaluator)."""
    th = np.tile(np.asarray(theta_inj, np.float32), (len(grid), 1))
    th[:, axis] = np.asarray(grid, np.float32)
    if evaluate == "linear":
        return lk.loglik_linear(th)
    return lk.loglik(th, _srw.PRECISIONS[evaluate])


def asimov_study(wl, theta_inj, scans, evaluate="fp16x3", counts=None):
    """Inject theta_inj (Asimov data from the library unless `counts` is given),
    move the fold's reference point there, and scan each (axis, grid) of
    `scans`.  Returns one interval() result per scan."""
    theta_inj = np.asarray(theta_inj, np.float64)
    with _srw.Likelihood(wl) as lk:
        if counts is None:
            # the background templates first (no counts yet), so that stage 3
            # returns the expectation at the injected point
            _srw.srw_set_data(lk.handle, np.zeros(wl["R"].shape[0]), wl.get("bkg"))
            n = asimov_counts(lk, theta_inj)
        else:
            n = np.asarray(counts, np.float64)
        _srw.srw_set_data(lk.handle, n, wl.get("bkg"))
        lk.set_reference(theta_inj)  # fold deviations from the injected point
        out = []
        for axis, grid in scans:
            v = scan_axis(lk, theta_inj, axis, grid, evaluate)
            r = interval(grid, v)
            r["axis"] = int(axis)
            out.append(r)
    return out


def main(argv=None):
    import workloads
    wl = workloads.solar_set_workload()
    theta_inj = np.array([0.05, 0.0, 0.0, 0.0, 3.0])  # eps^L_ee = 0.05, mu_nu = 3e-11 mu_B
    scans = [(0, np.linspace(0.0, 0.1, 401)), (4, np.linspace(0.0, 6.0, 601))]
    res = asimov_study(wl, theta_inj, scans)
    names = {0: "eps_L_ee", 4: "mu_nu / 1e-11 mu_B"}
    for r in res:
        r["parameter"] = names[r["axis"]]
    print(json.dumps(res, indent=1))
    return 0


if __name__ == "__main__":
    sys.exit(main())
