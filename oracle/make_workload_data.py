"""Write the stored pseudo-data counts of the synthetic workloads.

Data n_j ~ Poisson(mu_j(theta = 0)): the SM expectation of the FP64 oracle
(signal normalised to the workload's exposure, plus its background
templates), fluctuated with the workload's data seed.  For the joint-response
workload it also writes the normalised SM recoil spectra of the components,
from which the synthetic Monte Carlo histograms are sampled.  Run once:

    python -m oracle.make_workload_data            # everything
    python -m oracle.make_workload_data --joint    # the joint-response files only

Only the oracle computes the expectation; the counts are stored as text so
that every consumer reads the same bytes.
"""

from __future__ import annotations

import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import workloads  # noqa: E402
from oracle.joint_oracle import JointOracleModel, normalised_spectrum  # noqa: E402
from oracle.srw_oracle import OracleModel, recoil_spectrum  # noqa: E402
from workloads import joint as J  # noqa: E402


def sm_counts(wl):
    model = OracleModel.from_workload(wl)
    model.set_data(np.zeros(wl["R"].shape[0]), wl["bkg"])
    nu = model.mu(np.zeros(5))
    return workloads.poisson_counts(nu, wl["data_seed"])


def write_joint():
    t_edges, _ = J.solar_joint_grid()
    comps = J.solar_components()
    f_hat = [normalised_spectrum(recoil_spectrum([c], t_edges, np.zeros(5), workloads.solar.DEFAULT_T_MIN,
                                                 workloads.solar.DEFAULT_SIN2W, workloads.solar.DEFAULT_F_TAU))
             for c in comps]
    path = J.sm_spectra_path("solar_joint_4096")
    np.savetxt(path, np.concatenate(f_hat), fmt="%.17g",
               header="solar_joint_4096: normalised SM recoil spectra of pp, 7Be, pep, 13N, 15O, 8B "
                      "(4096 bins each, concatenated)")
    print(path)
    wl = J.solar_joint_workload(f_hat=f_hat)
    model = JointOracleModel.from_workload(wl)
    model.set_data(np.zeros(len(wl["live"])), wl["bkg"])
    n = workloads.poisson_counts(model.mu(np.zeros(5)), wl["data_seed"])
    path = workloads.counts_path(wl["name"])
    np.savetxt(path, n, fmt="%d", header="%s: Poisson(SM expectation), seed %d" % (wl["name"], wl["data_seed"]))
    print(path, int(n.sum()))


def main():
    if "--joint" in sys.argv[1:]:
        write_joint()
        return
    write_joint()
    gw = workloads.uneven_groups_workload()
    parts = []
    for g in range(len(gw["groups"])):
        wl = workloads.uneven_group_inputs(gw, g)
        parts.append(sm_counts(wl))
    path = workloads.group_counts_path(gw["name"])
    np.savetxt(path, np.concatenate(parts), fmt="%d",
               header="%s: Poisson(SM expectation) per configuration, seed 0 each, "
                      "configurations concatenated in order" % gw["name"])
    print(path, len(parts))
    for name, make in workloads.WORKLOADS.items():
        wl = make()
        n = sm_counts(wl)
        path = workloads.counts_path(name)
        os.makedirs(os.path.dirname(path), exist_ok=True)
        np.savetxt(path, n, fmt="%d", header="%s: Poisson(SM expectation), seed %d" % (name, wl["data_seed"]))
        print(path, int(n.sum()))


if __name__ == "__main__":
    main()
