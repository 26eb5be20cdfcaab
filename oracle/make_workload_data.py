"""Write the stored pseudo-data counts of the synthetic workloads.

Data n_j ~ Poisson(mu_j(theta = 0)): the SM expectation of the FP64 oracle
(signal normalised to the workload's exposure, plus its background
templates), fluctuated with the workload's data seed.  Run once:

    python -m oracle.make_workload_data

Only the oracle computes the expectation; the counts are stored as text so
that every consumer reads the same bytes.
"""

from __future__ import annotations

import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import workloads  # noqa: E402
from oracle.srw_oracle import OracleModel  # noqa: E402


def sm_counts(wl):
    model = OracleModel.from_workload(wl)
    model.set_data(np.zeros(wl["R"].shape[0]), wl["bkg"])
    nu = model.mu(np.zeros(5))
    return workloads.poisson_counts(nu, wl["data_seed"])


def main():
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
