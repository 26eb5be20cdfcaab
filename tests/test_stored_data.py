"""The stored inputs under workloads/data are exactly what the oracle's data
script writes: re-running its steps reproduces every stored value bit for bit
(Poisson pseudo-data of the SM expectation, seed 0; the components' normalised
SM recoil spectra of the joint-response set)."""

import numpy as np
import pytest

import workloads
from oracle.joint_oracle import JointOracleModel, normalised_spectrum
from oracle.make_workload_data import sm_counts
from oracle.srw_oracle import recoil_spectrum
from workloads import joint as J


@pytest.mark.parametrize("name", sorted(workloads.WORKLOADS))
def test_counts_regenerate(name):
    wl = workloads.WORKLOADS[name]()
    np.testing.assert_array_equal(sm_counts(wl), workloads.load_counts(name))


def test_grouped_counts_regenerate():
    gw = workloads.uneven_groups_workload()
    stored = workloads.load_group_counts(gw)
    for g in (0, 17, 42, 63):  # a sample: all 64 take ~30 s
        np.testing.assert_array_equal(sm_counts(workloads.uneven_group_inputs(gw, g)), stored[g])


def test_joint_spectra_and_counts_regenerate():
    t_edges, _ = J.solar_joint_grid()
    comps = J.solar_components()
    f_hat = [normalised_spectrum(recoil_spectrum([c], t_edges, np.zeros(5), workloads.solar.DEFAULT_T_MIN,
                                                 workloads.solar.DEFAULT_SIN2W, workloads.solar.DEFAULT_F_TAU))
             for c in comps]
    stored = J.load_sm_spectra("solar_joint_4096", len(comps))
    for f, s in zip(f_hat, stored):
        np.testing.assert_array_equal(f, s)  # written with 17 significant digits: round-trips exactly
    wl = J.solar_joint_workload(f_hat=f_hat)
    model = JointOracleModel.from_workload(wl)
    model.set_data(np.zeros(len(wl["live"])), wl["bkg"])
    n = workloads.poisson_counts(model.mu(np.zeros(5)), wl["data_seed"])
    np.testing.assert_array_equal(n, workloads.load_counts(wl["name"]))
