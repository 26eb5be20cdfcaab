"""The synthetic inputs follow their stated recipe (shapes, ranges, totals,
seeds); they carry none of the method's arithmetic, so these checks are about
the inputs alone."""

import math

import numpy as np
import pytest

import workloads
from workloads.solar import continuum_nodes, pee_solar, response_matrix
from workloads.joint import live_time, solar_joint_grid


def test_survival_probability_model():
    p = pee_solar(np.array([0.1, 1.0, math.sqrt(5.0), 5.0, 12.0]))
    # 0.55 up to 1 MeV, linear in ln E to 0.30 at 5 MeV (halfway in ln E at sqrt 5), 0.30 above
    np.testing.assert_allclose(p, [0.55, 0.55, 0.425, 0.30, 0.30], rtol=0, atol=1e-15)


def test_continuum_nodes_are_midpoints_with_beta_shape():
    e, w = continuum_nodes(1.2, 400, 3.0e8)
    de = 1.2 / 400
    np.testing.assert_allclose(e, (np.arange(400) + 0.5) * de, rtol=1e-15)
    assert w.sum() == pytest.approx(3.0e8, rel=1e-13)
    assert np.all(w > 0) and abs(e[np.argmax(w)] - 0.6) <= de  # E^2 (Q - E)^2 peaks at Q / 2
    np.testing.assert_allclose(w, w[::-1], rtol=1e-9)  # and is symmetric about it


def test_solar_set_shapes_and_totals(solar_workload):
    wl = solar_workload
    assert sum(s["e"].size for s in wl["sources"]) == 8003
    assert [s["name"] for s in wl["sources"]] == ["pp", "be7_862", "be7_384", "pep", "n13", "o15", "b8"]
    assert wl["R"].shape == (2048, 4096) and wl["R"].dtype == np.float32
    assert wl["t_edges"][0] == 0.0 and wl["t_edges"][-1] == 16.0 and wl["t_edges"].size == 4097
    assert wl["rec_edges"].size == 2049 and wl["exposure"] == 1.0e5
    assert wl["bkg"].shape == (8, 2048) and np.all(wl["bkg"] >= 0.0)
    assert wl["bkg"].sum() == pytest.approx(9.45e4, rel=1e-12)
    for s in wl["sources"]:
        assert np.all((s["pee"] >= 0.30) & (s["pee"] <= 0.55))
    th = wl["theta"]
    assert th.shape == (1, 5) and th.dtype == np.float32


def test_response_columns_are_efficiencies(solar_workload):
    r = solar_workload["R"].astype(np.float64)
    assert np.all(r >= 0.0)
    eff = r.sum(axis=0)
    assert np.all(eff <= 1.0 + 1e-5)
    # away from the window's edges nearly all of the smeared mass is inside
    tc = 0.5 * (solar_workload["t_edges"][1:] + solar_workload["t_edges"][:-1])
    inner = (tc > 1.0) & (tc < 14.0)
    assert np.all(eff[inner] > 0.999)
    # the resolution: a column's spread is about 5 % / sqrt(E_vis) at E_vis
    rc = 0.5 * (solar_workload["rec_edges"][1:] + solar_workload["rec_edges"][:-1])
    i = int(np.searchsorted(tc, 4.0))
    col = r[:, i] / eff[i]
    mean = (col * rc).sum()
    sd = math.sqrt((col * (rc - mean) ** 2).sum())
    assert mean == pytest.approx(tc[i] ** 2 / (tc[i] + 0.01), abs=0.02)
    assert sd == pytest.approx(0.05 * math.sqrt(mean), rel=0.05)


def test_be7_noise_is_one_percent(be7_workload):
    t, x = be7_workload["t_edges"], be7_workload["rec_edges"]
    clean = response_matrix(t, x, res=0.05, kq=0.01).astype(np.float64)
    noisy = be7_workload["R"].astype(np.float64)
    on = clean > 1e-12
    ratio = noisy[on] / clean[on]
    assert np.all(np.abs(ratio - 1.0) <= 0.01 + 1e-5)
    assert ratio.std() == pytest.approx(0.02 / math.sqrt(12.0), rel=0.1)  # U[0.99, 1.01]
    assert be7_workload["theta"].shape == (16, 5)
    np.testing.assert_array_equal(np.unique(be7_workload["theta"][:, 0]), np.linspace(-0.5, 0.5, 4).astype(np.float32))


def test_theta_box_is_seeded_and_bounded():
    a = workloads.theta_box(4096, 3)
    np.testing.assert_array_equal(a, workloads.theta_box(4096, 3))
    assert not np.array_equal(a, workloads.theta_box(4096, 4))
    assert np.all(np.abs(a[:, :4]) <= 0.3) and np.all((a[:, 4] >= 0.0) & (a[:, 4] <= 3.0))
    # uniform: every coordinate fills its range
    assert np.all(a[:, :4].min(axis=0) < -0.29) and np.all(a[:, :4].max(axis=0) > 0.29)
    assert a[:, 4].min() < 0.01 and a[:, 4].max() > 2.99


def test_uneven_configurations_follow_their_ranges():
    gw = workloads.uneven_groups_workload()
    g = gw["groups"]
    assert len(g) == 64 and sum(x["p"] for x in g) == 142_770
    assert all(512 <= x["n_t"] <= 8192 and 256 <= x["n_rec"] <= 4096 and 256 <= x["p"] <= 4096 for x in g)
    assert all(1.0e4 <= x["exposure"] <= 1.0e7 and 0.03 <= x["res"] <= 0.08 for x in g)
    small = workloads.uneven_groups_workload(scale=0.25)["groups"]
    assert all(s["n_t"] == max(8, int(x["n_t"] * 0.25)) for s, x in zip(small, g))
    counts = workloads.load_group_counts(gw)
    assert [c.size for c in counts] == [x["n_rec"] for x in g]
    assert all(np.all(c >= 0) and np.all(c == np.round(c)) for c in counts)


def test_live_time_and_joint_grid():
    t_edges, rec_edges = solar_joint_grid()
    assert t_edges.size == 4097 and rec_edges.size == 2049
    m = live_time(rec_edges)
    assert m[0] == pytest.approx(0.9, abs=1e-3) and m[-1] == pytest.approx(1.0, abs=1e-12)
    assert np.all(np.diff(m) >= 0.0)  # rises monotonically from the floor to 1
    c = 0.5 * (rec_edges[1:] + rec_edges[:-1])
    assert m[np.argmin(np.abs(c - 0.15))] == pytest.approx(0.95, abs=0.01)  # halfway at e_on


def test_stored_pseudo_data_have_the_workload_sizes(solar_workload):
    n = workloads.load_counts(solar_workload["name"])
    assert n.size == 2048 and np.all(n >= 0) and np.all(n == np.round(n))
    # Poisson pseudo-data of 1e5 signal plus 9.45e4 background events (sd 0.23 %)
    assert n.sum() == pytest.approx(1.0e5 + 9.45e4, rel=0.012)
