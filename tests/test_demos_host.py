"""Host logic of the Asimov demonstration (Sec. VI): the 90 % CL threshold and
the interval edges of a one-parameter scan, checked against closed forms."""

import statistics

import numpy as np
import pytest

from paper_2607_00488_gb300 import demos


def test_threshold_is_the_one_dof_chi2_quantile():
    # chi^2 with one degree of freedom is the square of a standard normal:
    # P(chi^2 <= q) = 0.90  <=>  q = z_{0.95}^2
    z = statistics.NormalDist().inv_cdf(0.95)
    assert demos.DCHI2_90 == pytest.approx(z * z, rel=1e-12)


def test_piecewise_linear_scan_has_exact_edges():
    # |x - x0| * slope is linear between grid points, so the interpolated
    # crossings are exact
    x0, slope = 0.3, 7.0
    grid = np.linspace(-1.0, 1.0, 201)  # x0 is a grid point
    r = demos.interval(grid, np.abs(grid - x0) * slope + 5.0)
    assert r["argmin"] == pytest.approx(x0)
    assert r["min"] == pytest.approx(5.0)
    assert r["lo"] == pytest.approx(x0 - demos.DCHI2_90 / slope, abs=1e-12)
    assert r["hi"] == pytest.approx(x0 + demos.DCHI2_90 / slope, abs=1e-12)


def test_parabola_edges_are_wilks_interval():
    # ((x - x0) / sigma)^2 crosses min + q at x0 +- sigma sqrt(q); linear
    # interpolation on a grid of step h is off by at most h^2 / (8 sigma^2)
    # in -2 ln L, i.e. O(h^2) in x
    x0, sigma = -0.125, 0.04
    grid = np.linspace(-0.5, 0.5, 4001)
    r = demos.interval(grid, ((grid - x0) / sigma) ** 2)
    half = sigma * np.sqrt(demos.DCHI2_90)
    h = grid[1] - grid[0]
    assert r["lo"] == pytest.approx(x0 - half, abs=h * h / sigma)
    assert r["hi"] == pytest.approx(x0 + half, abs=h * h / sigma)
    # the chord lies above the parabola, so the interpolated edges move inwards
    assert x0 - half < r["lo"] < x0 - half + h
    assert x0 + half - h < r["hi"] < x0 + half


def test_open_sides_and_edge_minimum():
    grid = np.linspace(0.0, 1.0, 11)
    # rises by less than the threshold to the left: no lower edge
    v = (grid - 0.2) ** 2 * 50.0
    r = demos.interval(grid, v)
    assert r["lo"] is None and r["hi"] is not None
    # minimum on the first grid point: no lower edge either
    r = demos.interval(grid, grid * 10.0)
    assert r["argmin"] == 0.0 and r["lo"] is None
    assert r["hi"] == pytest.approx(demos.DCHI2_90 / 10.0)
    # flat scan: neither edge
    r = demos.interval(grid, np.zeros_like(grid))
    assert r["lo"] is None and r["hi"] is None


def test_first_minimum_and_custom_level():
    grid = np.arange(6, dtype=float)
    v = [3.0, 0.0, 1.0, 0.0, 2.0, 9.0]
    r = demos.interval(grid, v, level=1.0)
    assert r["argmin"] == 1.0  # the first of equal minima
    assert r["lo"] == pytest.approx(1.0 - 1.0 / 3.0)
    assert r["hi"] == pytest.approx(2.0)  # reaches the level exactly at a grid point
