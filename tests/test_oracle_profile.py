"""Pins of the oracle's profiled signal normalisation (CPU).

* One bin without background: alpha-hat = n / s and the minimum is the data
  constant 2 [n - n ln n + lnGamma(n + 1)] (closed forms).
* Asimov data made with alpha = 1.3: alpha-hat = 1.3 and the minimum is the
  data constant (Gibbs' inequality: -2 ln L is smallest at mu = n).
* A vanishing pull width pins alpha to 1 (the unprofiled value); profiling
  never raises -2 ln L above the unprofiled value.
"""

import math

import numpy as np
import pytest

from oracle.mlp_oracle import data_constant
from oracle.srw_oracle import neg2lnl, profiled_neg2lnl


def test_single_bin_closed_form():
    v, a = profiled_neg2lnl(np.array([4.0]), np.array([0.0]), np.array([10.0]))
    assert a == pytest.approx(2.5, rel=1e-9)
    assert v == pytest.approx(2.0 * (10.0 - 10.0 * math.log(10.0) + math.lgamma(11.0)), rel=1e-12)


def test_asimov_recovers_the_injected_normalisation():
    rng = np.random.default_rng(0)
    sig = rng.uniform(5.0, 50.0, 40)
    bkg = rng.uniform(1.0, 5.0, 40)
    n = 1.3 * sig + bkg
    v, a = profiled_neg2lnl(sig, bkg, n)
    assert a == pytest.approx(1.3, rel=1e-7)
    assert v == pytest.approx(data_constant(n), rel=1e-12, abs=1e-9)


def test_pull_limits():
    rng = np.random.default_rng(1)
    sig = rng.uniform(5.0, 50.0, 30)
    bkg = rng.uniform(1.0, 5.0, 30)
    n = rng.poisson(1.2 * sig + bkg).astype(float)
    free, a_free = profiled_neg2lnl(sig, bkg, n)
    fixed = neg2lnl(sig + bkg, n)
    tight, a_tight = profiled_neg2lnl(sig, bkg, n, sigma_alpha=1e-6)
    loose, a_loose = profiled_neg2lnl(sig, bkg, n, sigma_alpha=0.1)
    assert free <= fixed + 1e-9
    assert a_tight == pytest.approx(1.0, abs=1e-6)
    assert tight == pytest.approx(fixed, rel=1e-9)
    assert free <= loose <= fixed + 1e-9
    assert min(1.0, a_free) - 1e-9 <= a_loose <= max(1.0, a_free) + 1e-9
