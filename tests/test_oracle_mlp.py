"""Pins of the surrogate's FP64 oracle and of the Sobol generator (CPU only).

* GELU against its closed form at special points and its limits.
* Backpropagation against central finite differences of the loss (every
  weight and bias of a small network, rel 1e-6).
* Adam's first step against its closed form: with m0 = v0 = 0 the bias-
  corrected step is -lr g / (|g| + eps), i.e. -lr sign(g) where |g| >> eps.
* Adam minimises a convex quadratic.
* Sobol points against SciPy's unscrambled Sobol (same Joe-Kuo numbers).
"""

import math

import numpy as np
import pytest

from oracle.mlp_oracle import MLPOracle, adam_step, data_constant, gelu, gelu_grad, standardization, \
    surrogate_neg2lnl
from oracle.sobol import direction_numbers, sobol_points
from workloads.mlp import BOX_CENTRE, BOX_HALF, init_weights, layer_shapes, round_to_bf16


def test_gelu_special_values():
    assert gelu(0.0) == 0.0
    assert gelu_grad(0.0) == pytest.approx(0.5, abs=1e-15)
    # Phi(1) = 0.841344746068543 (standard normal table)
    assert gelu(1.0) == pytest.approx(0.841344746068543, rel=1e-14)
    assert gelu(-1.0) == pytest.approx(-(1.0 - 0.841344746068543), rel=1e-13)
    # z Phi(z) -> z for large z, -> 0 for very negative z
    assert gelu(12.0) == pytest.approx(12.0, rel=1e-15)
    assert abs(gelu(-12.0)) < 1e-30
    # derivative by central differences
    z = np.linspace(-4, 4, 17)
    h = 1e-6
    np.testing.assert_allclose(gelu_grad(z), (gelu(z + h) - gelu(z - h)) / (2 * h), rtol=1e-8, atol=1e-10)


def _tiny(seed=0):
    rng = np.random.default_rng(seed)
    dims = [5, 4, 4, 4, 3]
    params = [(rng.normal(size=(dims[k + 1], dims[k])), rng.normal(size=dims[k + 1])) for k in range(4)]
    return MLPOracle(params, BOX_CENTRE, BOX_HALF), rng


def test_backprop_matches_finite_differences():
    net, rng = _tiny()
    theta = BOX_CENTRE + BOX_HALF * rng.uniform(-1, 1, size=(6, 5))
    t = rng.normal(size=(6, 3))
    _, grads = net.gradients(theta, t)
    h = 1e-6
    for k, (W, b) in enumerate(net.params):
        for arr, g in ((W, grads[k][0]), (b, grads[k][1])):
            num = np.zeros_like(arr)
            for idx in np.ndindex(arr.shape):
                keep = arr[idx]
                arr[idx] = keep + h
                lp = net.loss(net.forward(theta)[0], t)
                arr[idx] = keep - h
                lm = net.loss(net.forward(theta)[0], t)
                arr[idx] = keep
                num[idx] = (lp - lm) / (2 * h)
            np.testing.assert_allclose(g, num, rtol=1e-6, atol=1e-9)


def test_dropped_term_would_fail():
    # the check above is sharp: omitting gelu' in the backward pass changes the gradients
    net, rng = _tiny(1)
    theta = BOX_CENTRE + BOX_HALF * rng.uniform(-1, 1, size=(4, 5))
    t = rng.normal(size=(4, 3))
    _, grads = net.gradients(theta, t)
    y, cache = net.forward(theta)
    delta = 2.0 * (y - t) / y.size
    W4 = net.params[3][0]
    wrong = (delta @ W4).T @ cache["a"][2]  # without the gelu' factor
    assert np.max(np.abs(wrong - grads[2][0])) > 1e-3 * np.max(np.abs(grads[2][0]))


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(2)
    W = rng.normal(size=(3, 2))
    b = rng.normal(size=3)
    gW = rng.normal(size=(3, 2))
    gb = rng.normal(size=3)
    zeros = [(np.zeros_like(W), np.zeros_like(b))]
    lr, eps = 1e-3, 1e-8
    p, m, v = adam_step([(W, b)], [(gW, gb)], zeros, zeros, 1, lr, eps=eps)
    np.testing.assert_allclose(p[0][0], W - lr * gW / (np.abs(gW) + eps), rtol=0, atol=1e-15)
    np.testing.assert_allclose(p[0][1], b - lr * gb / (np.abs(gb) + eps), rtol=0, atol=1e-15)
    np.testing.assert_allclose(p[0][1], b - lr * np.sign(gb), rtol=0, atol=lr * eps / np.abs(gb).min() * 2)
    np.testing.assert_allclose(m[0][0], 0.1 * gW)
    np.testing.assert_allclose(v[0][0], 0.001 * gW * gW)


def test_adam_minimises_a_quadratic():
    target = np.array([[0.5, -1.0], [2.0, 0.25]])
    W = np.zeros((2, 2))
    b = np.zeros(2)
    m = [(np.zeros_like(W), np.zeros_like(b))]
    v = [(np.zeros_like(W), np.zeros_like(b))]
    params = [(W, b)]
    for step in range(1, 3001):
        g = [(2 * (params[0][0] - target), 2 * (params[0][1] - 1.0))]
        params, m, v = adam_step(params, g, m, v, step, 1e-2)
    np.testing.assert_allclose(params[0][0], target, atol=1e-3)
    np.testing.assert_allclose(params[0][1], 1.0, atol=1e-3)


def test_surrogate_likelihood_matches_direct_form():
    rng = np.random.default_rng(3)
    n = rng.poisson(20.0, size=50).astype(float)
    n[:3] = 0
    m = rng.normal(3.0, 0.1, size=50)
    s = rng.uniform(0.5, 1.5, size=50)
    y = rng.normal(size=50)
    mu = np.exp(m + s * y)
    direct = 2.0 * np.sum(mu - n * np.log(mu) + np.array([math.lgamma(x + 1) for x in n]))
    assert surrogate_neg2lnl(y, m, s, n, data_constant(n)) == pytest.approx(direct, rel=1e-12)


def test_standardization():
    x = np.array([[1.0, 5.0], [3.0, 5.0]])
    m, s = standardization(x)
    np.testing.assert_allclose(m, [2.0, 5.0])
    np.testing.assert_allclose(s, [1.0, 1.0])  # constant column -> 1


def test_sobol_matches_scipy():
    qmc = pytest.importorskip("scipy.stats.qmc")
    a = sobol_points(0, 2048, 5)
    b = qmc.Sobol(d=5, scramble=False).random(2048)
    assert np.array_equal(a, b)
    eng = qmc.Sobol(d=5, scramble=False)
    eng.fast_forward(123457)
    assert np.array_equal(sobol_points(123457, 64, 5), eng.random(64))


def test_sobol_stratification():
    # the first 2^k points hit every dyadic interval of length 2^-k once, per dimension
    x = sobol_points(0, 256, 5)
    for d in range(5):
        assert sorted(np.floor(x[:, d] * 256).astype(int)) == list(range(256))
    V = direction_numbers(5)
    assert all(int(V[d, 0]) == 1 << 31 for d in range(5))


def test_initial_weights_and_bf16_rounding():
    params = init_weights(2048, seed=5)
    assert [W.shape for W, _ in params] == layer_shapes(2048)
    W1 = params[1][0]
    assert abs(W1.std() - np.sqrt(2.0 / 256)) < 0.01 * np.sqrt(2.0 / 256) * 10
    r = round_to_bf16(np.array([1.0, 1.00390625, 1.005859375, -3.14159], np.float32))
    assert r[0] == 1.0 and r[1] == 1.0  # tie to even
    assert r[2] == np.float32(1.0078125)
    assert abs(r[3] - -3.140625) < 1e-7
