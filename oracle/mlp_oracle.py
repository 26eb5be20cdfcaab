"""FP64 oracle of the learned surrogate (test infrastructure).

TEST INFRASTRUCTURE: used by the tests, the smoke check and the benchmark's
CPU-baseline leg only; the CUDA library never imports it.

The surrogate maps a parameter point theta to the standardized logarithm of
the expected counts per reconstructed bin:

    x  = (theta - centre) / half_width                (the scan box -> [-1, 1]^5)
    h1 = gelu(W1 x  + b1),  h2 = gelu(W2 h1 + b2),  h3 = gelu(W3 h2 + b3)
    y  = W4 h3 + b4,        log mu_j ~ m_j + s_j y_j

with gelu(z) = z Phi(z) = z/2 (1 + erf(z / sqrt 2)) (the exact, erf form) and
widths 5 -> 256 -> 256 -> 256 -> N_rec.  Training minimises the mean squared
error L = mean_{p, j} (y_pj - t_pj)^2 against standardized targets
t = (log mu - m) / s, with Adam (Kingma & Ba, 2015, Algorithm 1):

    m <- b1 m + (1 - b1) g,   v <- b2 v + (1 - b2) g^2,
    w <- w - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Backpropagation is written out by hand (chain rule through each layer); the
tests check it against central finite differences.
"""

from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def gelu(z):
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * z * (1.0 + erf(z / SQRT2))


def gelu_grad(z):
    """d gelu / dz = Phi(z) + z phi(z)."""
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * (1.0 + erf(z / SQRT2)) + z * INV_SQRT_2PI * np.exp(-0.5 * z * z)


class MLPOracle:
    """The surrogate network in float64.  params: list of (W [out, in], b [out])."""

    def __init__(self, params, centre, half_width):
        self.params = [(np.array(W, dtype=np.float64), np.array(b, dtype=np.float64)) for W, b in params]
        self.centre = np.asarray(centre, dtype=np.float64)
        self.half = np.asarray(half_width, dtype=np.float64)

    def inputs(self, theta):
        return (np.asarray(theta, dtype=np.float64) - self.centre) / self.half

    def forward(self, theta):
        """Returns the output y [B, N] and the cache of pre-activations and activations."""
        a = self.inputs(theta)
        cache = {"a0": a, "z": [], "a": [a]}
        n = len(self.params)
        for k, (W, b) in enumerate(self.params):
            z = a @ W.T + b
            cache["z"].append(z)
            a = gelu(z) if k < n - 1 else z
            cache["a"].append(a)
        return a, cache

    @staticmethod
    def loss(y, t):
        d = np.asarray(y, dtype=np.float64) - np.asarray(t, dtype=np.float64)
        return float(np.mean(d * d))

    def gradients(self, theta, t):
        """Loss and its gradients [(dW, db), ...] by backpropagation."""
        y, cache = self.forward(theta)
        t = np.asarray(t, dtype=np.float64)
        count = y.size
        delta = 2.0 * (y - t) / count                 # dL/dy
        grads = [None] * len(self.params)
        for k in range(len(self.params) - 1, -1, -1):
            W, _ = self.params[k]
            a_in = cache["a"][k]
            grads[k] = (delta.T @ a_in, delta.sum(axis=0))
            if k > 0:
                delta = (delta @ W) * gelu_grad(cache["z"][k - 1])
        return self.loss(y, t), grads


def adam_step(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Algorithm 1 of Kingma & Ba); step counts from 1.
    Returns new (params, m, v) lists of (W, b) pairs."""
    out_p, out_m, out_v = [], [], []
    c1 = 1.0 - beta1 ** step
    c2 = 1.0 - beta2 ** step
    for (W, b), (gW, gb), (mW, mb), (vW, vb) in zip(params, grads, m, v):
        pair_p, pair_m, pair_v = [], [], []
        for w, g, mm, vv in ((W, gW, mW, vW), (b, gb, mb, vb)):
            mm = beta1 * mm + (1.0 - beta1) * g
            vv = beta2 * vv + (1.0 - beta2) * g * g
            w = w - lr * (mm / c1) / (np.sqrt(vv / c2) + eps)
            pair_p.append(w)
            pair_m.append(mm)
            pair_v.append(vv)
        out_p.append(tuple(pair_p))
        out_m.append(tuple(pair_m))
        out_v.append(tuple(pair_v))
    return out_p, out_m, out_v


def standardization(log_mu):
    """Per-bin mean and standard deviation of training targets log mu [P, N]."""
    log_mu = np.asarray(log_mu, dtype=np.float64)
    m = log_mu.mean(axis=0)
    s = log_mu.std(axis=0)
    s = np.where(s > 0.0, s, 1.0)
    return m, s


def surrogate_neg2lnl(y, m, s, counts, c_data):
    """-2 ln L of the surrogate's expected counts mu = exp(m + s y) (eq. logL in
    the deviance form with the data constant c_data)."""
    mu = np.exp(np.asarray(m) + np.asarray(s) * np.asarray(y, dtype=np.float64))
    n = np.asarray(counts, dtype=np.float64)
    t = np.where(n > 0, mu - n + n * np.log(np.where(n > 0, n, 1.0) / mu), mu)
    return 2.0 * t.sum(axis=-1) + c_data


def data_constant(counts):
    """C = 2 sum_j [n_j - n_j ln n_j + ln Gamma(n_j + 1)] (0 ln 0 = 0)."""
    n = np.asarray(counts, dtype=np.float64)
    lg = np.array([math.lgamma(x + 1.0) for x in n])
    return 2.0 * float(np.sum(n - np.where(n > 0, n * np.log(np.where(n > 0, n, 1.0)), 0.0) + lg))
